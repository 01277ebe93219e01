/*
 * isg_oracle.c -- plain CPU oracle (TEST INFRASTRUCTURE ONLY; see isg_oracle.h).
 *
 * Slow and direct on purpose: one int8_t per spin and per coupling, the energy
 * change counted bond by bond, every acceptance decided with the integer
 * comparison of Sec. 4.  Threads split the streams of one colour; sites of one
 * colour only read sites of the other colour (Sec. 1), so the result does not
 * depend on the thread count.
 *
 * Conventions fixed here (the paper leaves them open):
 *   site i = x + L*y + L*L*z, periodic in x, y, z; colour c(i) = (x+y+z) & 1;
 *   colour 0 ("red") is updated first in every sweep.
 *   coupling J[d][i] joins site i and its +d neighbour (d = 0,1,2 for x,y,z).
 *   row r = y + L*z; stream t owns rows [t*R, min((t+1)*R, L*L)).
 *   inside a colour pass a stream visits its rows in order and, inside a row,
 *   the sites of that colour in ascending x; every attempt consumes one draw.
 */
#include "isg_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* SplitMix64, counter form: state_n = seed + (n+1)*gamma, output = mix(state_n) */
uint64_t or_splitmix64(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + (n + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Salts that separate the hash families drawn from one user seed. */
#define SALT_COUPLINGS 0x6A09E667F3BCC908ull
#define SALT_SPINS     0xBB67AE8584CAA73Bull
#define SALT_STREAMS   0x3C6EF372FE94F82Bull
#define SALT_HASH      0xA54FF53A5F1D36F1ull

/* ------------------------------------------------------------------------ */
/* Sec. 4: R < Rmax exp(-beta dE) with Rmax = 2^32, dE = 4k. */
void or_thresholds(double beta, uint32_t thr[4])
{
    thr[0] = 0;
    for (int k = 1; k <= 3; ++k) {
        double v = floor(4294967296.0 * exp(-4.0 * (double)k * beta));
        if (v < 0.0) v = 0.0;
        if (v > 4294967295.0) v = 4294967295.0;
        thr[k] = (uint32_t)v;
    }
}

/* ------------------------------------------------------------------------ */
/* Stream partition: about L^3/2 / 16384 streams (at least 1, at most 8192),
 * each owning R consecutive rows; the last stream may own fewer rows. */
int64_t or_rows_per_stream(int L)
{
    int64_t rows = (int64_t)L * L;
    int64_t s = ((int64_t)L * L * L) / 32768;
    if (s < 1) s = 1;
    if (s > 8192) s = 8192;
    return (rows + s - 1) / s;
}

int64_t or_num_streams(int L)
{
    int64_t rows = (int64_t)L * L, R = or_rows_per_stream(L);
    return (rows + R - 1) / R;
}

/* ------------------------------------------------------------------------ */
/* MT19937 (Matsumoto & Nishimura 1998), kept as the 624-word recurrence
 *   x[k+624] = x[k+397] ^ ((upper(x[k]) | lower(x[k+1])) >> 1) ^ (x[k+1] odd ? A : 0)
 * evaluated one word at a time; output k is the tempered x[k+624]. */
typedef struct {
    uint32_t x[624];
    int i; /* next word to regenerate */
} mt_state;

static void mt_seed(mt_state *m, uint32_t seed)
{
    m->x[0] = seed;
    for (int k = 1; k < 624; ++k)
        m->x[k] = 1812433253u * (m->x[k - 1] ^ (m->x[k - 1] >> 30)) + (uint32_t)k;
    m->i = 0;
}

static uint32_t mt_next(mt_state *m)
{
    int i = m->i, i1 = (i + 1) % 624, im = (i + 397) % 624;
    uint32_t y = (m->x[i] & 0x80000000u) | (m->x[i1] & 0x7FFFFFFFu);
    uint32_t v = m->x[im] ^ (y >> 1) ^ ((y & 1u) ? 0x9908B0DFu : 0u);
    m->x[i] = v;
    m->i = i1;
    v ^= v >> 11;
    v ^= (v << 7) & 0x9D2C5680u;
    v ^= (v << 15) & 0xEFC60000u;
    v ^= v >> 18;
    return v;
}

void or_mt19937_outputs(uint32_t seed, uint32_t *out, int64_t n)
{
    mt_state m;
    mt_seed(&m, seed);
    for (int64_t k = 0; k < n; ++k) out[k] = mt_next(&m);
}

/* MINSTD (Sec. 3): R <- 16807 R mod (2^31 - 1). */
static uint32_t minstd_next(uint32_t *x)
{
    *x = (uint32_t)(((uint64_t)16807u * (uint64_t)(*x)) % 2147483647u);
    return *x;
}

void or_minstd_outputs(uint32_t x0, uint32_t *out, int64_t n)
{
    uint32_t x = x0;
    for (int64_t k = 0; k < n; ++k) out[k] = minstd_next(&x);
}

/* Parisi-Rapuano (Sec. 3): ira[i] = ira[i-24] + ira[i-55] (mod 2^32) and the
 * output is R = ira[i] ^ ira[i-61].  The state is the 61 most recent words,
 * kept as a ring: w[k] is ira[i-61] for the next i, so ira[i-m] sits at
 * w[(k + 61 - m) % 61].  Seeding (the paper gives none): ira[j] = the upper
 * 32 bits of SplitMix64(v, j) for j = 0..60, with ira[60] made odd so that the
 * low bits (a lag-(24, 55) shift register) never start from all zeros; the
 * first output is R for i = 61. */
typedef struct {
    uint32_t w[61];
    int k;
} pr_state;

static void pr_seed(pr_state *p, uint64_t v)
{
    for (int j = 0; j < 61; ++j) p->w[j] = (uint32_t)(or_splitmix64(v, (uint64_t)j) >> 32);
    p->w[60] |= 1u;
    p->k = 0;
}

static uint32_t pr_next(pr_state *p)
{
    int k = p->k;
    uint32_t lag24 = p->w[(k + 61 - 24) % 61];
    uint32_t lag55 = p->w[(k + 61 - 55) % 61];
    uint32_t lag61 = p->w[k];
    uint32_t v = lag24 + lag55;
    p->w[k] = v; /* ira[i] replaces ira[i-61] */
    p->k = (k + 1) % 61;
    return v ^ lag61;
}

void or_pr_outputs(uint64_t v, uint32_t *out, int64_t n)
{
    pr_state p;
    pr_seed(&p, v);
    for (int64_t k = 0; k < n; ++k) out[k] = pr_next(&p);
}

/* One stream: the 32-bit draw d compared with the thresholds.  MT19937 and
 * Parisi-Rapuano give their 32-bit outputs; MINSTD's state (at most 2^31 - 2)
 * is doubled so that every kind is compared with the same 32-bit table. */
typedef struct {
    int kind;
    uint32_t minstd;
    mt_state mt;
    pr_state pr;
    int64_t used; /* draws consumed so far */
} stream_t;

static uint32_t stream_draw(stream_t *st)
{
    st->used++;
    if (st->kind == OR_RNG_MT19937) return mt_next(&st->mt);
    if (st->kind == OR_RNG_PR) return pr_next(&st->pr);
    return minstd_next(&st->minstd) << 1;
}

/* Stream t of a lattice from v_t = SplitMix64(seed_rng ^ K_R, t). */
static void stream_seed(stream_t *st, int kind, uint64_t v)
{
    memset(st, 0, sizeof *st);
    st->kind = kind;
    if (kind == OR_RNG_MT19937) mt_seed(&st->mt, (uint32_t)v);
    else if (kind == OR_RNG_PR) pr_seed(&st->pr, v);
    else st->minstd = 1u + (uint32_t)(v % 2147483646u);
}

/* ------------------------------------------------------------------------ */
int or_initial_spin(uint64_t seed_spin, int64_t i)
{
    return (or_splitmix64(seed_spin ^ SALT_SPINS, (uint64_t)i) >> 63) ? -1 : 1;
}

int or_initial_coupling(uint64_t seed_J, int64_t i, int d)
{
    return (or_splitmix64(seed_J ^ SALT_COUPLINGS, 3 * (uint64_t)i + (uint64_t)d) >> 63) ? -1 : 1;
}

uint64_t or_stream_word(uint64_t seed_rng, int64_t t)
{
    return or_splitmix64(seed_rng ^ SALT_STREAMS, (uint64_t)t);
}

/* ------------------------------------------------------------------------ */
int or_unsatisfied(int8_t s, const int8_t nb[6], const int8_t J[6])
{
    int u = 0;
    for (int k = 0; k < 6; ++k)
        if (J[k] * s * nb[k] == -1) ++u; /* bond energy -J s s' = +1 */
    return u;
}

/* Flipping a site with u unsatisfied bonds changes E by dE = 12 - 4u.
 * dE <= 0 is always accepted; otherwise accept when d < thr[dE/4]. */
int or_accept(int u, uint32_t d, const uint32_t thr[4])
{
    int dE = 12 - 4 * u;
    if (dE <= 0) return 1;
    return d < thr[dE / 4];
}

/* ------------------------------------------------------------------------ */
struct or_sim {
    int L;
    int64_t N;
    int kind;
    double beta;
    uint32_t thr[4];
    int8_t *s;      /* N spins */
    int8_t *J;      /* 3N couplings, J[d*N + i] */
    int64_t R, S;   /* rows per stream, streams */
    stream_t *st;   /* S streams */
    int64_t E0;     /* energy when tracking (re)started */
    int64_t dE;     /* sum of accepted energy changes since then */
    int64_t attempts[7], accepts[7];
};

static inline int64_t idx(int L, int x, int y, int z)
{
    return (int64_t)x + (int64_t)L * y + (int64_t)L * L * z;
}

or_sim *or_create(int L, uint64_t seed_J, uint64_t seed_spin, double beta, int kind)
{
    return or_create2(L, seed_J, seed_spin, seed_spin, beta, kind);
}

or_sim *or_create2(int L, uint64_t seed_J, uint64_t seed_spin, uint64_t seed_rng, double beta, int kind)
{
    if (L < 4 || (L & 1) || L > 2048) return NULL;
    if (!(beta > 0.0)) return NULL; /* rejects 0, negatives and NaN; +inf allowed */
    if (kind != OR_RNG_MINSTD && kind != OR_RNG_MT19937 && kind != OR_RNG_PR) return NULL;
    or_sim *o = (or_sim *)calloc(1, sizeof(or_sim));
    if (!o) return NULL;
    o->L = L;
    o->N = (int64_t)L * L * L;
    o->kind = kind;
    o->beta = beta;
    or_thresholds(beta, o->thr);
    o->s = (int8_t *)malloc((size_t)o->N);
    o->J = (int8_t *)malloc((size_t)(3 * o->N));
    o->R = or_rows_per_stream(L);
    o->S = or_num_streams(L);
    o->st = (stream_t *)calloc((size_t)o->S, sizeof(stream_t));
    if (!o->s || !o->J || !o->st) { or_destroy(o); return NULL; }

    /* Eq. (2): J = +1 or -1 with probability 1/2 each; random +-1 initial spins. */
    for (int64_t i = 0; i < o->N; ++i) {
        for (int d = 0; d < 3; ++d) o->J[d * o->N + i] = (int8_t)or_initial_coupling(seed_J, i, d);
        o->s[i] = (int8_t)or_initial_spin(seed_spin, i);
    }
    for (int64_t t = 0; t < o->S; ++t) stream_seed(&o->st[t], kind, or_stream_word(seed_rng, t));
    o->E0 = or_energy(o);
    o->dE = 0;
    return o;
}

void or_destroy(or_sim *o)
{
    if (!o) return;
    free(o->s);
    free(o->J);
    free(o->st);
    free(o);
}

/* One colour pass of stream t: returns the sum of accepted dE. */
static int64_t stream_pass(or_sim *o, int64_t t, int c, int64_t att[7], int64_t acc[7])
{
    const int L = o->L;
    const int64_t N = o->N;
    const int8_t *Jx = o->J, *Jy = o->J + N, *Jz = o->J + 2 * N;
    int8_t *s = o->s;
    int64_t dE = 0;
    int64_t r_end = (t + 1) * o->R;
    if (r_end > (int64_t)L * L) r_end = (int64_t)L * L;
    for (int64_t r = t * o->R; r < r_end; ++r) {
        int y = (int)(r % L), z = (int)(r / L);
        int yp = (y + 1) % L, ym = (y + L - 1) % L, zp = (z + 1) % L, zm = (z + L - 1) % L;
        for (int x = 0; x < L; ++x) {
            if (((x + y + z) & 1) != c) continue;
            int xp = (x + 1) % L, xm = (x + L - 1) % L;
            int64_t i = idx(L, x, y, z);
            int8_t nb[6], Jb[6];
            nb[0] = s[idx(L, xp, y, z)]; Jb[0] = Jx[i];
            nb[1] = s[idx(L, xm, y, z)]; Jb[1] = Jx[idx(L, xm, y, z)];
            nb[2] = s[idx(L, x, yp, z)]; Jb[2] = Jy[i];
            nb[3] = s[idx(L, x, ym, z)]; Jb[3] = Jy[idx(L, x, ym, z)];
            nb[4] = s[idx(L, x, y, zp)]; Jb[4] = Jz[i];
            nb[5] = s[idx(L, x, y, zm)]; Jb[5] = Jz[idx(L, x, y, zm)];
            uint32_t d = stream_draw(&o->st[t]);
            int u = or_unsatisfied(s[i], nb, Jb);
            att[u]++;
            if (or_accept(u, d, o->thr)) {
                s[i] = (int8_t)(-s[i]);
                dE += 12 - 4 * u;
                acc[u]++;
            }
        }
    }
    return dE;
}

typedef struct {
    or_sim *o;
    int c;
    int64_t t0, t1;
    int64_t dE;
    int64_t att[7], acc[7];
} pass_job;

static void *pass_worker(void *arg)
{
    pass_job *j = (pass_job *)arg;
    j->dE = 0;
    memset(j->att, 0, sizeof j->att);
    memset(j->acc, 0, sizeof j->acc);
    for (int64_t t = j->t0; t < j->t1; ++t) j->dE += stream_pass(j->o, t, j->c, j->att, j->acc);
    return NULL;
}

static void colour_pass(or_sim *o, int c, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > o->S) nthreads = (int)o->S;
    if (nthreads == 1) {
        for (int64_t t = 0; t < o->S; ++t) o->dE += stream_pass(o, t, c, o->attempts, o->accepts);
        return;
    }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    pass_job *jobs = (pass_job *)malloc(sizeof(pass_job) * (size_t)nthreads);
    int started = 0;
    for (int k = 0; k < nthreads; ++k) {
        jobs[k].o = o;
        jobs[k].c = c;
        jobs[k].t0 = o->S * k / nthreads;
        jobs[k].t1 = o->S * (k + 1) / nthreads;
        if (pthread_create(&th[k], NULL, pass_worker, &jobs[k]) == 0) started = k + 1;
        else { pass_worker(&jobs[k]); th[k] = 0; }
    }
    for (int k = 0; k < nthreads; ++k) {
        if (k < started && th[k]) pthread_join(th[k], NULL);
        o->dE += jobs[k].dE;
        for (int u = 0; u < 7; ++u) {
            o->attempts[u] += jobs[k].att[u];
            o->accepts[u] += jobs[k].acc[u];
        }
    }
    free(th);
    free(jobs);
}

void or_pass_range(or_sim *o, int c, int64_t t0, int64_t t1, int nthreads)
{
    if (t0 < 0) t0 = 0;
    if (t1 > o->S) t1 = o->S;
    if (t1 <= t0) return;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > t1 - t0) nthreads = (int)(t1 - t0);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    pass_job *jobs = (pass_job *)malloc(sizeof(pass_job) * (size_t)nthreads);
    for (int k = 0; k < nthreads; ++k) {
        jobs[k].o = o;
        jobs[k].c = c;
        jobs[k].t0 = t0 + (t1 - t0) * k / nthreads;
        jobs[k].t1 = t0 + (t1 - t0) * (k + 1) / nthreads;
        if (pthread_create(&th[k], NULL, pass_worker, &jobs[k]) != 0) { pass_worker(&jobs[k]); th[k] = 0; }
    }
    for (int k = 0; k < nthreads; ++k) {
        if (th[k]) pthread_join(th[k], NULL);
        o->dE += jobs[k].dE;
        for (int u = 0; u < 7; ++u) {
            o->attempts[u] += jobs[k].att[u];
            o->accepts[u] += jobs[k].acc[u];
        }
    }
    free(th);
    free(jobs);
}

void or_sweep(or_sim *o, int64_t n, int nthreads)
{
    for (int64_t k = 0; k < n; ++k) {
        colour_pass(o, 0, nthreads); /* red */
        colour_pass(o, 1, nthreads); /* blue */
    }
}

/* ------------------------------------------------------------------------ */
int64_t or_energy(const or_sim *o)
{
    const int L = o->L;
    const int64_t N = o->N;
    int64_t E = 0;
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int64_t i = idx(L, x, y, z);
                E -= o->J[i] * o->s[i] * o->s[idx(L, (x + 1) % L, y, z)];
                E -= o->J[N + i] * o->s[i] * o->s[idx(L, x, (y + 1) % L, z)];
                E -= o->J[2 * N + i] * o->s[i] * o->s[idx(L, x, y, (z + 1) % L)];
            }
    return E;
}

int64_t or_tracked_energy(const or_sim *o) { return o->E0 + o->dE; }

int64_t or_overlap(const or_sim *a, const or_sim *b)
{
    if (a->N != b->N) return 0;
    int64_t q = 0;
    for (int64_t i = 0; i < a->N; ++i) q += a->s[i] * b->s[i];
    return q;
}

uint64_t or_hash(const or_sim *o)
{
    uint64_t h = 0;
    for (int64_t i = 0; i < o->N; ++i)
        if (o->s[i] == 1) h ^= or_splitmix64(SALT_HASH, (uint64_t)i);
    return h;
}

int64_t or_draws_per_stream_done(const or_sim *o, int64_t t)
{
    return (t >= 0 && t < o->S) ? o->st[t].used : -1;
}

void or_get_spins(const or_sim *o, int8_t *out) { memcpy(out, o->s, (size_t)o->N); }

void or_set_spins(or_sim *o, const int8_t *in)
{
    memcpy(o->s, in, (size_t)o->N);
    o->E0 = or_energy(o);
    o->dE = 0;
}

void or_get_couplings(const or_sim *o, int8_t *out) { memcpy(out, o->J, (size_t)(3 * o->N)); }

void or_set_couplings(or_sim *o, const int8_t *in)
{
    memcpy(o->J, in, (size_t)(3 * o->N));
    o->E0 = or_energy(o);
    o->dE = 0;
}

void or_move_counts(const or_sim *o, int64_t attempts[7], int64_t accepts[7])
{
    for (int u = 0; u < 7; ++u) {
        attempts[u] = o->attempts[u];
        accepts[u] = o->accepts[u];
    }
}

void or_peek_draws(const or_sim *o, int64_t t, int64_t n, uint32_t *out)
{
    if (t < 0 || t >= o->S) return;
    stream_t copy = o->st[t];
    for (int64_t k = 0; k < n; ++k) out[k] = stream_draw(&copy);
}

void or_acceptance_trial(int kind, uint32_t seed, double beta, int64_t n, int64_t accepts[3])
{
    uint32_t thr[4];
    stream_t st;
    memset(&st, 0, sizeof st);
    st.kind = kind;
    if (kind == OR_RNG_MT19937) mt_seed(&st.mt, seed);
    else if (kind == OR_RNG_PR) pr_seed(&st.pr, seed);
    else st.minstd = seed;
    or_thresholds(beta, thr);
    for (int u = 0; u < 3; ++u) {
        accepts[u] = 0;
        for (int64_t k = 0; k < n; ++k) accepts[u] += or_accept(u, stream_draw(&st), thr);
    }
}
