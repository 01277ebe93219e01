/*
 * isg_oracle.h -- plain CPU oracle for the checkerboard Metropolis sweep of the
 * 3D Edwards-Anderson +-J spin glass (Lulli, Bernaschi, Parisi, arXiv:1411.0127).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or constant generator with the GPU
 * library; it stores one int8_t per spin and one int8_t per coupling and follows
 * the definitions of the paper and of the generators it names, written out
 * plainly:
 *
 *   Hamiltonian            Sec. 1, Eq. (1)           H = -sum_<ik> J_ik s_i s_k
 *   bimodal disorder       Sec. 1, Eq. (2)           J = +-1 with p = 1/2
 *   checkerboard colours   Sec. 1 (red/blue split)   red first, then blue
 *   Metropolis rule        Sec. 4, Eq. for P_flip    accept if dE <= 0, else
 *                                                    with prob. exp(-beta dE)
 *   integer comparison     Sec. 4 (R vs Rmax exp)    accept if d < thr[dE/4]
 *   MINSTD                 Sec. 3, Eq. for R_{n+1}   R <- 16807 R mod (2^31-1)
 *   MT19937                Sec. 3 (by name)          Matsumoto & Nishimura 1998
 *
 * Where the paper is silent this oracle reads it as follows: red (x+y+z even)
 * is updated first; every attempt consumes one draw, dE <= 0 included; the
 * site -> (stream, draw) map is the row partition of or_rows_per_stream with
 * sites in row order and ascending x; couplings, spins and stream seeds come
 * from the SplitMix64 counter hash; MINSTD's draw is 2x so that one 32-bit
 * threshold table serves every generator; Parisi-Rapuano starts from 61 hashed
 * words with the last one made odd.
 */
#ifndef ISG_ORACLE_H
#define ISG_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { OR_RNG_MINSTD = 0, OR_RNG_MT19937 = 1, OR_RNG_PR = 2 };

typedef struct or_sim or_sim;

/* SplitMix64 (Steele, Lea & Flood 2014): the n-th output (n = 0, 1, ...) of the
 * generator whose state starts at `seed`. */
uint64_t or_splitmix64(uint64_t seed, uint64_t n);

/* Acceptance thresholds thr[k] = floor(2^32 exp(-4 k beta)), k = 1..3; thr[0] is
 * unused (set to 0).  beta = +inf gives 0. */
void or_thresholds(double beta, uint32_t thr[4]);

/* Stream partition of an L^3 lattice: S(L) streams of R(L) consecutive rows. */
int64_t or_rows_per_stream(int L);
int64_t or_num_streams(int L);

/* Raw generator streams (for the generator pins). */
void or_mt19937_outputs(uint32_t seed, uint32_t *out, int64_t n);   /* init_genrand(seed) */
void or_minstd_outputs(uint32_t x0, uint32_t *out, int64_t n);      /* successive states */
/* Parisi-Rapuano (Sec. 3) from the seed word v: ira[j] = SplitMix64(v, j) >> 32
 * for j < 61, ira[60] |= 1; output n is ira[61+n] ^ ira[n]. */
void or_pr_outputs(uint64_t v, uint32_t *out, int64_t n);

/* The initial state one site at a time, as or_create draws it (Eq. (2)):
 * the spin of site i, the coupling J[d][i] (d = 0, 1, 2 for x, y, z), and the
 * 64-bit seed word v_t of RNG stream t (MT19937 is seeded with the low 32 bits
 * of v_t, MINSTD with 1 + v_t mod (2^31 - 2), Parisi-Rapuano with v_t). */
int or_initial_spin(uint64_t seed_spin, int64_t i);
int or_initial_coupling(uint64_t seed_J, int64_t i, int d);
uint64_t or_stream_word(uint64_t seed_rng, int64_t t);

/* Number of unsatisfied bonds around a site (0..6); s, nb[k], J[k] are +-1. */
int or_unsatisfied(int8_t s, const int8_t nb[6], const int8_t J[6]);
/* Metropolis decision for u unsatisfied bonds and a 32-bit draw d: 1 = flip. */
int or_accept(int u, uint32_t d, const uint32_t thr[4]);

/* Simulator.  Returns NULL on a bad argument (L odd, L < 4, bad kind, beta <= 0
 * or NaN) or out of memory. */
or_sim *or_create(int L, uint64_t seed_J, uint64_t seed_spin, double beta, int kind);
/* The same with the RNG streams seeded from seed_rng instead of seed_spin.
 * Sec. 4's asynchronous multispin coding runs 32 samples on one shared draw per
 * site: sample b of such a word follows exactly the trajectory of
 * or_create2(L, seed_J_b, seed_spin_b, seed_rng, ...), because every attempt
 * consumes one draw whatever its outcome (Reading 4). */
or_sim *or_create2(int L, uint64_t seed_J, uint64_t seed_spin, uint64_t seed_rng, double beta, int kind);
void    or_destroy(or_sim *s);
/* n full sweeps (red then blue) using up to nthreads threads; the result does
 * not depend on nthreads. */
void    or_sweep(or_sim *s, int64_t n, int nthreads);
/* One colour pass (c = 0 red, 1 blue) over streams [t0, t1) only: a bounded
 * sample of a sweep, used to time the oracle on large lattices. */
void    or_pass_range(or_sim *s, int c, int64_t t0, int64_t t1, int nthreads);
int64_t or_energy(const or_sim *s);           /* from scratch, Eq. (1) */
int64_t or_tracked_energy(const or_sim *s);   /* initial energy + sum of accepted dE */
int64_t or_overlap(const or_sim *a, const or_sim *b);  /* sum_i s^a_i s^b_i */
uint64_t or_hash(const or_sim *s);            /* Zobrist hash of the +1 spins */
int64_t or_draws_per_stream_done(const or_sim *s, int64_t t);
void    or_get_spins(const or_sim *s, int8_t *out);       /* N values, i = x + L y + L^2 z */
void    or_set_spins(or_sim *s, const int8_t *in);        /* resets the tracked energy */
void    or_get_couplings(const or_sim *s, int8_t *out);   /* 3N values, [d][i], d = x,y,z */
void    or_set_couplings(or_sim *s, const int8_t *in);    /* resets the tracked energy */
/* Per-u tallies of the sweeps so far: attempts[u], accepts[u], u = 0..6. */
void    or_move_counts(const or_sim *s, int64_t attempts[7], int64_t accepts[7]);
/* The next n draws of stream t, without advancing it. */
void    or_peek_draws(const or_sim *s, int64_t t, int64_t n, uint32_t *out);
/* n Metropolis decisions for each u = 0,1,2 with draws from one stream of the
 * given kind and seed word (MT19937: init_genrand(seed); MINSTD: x0 = seed;
 * Parisi-Rapuano: seed word v = seed). */
void    or_acceptance_trial(int kind, uint32_t seed, double beta, int64_t n, int64_t accepts[3]);

#ifdef __cplusplus
}
#endif
#endif
