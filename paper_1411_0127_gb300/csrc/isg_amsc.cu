// isg_amsc.cu -- asynchronous multispin coding (Sec. 4): 32 disorder samples of
// one size L stored bit-parallel, bit b of every word belonging to sample b,
// all updated with ONE shared draw per site.
//
// The paper's scheme: the spins of different samples at the same vertex share a
// word, and one random number serves the whole word: cond_k = -(R < EXP_k) is
// all ones or all zeros (Sec. 4), and the mask is applied with one XOR.  Here:
//   * planes: per colour c, S_c, Jx_c, Jy_c, Jz_c, one 32-bit word per site of
//     that colour, row r = y + L*z holding the L/2 sites x = 2h + ((c+y+z) & 1)
//     at words r*(L/2) + h;
//   * draws: the map of the single-sample engine (streams of R(L) rows, sites
//     visited in row order and ascending x, one draw per site and colour
//     pass), seeded from seed_rng; so sample b follows exactly the
//     trajectory of a lone lattice with (seed_J[b], seed_spin[b], seed_rng);
//   * a lane takes a site's draw, loads the site word and the twelve neighbour
//     and coupling words, counts unsatisfied bonds of the 32 samples with the
//     bit-sliced adder, and flips with the broadcast masks; rows of a multiple
//     of 128 sites take the chunked form (four consecutive sites per lane,
//     16-byte loads, the next chunk's loads in flight), other sizes the
//     site-strided form (sites l, l + 32, ... of the stream per lane).
#include <new>

#include "isg_stream.cuh"

struct isg_amsc {
    int L = 0, half = 0, kind = 0;
    double beta = 0.0;
    uint32_t thr[4] = {0, 0, 0, 0};
    uint64_t seed_rng = 0;
    uint64_t seed_J[32] = {}, seed_spin[32] = {};
    int64_t rows = 0, R = 0, S = 0, plane_words = 0;
    uint32_t* planes = nullptr;         // 8 planes of plane_words words: index 4*c + q
    uint32_t* rng = nullptr;
    uint32_t* rng_pos = nullptr;
    unsigned long long* ctr = nullptr;  // [0] stream tickets, [1..32] energy counters
    unsigned long long tickets = 0;
    int64_t sweeps = 0;
};

namespace isg {

constexpr int kAmscWarps = 4;
constexpr int kAmscSlack = 1024;
constexpr int64_t kAmscDeepStreamsPerSM = 16;  // below: 8 blocks of sites in flight per warp

struct AmscArgs {
    uint32_t* planes;
    int64_t plane_words;
    int L, half, c;
    int64_t R, S, rows;
    uint32_t cmp1, cmp2, cmp3;
};

struct AmscSeeds {
    uint64_t J[32], S[32];
};

// The planes of one colour pass: the updated colour's spins (read and written,
// each word by one lane only) and the seven read-only planes.
struct AmscPtrs {
    uint32_t* Sc;
    const uint32_t *Jxc, *Jyc, *Jzc, *Sn, *Jxn, *Jyn, *Jzn;
};

__device__ __forceinline__ AmscPtrs amsc_ptrs(const AmscArgs& a) {
    const int c = a.c, n = c ^ 1;
    const int64_t pw = a.plane_words;
    AmscPtrs P;
    P.Sc = a.planes + (4 * c) * pw;
    P.Jxc = a.planes + (4 * c + 1) * pw;
    P.Jyc = a.planes + (4 * c + 2) * pw;
    P.Jzc = a.planes + (4 * c + 3) * pw;
    P.Sn = a.planes + (4 * n) * pw;
    P.Jxn = a.planes + (4 * n + 1) * pw;
    P.Jyn = a.planes + (4 * n + 2) * pw;
    P.Jzn = a.planes + (4 * n + 3) * pw;
    return P;
}

// Lane position inside the stream's site sequence (row-major, one draw each).
struct SitePos {
    int r, h, y, z;  // row r = y + L z of the site, its position in the row
};

__device__ __forceinline__ void advance(SitePos& q, int by, int half, int L) {
    q.h += by;
    while (q.h >= half) {
        q.h -= half;
        ++q.r;
        if (++q.y == L) {
            q.y = 0;
            ++q.z;
        }
    }
}

// The words one site update reads: its spin word and forward couplings, and
// for each of the six bonds the neighbour's spin word (backward couplings from
// the other colour's planes at the -x, -y, -z neighbour).  Offsets fit in 32
// bits (a plane has at most 1024^2 * 512 words).
struct SiteIn {
    int o;
    uint32_t s, jxp, jyp, jzp, sxp, sxm, jxm, syp, sym, jym, szp, szm, jzm;
};

__device__ __forceinline__ void site_load(const AmscPtrs& P, int L, int half, int c, const SitePos& q, SiteIn& w) {
    const int p = (c + q.y + q.z) & 1;
    const int rh = q.r * half;
    const int o = rh + q.h;
    const int dym = (q.y == 0 ? L - 1 : -1) * half, dyp = (q.y == L - 1 ? 1 - L : 1) * half;
    const int Lh = L * half;
    const int dzm = q.z == 0 ? (L - 1) * Lh : -Lh, dzp = q.z == L - 1 ? -(L - 1) * Lh : Lh;
    // the x neighbour that is not at the same h: h - 1 for p = 0, h + 1 for p = 1
    const int hs = p == 0 ? (q.h == 0 ? half - 1 : q.h - 1) : (q.h == half - 1 ? 0 : q.h + 1);
    const int os = rh + hs;
    w.o = o;
    w.s = P.Sc[o];
    w.jxp = __ldg(P.Jxc + o);
    w.jyp = __ldg(P.Jyc + o);
    w.jzp = __ldg(P.Jzc + o);
    const uint32_t na = __ldg(P.Sn + o), ns = __ldg(P.Sn + os);
    w.sxp = p == 0 ? na : ns;
    w.sxm = p == 0 ? ns : na;
    w.jxm = __ldg(P.Jxn + (p == 0 ? os : o));
    w.syp = __ldg(P.Sn + o + dyp);
    w.sym = __ldg(P.Sn + o + dym);
    w.jym = __ldg(P.Jyn + o + dym);
    w.szp = __ldg(P.Sn + o + dzp);
    w.szm = __ldg(P.Sn + o + dzm);
    w.jzm = __ldg(P.Jzn + o + dzm);
}

// Sec. 4: e = J ^ s ^ s' per bond, u = sum of the six e (bit-sliced), and the
// draw's comparisons broadcast to all 32 systems as all-ones / all-zeros masks.
__device__ __forceinline__ void site_flip(uint32_t* Sc, const SiteIn& w, uint32_t d, const AmscArgs& a) {
    const uint32_t s = w.s;
    uint32_t u0, u1, u2;
    Logic<uint32_t>::count6(w.jxp ^ s ^ w.sxp, w.jxm ^ s ^ w.sxm, w.jyp ^ s ^ w.syp, w.jym ^ s ^ w.sym,
                            w.jzp ^ s ^ w.szp, w.jzm ^ s ^ w.szm, u0, u1, u2);
    const uint32_t c4 = d < a.cmp1 ? ~0u : 0u, c8 = d < a.cmp2 ? ~0u : 0u, c12 = d < a.cmp3 ? ~0u : 0u;
    Sc[w.o] = s ^ Logic<uint32_t>::flip(u0, u1, u2, c4, c8, c12);
}

// One warp per stream; lane l updates the sites l, l + 32, ... of the stream's
// sequence with the draws of the same index.  NB blocks of 32 sites at a time:
// the NB sites' loads are issued before the draws are made and the flips
// applied, so each lane has 13 NB independent loads in flight.  NB = 4 where
// HBM binds (many streams); NB = 8 for ensembles with fewer than 16 streams per
// SM, where each warp's memory latency binds.
template <int KIND, int NB>
__global__ void __launch_bounds__(kAmscWarps * 32) amsc_kernel(AmscArgs a, FlipArgs gen, StreamConst k,
                                                               unsigned long long* tickets,
                                                               unsigned long long base) {
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* B = smem + wid * (KIND == ISG_RNG_MT19937 ? mt_window(kAmscSlack) : 0);
    const int half = a.half, L = a.L, c = a.c;
    const AmscPtrs P = amsc_ptrs(a);
    for (;;) {
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(tickets, 1ull);
        v = __shfl_sync(kFull, v, 0);
        const int64_t t = (int64_t)(v - base);
        if (t >= a.S) break;
        StreamRegs st;
        load_stream<KIND>(gen, t, B, st, k, lane);
        const int64_t r0 = t * a.R;
        const int64_t r1 = r0 + a.R < a.rows ? r0 + a.R : a.rows;
        const int64_t D = (r1 - r0) * half;
        SitePos q;
        {
            const int rl = lane / half;
            q.r = (int)r0 + rl;
            q.h = lane - rl * half;
            q.y = q.r % L;
            q.z = q.r / L;
        }
        int64_t done = 0;
        for (; done + 32 * NB <= D; done += 32 * NB) {
            SiteIn w[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                site_load(P, L, half, c, q, w[j]);
                advance(q, 32, half, L);
            }
            uint32_t d[NB];
            if (KIND == ISG_RNG_MT19937) {
#pragma unroll
                for (int j = 0; j < NB; j += 4) mt_quad<kAmscSlack>(B, st.iA, d + j, k.mul, lane);
            } else if (KIND == ISG_RNG_PARISI_RAPUANO) {
#pragma unroll
                for (int j = 0; j < NB; ++j) d[j] = pr_warp_step(st.xA, st.xB, lane, 32);
            } else {
                // lane l holds draws n+l+1 (xA) and n+l+33 (xB); 16807^64 steps both by 64
                d[0] = st.xA;
                d[1] = st.xB;
#pragma unroll
                for (int j = 2; j < NB; ++j) d[j] = minstd_mulmod(d[j - 2], k.a64);
                st.xA = minstd_mulmod(d[NB - 2], k.a64);
                st.xB = minstd_mulmod(d[NB - 1], k.a64);
            }
#pragma unroll
            for (int j = 0; j < NB; ++j) site_flip(P.Sc, w[j], d[j], a);
        }
        for (; done < D; done += 32) {
            const int nvalid = D - done < 32 ? (int)(D - done) : 32;
            uint32_t d;
            if (KIND == ISG_RNG_MT19937) {
                d = mt_single<kAmscSlack>(B, st.iA, lane, nvalid, k.mul);
            } else if (KIND == ISG_RNG_PARISI_RAPUANO) {
                d = pr_warp_step(st.xA, st.xB, lane, nvalid);
            } else {
                d = st.xA;
                const int src = lane + nvalid;
                const uint32_t pa = __shfl_sync(kFull, st.xA, src & 31);
                const uint32_t pb = __shfl_sync(kFull, st.xB, src & 31);
                st.xA = src < 32 ? pa : pb;
                st.xB = minstd_mulmod(st.xA, k.a32);
            }
            if (lane < nvalid) {
                SiteIn w;
                site_load(P, L, half, c, q, w);
                site_flip(P.Sc, w, d, a);
            }
            advance(q, 32, half, L);
        }
        if (KIND == ISG_RNG_MT19937) st.pos = (int)((st.pos + D) % kMtN);
        store_stream<KIND>(gen, t, B, st, lane);
    }
}

// ---------------------------------------------------------------------------
// Chunked forms for lattices whose rows hold a multiple of 128 sites per
// colour (L a multiple of 256).  A warp still owns one stream at a time and
// makes its draws 128 at a time in stream order (block j, lane l: site 32j + l
// of the chunk), but lane l updates the four consecutive sites h0+4l ..
// h0+4l+3 of the chunk, so every plane segment the chunk needs is one 16-byte
// access per lane:
//   S_c, Jx_c, Jy_c, Jz_c of the chunk's sites (the spins read and written);
//   S_n and Jx_n of the same row (the x neighbours and the -x coupling at h);
//   S_n of rows y+1 and y-1, Jy_n of row y-1; S_n of rows z+1 and z-1, Jz_n of
//   row z-1;
// and one halo word of S_n (and, for p = 0, of Jx_n) next to the chunk on the
// side of the row's shifted x neighbour: h0-1 when p = 0, h0+128 when p = 1,
// wrapping around the row.  Each lane takes its four sites' levels out of the
// warp-wide ballots of the four blocks of draws.  The next chunk's words are
// loaded into registers (two buffers) before the current chunk's draws are
// made, so every lane keeps twelve 16-byte loads in flight while it computes.
constexpr int kChunk = 128;  // sites per chunk (4 per lane)

// Position of a chunk: row r = y + L z, first site h0.
struct RowCursor {
    int r, h0, y, z;
};

__device__ __forceinline__ RowCursor cursor_at(const AmscArgs& a, int64_t r0) {
    RowCursor c;
    c.r = (int)r0;
    c.h0 = 0;
    c.y = c.r % a.L;
    c.z = c.r / a.L;
    return c;
}

__device__ __forceinline__ void cursor_next(RowCursor& c, int half, int L) {
    c.h0 += kChunk;
    if (c.h0 == half) {
        c.h0 = 0;
        ++c.r;
        if (++c.y == L) {
            c.y = 0;
            ++c.z;
        }
    }
}

// Word offsets (within a plane) of a chunk's rows and of its halo word.
struct ChunkOffs {
    int o, yp, ym, zp, zm, halo, p;
};

__device__ __forceinline__ ChunkOffs chunk_offs(const AmscArgs& a, const RowCursor& c) {
    const int half = a.half, L = a.L;
    ChunkOffs q;
    q.o = c.r * half + c.h0;
    q.yp = q.o + (c.y == L - 1 ? 1 - L : 1) * half;
    q.ym = q.o + (c.y == 0 ? L - 1 : -1) * half;
    const int Lh = L * half;
    q.zp = q.o + (c.z == L - 1 ? -(L - 1) * Lh : Lh);
    q.zm = q.o + (c.z == 0 ? (L - 1) * Lh : -Lh);
    q.p = (a.c + c.y + c.z) & 1;
    q.halo = c.r * half + (q.p == 0 ? (c.h0 == 0 ? half - 1 : c.h0 - 1) : (c.h0 + kChunk == half ? 0 : c.h0 + kChunk));
    return q;
}

// A chunk's words as one lane sees them.
struct ChunkData {
    uint4 s, jx, jy, jz, na, jxn, syp, sym, jym, szp, szm, jzm;
    uint32_t hs, hj;  // halo words of S_n and Jx_n (meaningful in the edge lane only)
    int o, p;
};

__device__ __forceinline__ uint4 ldg4(const uint32_t* p) { return __ldg((const uint4*)p); }

__device__ __forceinline__ void chunk_load(const AmscPtrs& P, const ChunkOffs& q, int lane, ChunkData& d) {
    const int l4 = 4 * lane;
    d.s = *(const uint4*)(P.Sc + q.o + l4);  // read here and written back by this lane only
    d.jx = ldg4(P.Jxc + q.o + l4);
    d.jy = ldg4(P.Jyc + q.o + l4);
    d.jz = ldg4(P.Jzc + q.o + l4);
    d.na = ldg4(P.Sn + q.o + l4);
    d.jxn = ldg4(P.Jxn + q.o + l4);
    d.syp = ldg4(P.Sn + q.yp + l4);
    d.sym = ldg4(P.Sn + q.ym + l4);
    d.jym = ldg4(P.Jyn + q.ym + l4);
    d.szp = ldg4(P.Sn + q.zp + l4);
    d.szm = ldg4(P.Sn + q.zm + l4);
    d.jzm = ldg4(P.Jzn + q.zm + l4);
    const bool edge = lane == (q.p == 0 ? 0 : 31);
    d.hs = edge ? __ldg(P.Sn + q.halo) : 0u;
    d.hj = edge && q.p == 0 ? __ldg(P.Jxn + q.halo) : 0u;
    d.o = q.o;
    d.p = q.p;
}

__device__ __forceinline__ uint32_t comp(const uint4& v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w)); }

// all ones if bit i of v is set, else zero
__device__ __forceinline__ uint32_t bitmask(uint32_t v, int i) { return (uint32_t)((int32_t)(v << (31 - i)) >> 31); }

// Updates the lane's four sites of a chunk (parity P) with the levels of their
// draws (lo4 / hi4: bits 4l..4l+3 of the chunk's lo / hi ballot streams) and
// writes them back with one 16-byte store.  A site flips when u + level >= 3
// (Sec. 4 with dE = 12 - 4u: u >= 3 always, u = 2 when d < thr1, u = 1 when
// d < thr2, u = 0 when d < thr3).
template <int P>
__device__ __forceinline__ void chunk_update(const ChunkData& d, uint32_t* Sc, uint32_t lo4, uint32_t hi4, int lane) {
    // the shifted x neighbour (and, for p = 0, the -x coupling) of the lane's
    // edge site comes from the next lane over, or the halo at the chunk's edge
    uint32_t edge_s, edge_j = 0;
    if (P == 0) {
        edge_s = __shfl_up_sync(kFull, d.na.w, 1);
        edge_j = __shfl_up_sync(kFull, d.jxn.w, 1);
        if (lane == 0) {
            edge_s = d.hs;
            edge_j = d.hj;
        }
    } else {
        edge_s = __shfl_down_sync(kFull, d.na.x, 1);
        if (lane == 31) edge_s = d.hs;
    }
    const uint32_t L4 = lo4 | hi4, L8 = hi4, L12 = lo4 & hi4;
    uint32_t out[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t sv = comp(d.s, i), nav = comp(d.na, i);
        uint32_t ns, jxm;
        if (P == 0) {
            ns = i == 0 ? edge_s : comp(d.na, i - 1);
            jxm = i == 0 ? edge_j : comp(d.jxn, i - 1);
        } else {
            ns = i == 3 ? edge_s : comp(d.na, i + 1);
            jxm = comp(d.jxn, i);
        }
        const uint32_t sxp = P == 0 ? nav : ns, sxm = P == 0 ? ns : nav;
        uint32_t u0, u1, u2;
        Logic<uint32_t>::count6(comp(d.jx, i) ^ sv ^ sxp, jxm ^ sv ^ sxm, comp(d.jy, i) ^ sv ^ comp(d.syp, i),
                                comp(d.jym, i) ^ sv ^ comp(d.sym, i), comp(d.jz, i) ^ sv ^ comp(d.szp, i),
                                comp(d.jzm, i) ^ sv ^ comp(d.szm, i), u0, u1, u2);
        // u + level >= 3, level = c4 + c8 + c12 as all-ones / all-zeros masks
        const uint32_t c4 = bitmask(L4, i), c8 = bitmask(L8, i), c12 = bitmask(L12, i);
        out[i] = sv ^ (u2 | (u1 & (u0 | c4)) | (u0 & c8) | c12);
    }
    *(uint4*)(Sc + d.o + 4 * lane) = make_uint4(out[0], out[1], out[2], out[3]);
}

// The chunk's 128 draws in stream order and each lane's four levels.
template <int KIND>
__device__ __forceinline__ void chunk_levels(uint32_t* B, StreamRegs& st, const StreamConst& k, const Cmp& cm,
                                             int lane, uint32_t& lo4, uint32_t& hi4) {
    uint32_t d[4];
    if (KIND == ISG_RNG_MT19937) {
        mt_quad<kAmscSlack>(B, st.iA, d, k.mul, lane);
    } else if (KIND == ISG_RNG_PARISI_RAPUANO) {
#pragma unroll
        for (int j = 0; j < 4; ++j) d[j] = pr_warp_step(st.xA, st.xB, lane, 32);
    } else {
        d[0] = st.xA;
        d[1] = st.xB;
        d[2] = minstd_mulmod(st.xA, k.a64);
        d[3] = minstd_mulmod(st.xB, k.a64);
        st.xA = minstd_mulmod(d[2], k.a64);
        st.xB = minstd_mulmod(d[3], k.a64);
    }
    uint32_t lo[4], hi[4];
    const uint32_t dmin = min(min(d[0], d[1]), min(d[2], d[3]));
    if (__any_sync(kFull, dmin < cm.c2)) {
        level_ballots<4>(d, cm, lo, hi);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            lo[j] = __ballot_sync(kFull, d[j] < cm.c1);
            hi[j] = 0u;
        }
    }
    // site 4l + i of the chunk is bit 4(l & 7) + i of block l >> 3
    const int jsel = lane >> 3, sh = 4 * (lane & 7);
    const uint32_t lw = jsel == 0 ? lo[0] : (jsel == 1 ? lo[1] : (jsel == 2 ? lo[2] : lo[3]));
    const uint32_t hw = jsel == 0 ? hi[0] : (jsel == 1 ? hi[1] : (jsel == 2 ? hi[2] : hi[3]));
    lo4 = (lw >> sh) & 15u;
    hi4 = (hw >> sh) & 15u;
}

__device__ __forceinline__ void chunk_process(const ChunkData& d, uint32_t* Sc, uint32_t lo4, uint32_t hi4, int lane) {
    if (d.p == 0) chunk_update<0>(d, Sc, lo4, hi4, lane);
    else chunk_update<1>(d, Sc, lo4, hi4, lane);
}

// Chunk n + 1's words are loaded (two buffers, A and B) before chunk n's draws
// are made and its sites updated.
template <int KIND>
__global__ void __launch_bounds__(kAmscWarps * 32) amsc_chunk_kernel(AmscArgs a, FlipArgs gen, StreamConst k,
                                                                     unsigned long long* tickets,
                                                                     unsigned long long base) {
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* B = smem + wid * (KIND == ISG_RNG_MT19937 ? mt_window(kAmscSlack) : 0);
    const AmscPtrs P = amsc_ptrs(a);
    const Cmp cm{a.cmp1, a.cmp2, a.cmp3};
    const int half = a.half, L = a.L;
    for (;;) {
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(tickets, 1ull);
        v = __shfl_sync(kFull, v, 0);
        const int64_t t = (int64_t)(v - base);
        if (t >= a.S) break;
        StreamRegs st;
        load_stream<KIND>(gen, t, B, st, k, lane);
        const int64_t r0 = t * a.R;
        const int64_t r1 = r0 + a.R < a.rows ? r0 + a.R : a.rows;
        const int64_t D = (r1 - r0) * half;
        const int nch = (int)(D / kChunk);
        RowCursor cur = cursor_at(a, r0);
        ChunkData dA, dB;
        chunk_load(P, chunk_offs(a, cur), lane, dA);
        for (int n = 0; n < nch; n += 2) {
            if (n + 1 < nch) {
                cursor_next(cur, half, L);
                chunk_load(P, chunk_offs(a, cur), lane, dB);
            }
            uint32_t lo4, hi4;
            chunk_levels<KIND>(B, st, k, cm, lane, lo4, hi4);
            chunk_process(dA, P.Sc, lo4, hi4, lane);
            if (n + 1 >= nch) break;
            if (n + 2 < nch) {
                cursor_next(cur, half, L);
                chunk_load(P, chunk_offs(a, cur), lane, dA);
            }
            chunk_levels<KIND>(B, st, k, cm, lane, lo4, hi4);
            chunk_process(dB, P.Sc, lo4, hi4, lane);
        }
        if (KIND == ISG_RNG_MT19937) st.pos = (int)((st.pos + D) % kMtN);
        store_stream<KIND>(gen, t, B, st, lane);
    }
}

// Planes from the counter hash: bit b of the site word of sample b (Eq. 2).
__global__ void amsc_init_kernel(uint32_t* planes, int64_t plane_words, int L, int half, AmscSeeds sd) {
    const int64_t rows = (int64_t)L * L;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < 2 * plane_words;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int c = w >= plane_words;
        const int64_t o = w - c * plane_words;
        const int64_t r = o / half;
        const int h = (int)(o - r * half);
        if (r >= rows) continue;
        const int y = (int)(r % L), z = (int)(r / L);
        const uint64_t i = (uint64_t)(2 * h + ((c + y + z) & 1)) + (uint64_t)L * y + (uint64_t)L * L * z;
        uint32_t ws = 0, wx = 0, wy = 0, wz = 0;
        for (int b = 0; b < 32; ++b) {
            const uint32_t bit = 1u << b;
            if (!(splitmix64(sd.S[b] ^ kSaltSpins, i) >> 63)) ws |= bit;
            if (splitmix64(sd.J[b] ^ kSaltCouplings, 3 * i + 0) >> 63) wx |= bit;
            if (splitmix64(sd.J[b] ^ kSaltCouplings, 3 * i + 1) >> 63) wy |= bit;
            if (splitmix64(sd.J[b] ^ kSaltCouplings, 3 * i + 2) >> 63) wz |= bit;
        }
        planes[(4 * c + 0) * plane_words + o] = ws;
        planes[(4 * c + 1) * plane_words + o] = wx;
        planes[(4 * c + 2) * plane_words + o] = wy;
        planes[(4 * c + 3) * plane_words + o] = wz;
    }
}

// Per-sample count of unsatisfied bonds: the three forward bonds of every site
// of both colours, added bit-parallel into 16-bit vertical counters (bit b of
// counter plane j = bit j of sample b's count), flushed per thread.
__global__ void amsc_unsat_kernel(const uint32_t* planes, int64_t plane_words, int L, int half,
                                  unsigned long long* counts) {
    __shared__ unsigned long long sc[32];
    if (threadIdx.x < 32) sc[threadIdx.x] = 0;
    __syncthreads();
    uint32_t cnt[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) cnt[j] = 0;
    const int64_t rows = (int64_t)L * L;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < 2 * plane_words;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int c = w >= plane_words;
        const int64_t o = w - c * plane_words;
        const int64_t r = o / half;
        const int h = (int)(o - r * half);
        if (r >= rows) continue;
        const int y = (int)(r % L), z = (int)(r / L);
        const int p = (c + y + z) & 1, n = c ^ 1;
        const uint32_t* Sn = planes + (4 * n) * plane_words;
        const uint32_t s = planes[(4 * c) * plane_words + o];
        const int hx = p == 0 ? h : (h == half - 1 ? 0 : h + 1);   // site x + 1 in the other colour
        const int64_t oyp = ((int64_t)(y == L - 1 ? 0 : y + 1) + (int64_t)L * z) * half + h;
        const int64_t ozp = ((int64_t)y + (int64_t)L * (z == L - 1 ? 0 : z + 1)) * half + h;
        const uint32_t e[3] = {planes[(4 * c + 1) * plane_words + o] ^ s ^ Sn[r * half + hx],
                               planes[(4 * c + 2) * plane_words + o] ^ s ^ Sn[oyp],
                               planes[(4 * c + 3) * plane_words + o] ^ s ^ Sn[ozp]};
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            uint32_t carry = e[m];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const uint32_t tj = cnt[j] & carry;
                cnt[j] ^= carry;
                carry = tj;
            }
        }
    }
    for (int b = 0; b < 32; ++b) {
        unsigned v = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) v |= ((cnt[j] >> b) & 1u) << j;
        if (v) atomicAdd(&sc[b], (unsigned long long)v);
    }
    __syncthreads();
    if (threadIdx.x < 32 && sc[threadIdx.x]) atomicAdd(&counts[threadIdx.x], sc[threadIdx.x]);
}

__global__ void amsc_unpack_kernel(const uint32_t* planes, int64_t plane_words, int L, int half, int b, int8_t* out) {
    const int64_t N = (int64_t)L * L * L;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % L), y = (int)((i / L) % L), z = (int)(i / ((int64_t)L * L));
        const int c = (x + y + z) & 1;
        const uint32_t w = planes[(4 * c) * plane_words + ((int64_t)y + (int64_t)L * z) * half + (x >> 1)];
        out[i] = ((w >> b) & 1u) ? 1 : -1;
    }
}

// Resident blocks per SM of the AMSC kernel of this kind and depth on the
// current device (cached per device and instantiation).
static int amsc_occupancy(int kind, int deep, size_t smem) {
    return with_kind(kind, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        static std::atomic<int> c8[kDeviceSlots], c4[kDeviceSlots];
        return deep ? occupancy_cached(c8, amsc_kernel<K, 8>, kAmscWarps * 32, smem)
                    : occupancy_cached(c4, amsc_kernel<K, 4>, kAmscWarps * 32, smem);
    });
}

// The sweep kernel's form for this ensemble on the current device: 0 = the
// chunked form (rows of a multiple of 128 sites per colour), else the blocks
// of 32 sites each lane keeps in flight in the site-strided form: 8 with fewer
// than 16 streams per SM, 4 otherwise.
static int amsc_form(const isg_amsc* m) {
    if (m->half % kChunk == 0) return 0;
    return m->S < kAmscDeepStreamsPerSM * (int64_t)sm_count() ? 8 : 4;
}

// Resident blocks per SM of the chunked kernel in registers.
static int amsc_chunk_occupancy(int kind, size_t smem) {
    return with_kind(kind, [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        static std::atomic<int> cache[kDeviceSlots];
        return occupancy_cached(cache, amsc_chunk_kernel<K>, kAmscWarps * 32, smem);
    });
}

static unsigned amsc_grid(int64_t n, int threads, int64_t per_thread) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t need = (n + threads * per_thread - 1) / (threads * per_thread);
    if (b > 152 * 16) b = 152 * 16;
    if (b < need) b = need;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace isg

using namespace isg;

extern "C" {

int isg_amsc_create(int L, const uint64_t* seed_J, const uint64_t* seed_spin, uint64_t seed_rng, double beta,
                    int rng_kind, isg_amsc** out) {
    if (!out || !seed_J || !seed_spin) { set_error("isg_amsc_create: NULL argument"); return ISG_ERR_ARG; }
    *out = nullptr;
    if (L < 4 || L > 1024 || (L & 1)) { set_error("isg_amsc_create: L=%d must be even and in [4, 1024]", L); return ISG_ERR_ARG; }
    if (!(beta > 0.0)) { set_error("isg_amsc_create: beta must be > 0 (got %g)", beta); return ISG_ERR_ARG; }
    if (!rng_kind_valid(rng_kind)) {
        set_error("isg_amsc_create: unknown rng_kind %d", rng_kind);
        return ISG_ERR_ARG;
    }
    isg_amsc* m = new (std::nothrow) isg_amsc();
    if (!m) { set_error("isg_amsc_create: out of host memory"); return ISG_ERR_NOMEM; }
    m->L = L;
    m->half = L / 2;
    m->kind = rng_kind;
    m->beta = beta;
    thresholds(beta, m->thr);
    m->seed_rng = seed_rng;
    for (int b = 0; b < 32; ++b) {
        m->seed_J[b] = seed_J[b];
        m->seed_spin[b] = seed_spin[b];
    }
    m->rows = (int64_t)L * L;
    {
        int64_t s0 = (int64_t)L * L * L / 32768;
        s0 = s0 < 1 ? 1 : (s0 > 8192 ? 8192 : s0);
        m->R = (m->rows + s0 - 1) / s0;
        m->S = (m->rows + m->R - 1) / m->R;
    }
    m->plane_words = (m->rows * m->half + 63) / 64 * 64;
    const size_t rng_words = (size_t)m->S * rng_state_words(rng_kind);
    cudaError_t e = cudaMalloc(&m->planes, (size_t)m->plane_words * 8 * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->rng, rng_words * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->rng_pos, (size_t)m->S * 4);
    if (e == cudaSuccess) e = cudaMalloc(&m->ctr, 33 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(m->ctr, 0, 33 * sizeof(unsigned long long));
    if (e == cudaSuccess) {
        AmscSeeds sd;
        for (int b = 0; b < 32; ++b) {
            sd.J[b] = seed_J[b];
            sd.S[b] = seed_spin[b];
        }
        amsc_init_kernel<<<amsc_grid(2 * m->plane_words, 256, 1), 256>>>(m->planes, m->plane_words, L, m->half, sd);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        isg_sim g;  // the fields the stream-seeding kernel reads
        g.kind = rng_kind;
        g.seed_rng = seed_rng;
        g.S = m->S;
        g.rng = m->rng;
        g.rng_pos = m->rng_pos;
        e = launch_init_rng(&g, 0);
        g.rng = nullptr;
        g.rng_pos = nullptr;
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        isg_amsc_destroy(m);
        return cuda_fail(e, "isg_amsc_create");
    }
    *out = m;
    return ISG_OK;
}

void isg_amsc_destroy(isg_amsc* m) {
    if (!m) return;
    cudaDeviceSynchronize();
    cudaFree(m->planes);
    cudaFree(m->rng);
    cudaFree(m->rng_pos);
    cudaFree(m->ctr);
    delete m;
}

int isg_amsc_sweep(isg_amsc* m, int64_t n, void* cuda_stream) {
    if (!m || n < 0) { set_error("isg_amsc_sweep: bad argument"); return ISG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const StreamConst k = stream_const();
    FlipArgs gen;
    memset(&gen, 0, sizeof gen);
    gen.rng = m->rng;
    gen.rng_pos = m->rng_pos;
    gen.mt = minstd_table();
    AmscArgs a;
    a.planes = m->planes;
    a.plane_words = m->plane_words;
    a.L = m->L;
    a.half = m->half;
    a.R = m->R;
    a.S = m->S;
    a.rows = m->rows;
    if (m->kind != ISG_RNG_MINSTD) {
        a.cmp1 = m->thr[1];
        a.cmp2 = m->thr[2];
        a.cmp3 = m->thr[3];
    } else {
        a.cmp1 = (uint32_t)(((uint64_t)m->thr[1] + 1) / 2);
        a.cmp2 = (uint32_t)(((uint64_t)m->thr[2] + 1) / 2);
        a.cmp3 = (uint32_t)(((uint64_t)m->thr[3] + 1) / 2);
    }
    const int sms = sm_count();
    const int form = amsc_form(m);
    const bool chunked = form == 0, deep = form == 8;  // deep: NB = 8, latency binds
    const size_t smem = m->kind == ISG_RNG_MT19937 ? (size_t)kAmscWarps * mt_window(kAmscSlack) * 4 : 0;
    const int oc = chunked ? amsc_chunk_occupancy(m->kind, smem) : amsc_occupancy(m->kind, deep ? 1 : 0, smem);
    int64_t blocks = (int64_t)sms * oc;
    const int64_t need = (m->S + kAmscWarps - 1) / kAmscWarps;
    if (blocks > need) blocks = need;
    for (int64_t sw = 0; sw < n; ++sw) {
        for (int c = 0; c < 2; ++c) {
            a.c = c;
            const cudaError_t e = with_kind(m->kind, [&](auto kc) {
                constexpr int K = decltype(kc)::value;
                if (chunked)
                    amsc_chunk_kernel<K><<<(unsigned)blocks, kAmscWarps * 32, smem, s>>>(a, gen, k, m->ctr,
                                                                                       m->tickets);
                else if (deep)
                    amsc_kernel<K, 8><<<(unsigned)blocks, kAmscWarps * 32, smem, s>>>(a, gen, k, m->ctr, m->tickets);
                else
                    amsc_kernel<K, 4><<<(unsigned)blocks, kAmscWarps * 32, smem, s>>>(a, gen, k, m->ctr, m->tickets);
                return cudaGetLastError();
            });
            if (e != cudaSuccess) return cuda_fail(e, "isg_amsc_sweep");
            m->tickets += (unsigned long long)m->S + (unsigned long long)blocks * kAmscWarps;
        }
    }
    m->sweeps += n;
    return ISG_OK;
}

int isg_amsc_info(const isg_amsc* m, int* L, int64_t* streams, int64_t* rows_per_stream, int* form) {
    if (!m) { set_error("isg_amsc_info: NULL handle"); return ISG_ERR_ARG; }
    if (L) *L = m->L;
    if (streams) *streams = m->S;
    if (rows_per_stream) *rows_per_stream = m->R;
    if (form) *form = amsc_form(m);
    return ISG_OK;
}

int isg_amsc_energies(isg_amsc* m, int64_t* E, void* cuda_stream) {
    if (!m || !E) { set_error("isg_amsc_energies: NULL argument"); return ISG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned long long* counts = m->ctr + 1;
    unsigned long long h[32];
    cudaError_t e = cudaMemsetAsync(counts, 0, 32 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        // at most 20000 site words per thread keeps the 16-bit counters exact (3 bonds each)
        amsc_unsat_kernel<<<amsc_grid(2 * m->plane_words, 256, 20000), 256, 0, s>>>(m->planes, m->plane_words, m->L,
                                                                                   m->half, counts);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, counts, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "isg_amsc_energies");
    const int64_t threeN = 3 * (int64_t)m->L * m->L * m->L;
    for (int b = 0; b < 32; ++b) E[b] = 2 * (int64_t)h[b] - threeN;
    return ISG_OK;
}

int isg_amsc_read_spins(const isg_amsc* m, int sample, int8_t* out, size_t n, void* cuda_stream) {
    const int64_t N = m ? (int64_t)m->L * m->L * m->L : 0;
    if (!m || !out || sample < 0 || sample >= 32 || (int64_t)n < N) {
        set_error("isg_amsc_read_spins: bad argument");
        return ISG_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int8_t* d = nullptr;
    cudaError_t e = cudaMalloc(&d, (size_t)N);
    if (e == cudaSuccess) {
        amsc_unpack_kernel<<<amsc_grid(N, 256, 1), 256, 0, s>>>(m->planes, m->plane_words, m->L, m->half, sample, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, (size_t)N, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    return e == cudaSuccess ? ISG_OK : cuda_fail(e, "isg_amsc_read_spins");
}

}  // extern "C"
