// isg_flip.cu -- the per-colour Metropolis flip kernel (Sec. 4) and the small
// kernels that expose its generator and bit logic to the tests.
//
// One warp owns one RNG stream, i.e. R consecutive rows r = y + L*z.  It walks
// its rows in groups of G = 32 / W rows (W words per row), so that one word of
// the group belongs to one lane:
//   1. draw phase: the warp produces the group's draws 32 at a time in stream
//      order (row by row, ascending x), compares each with the three integer
//      thresholds and stores the three ballots as bit streams in shared memory;
//   2. logic phase: each lane loads its word of S_c, its three forward coupling
//      words, the neighbour words of the other colour, counts unsatisfied bonds
//      with a bit-sliced adder, cuts its window out of the ballot bit streams,
//      forms the flip mask, XORs it into S_c and accumulates dE = 12 - 4u.
#include <algorithm>

#include "isg_common.cuh"

namespace isg {

constexpr int kFlipWarps = 4;

// Shared-memory words of one warp's generator state: MT19937 keeps its
// 624-word ring there; MINSTD and Parisi-Rapuano live in registers.
template <int KIND>
struct RingWords {
    static constexpr int value = (KIND == ISG_RNG_MT19937) ? kMtN : 0;
};

// The logic phase for one word: returns the flip mask and adds its dE.
template <typename Word>
__device__ __forceinline__ Word flip_word(const FlipArgs& a, int r, int k, int off, const uint32_t* cond,
                                          int& dEsum) {
    constexpr int w = 8 * sizeof(Word);
    const int c = a.c, L = a.L, W = a.W, nt = a.nt;
    const int64_t pb = a.plane_bytes;
    Word* Sc = (Word*)(a.planes + (size_t)(4 * c + 0) * pb);
    const Word* Jxc = (const Word*)(a.planes + (size_t)(4 * c + 1) * pb);
    const Word* Jyc = (const Word*)(a.planes + (size_t)(4 * c + 2) * pb);
    const Word* Jzc = (const Word*)(a.planes + (size_t)(4 * c + 3) * pb);
    const int n = c ^ 1;
    const Word* Sn = (const Word*)(a.planes + (size_t)(4 * n + 0) * pb);
    const Word* Jxn = (const Word*)(a.planes + (size_t)(4 * n + 1) * pb);
    const Word* Jyn = (const Word*)(a.planes + (size_t)(4 * n + 2) * pb);
    const Word* Jzn = (const Word*)(a.planes + (size_t)(4 * n + 3) * pb);

    const int y = r % L, z = r / L;
    const int p = (c + y + z) & 1;
    const int ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
    const int zm = z == 0 ? L - 1 : z - 1, zp = z == L - 1 ? 0 : z + 1;
    const size_t o = (size_t)r * W + k;
    const size_t oym = (size_t)(ym + L * z) * W + k, oyp = (size_t)(yp + L * z) * W + k;
    const size_t ozm = (size_t)(y + L * zm) * W + k, ozp = (size_t)(y + L * zp) * W + k;

    const Word s = Sc[o];
    const Word na = Sn[o];
    const Word e_yp = Jyc[o] ^ s ^ Sn[oyp];
    const Word e_ym = Jyn[oym] ^ s ^ Sn[oym];
    const Word e_zp = Jzc[o] ^ s ^ Sn[ozp];
    const Word e_zm = Jzn[ozm] ^ s ^ Sn[ozm];
    Word e_xp, e_xm;
    if (p == 0) {
        // +x neighbour is the aligned bit h, -x neighbour is bit h-1
        const size_t onb = (size_t)r * W + (k == 0 ? W - 1 : k - 1);
        e_xp = Jxc[o] ^ s ^ na;
        e_xm = row_down<Word>(Jxn[o] ^ na, Jxn[onb] ^ Sn[onb], k, nt) ^ s;
    } else {
        // +x neighbour is bit h+1, -x neighbour is the aligned bit h
        const size_t onb = (size_t)r * W + (k == W - 1 ? 0 : k + 1);
        e_xp = Jxc[o] ^ s ^ row_up<Word>(na, Sn[onb], k, W, nt);
        e_xm = Jxn[o] ^ s ^ na;
    }
    Word u0, u1, u2;
    Logic<Word>::count6(e_xp, e_xm, e_yp, e_ym, e_zp, e_zm, u0, u1, u2);
    const Word c4 = take_bits<Word>(cond, off);
    const Word c8 = take_bits<Word>(cond + kCondWords, off);
    const Word c12 = take_bits<Word>(cond + 2 * kCondWords, off);
    Word f = Logic<Word>::flip(u0, u1, u2, c4, c8, c12);
    if (k == W - 1 && nt < w) f &= (Word)((Word(1) << nt) - 1);
    Sc[o] = s ^ f;
    dEsum += Logic<Word>::dE(f, u0, u1, u2);
    return f;
}

template <typename Word, int KIND>
__global__ void __launch_bounds__(kFlipWarps * 32) flip_plain_kernel(FlipArgs a) {
    extern __shared__ uint32_t smem[];
    constexpr int w = 8 * sizeof(Word);
    constexpr int kRing = RingWords<KIND>::value;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * kFlipWarps + wid;
    if (t >= a.S) return;  // whole warp leaves together; no block barrier below
    uint32_t* ring = smem + wid * (kRing + 3 * kCondWords);
    uint32_t* cond = ring + kRing;

    int pos = 0;
    uint32_t x = 0, x2 = 0;
    if (KIND == ISG_RNG_MT19937) {
        for (int i = lane; i < kMtN; i += 32) ring[i] = a.rng[t * kMtN + i];
        pos = (int)a.rng_pos[t];
        __syncwarp();
    } else if (KIND == ISG_RNG_PARISI_RAPUANO) {
        pr_load(a.rng + t * kPrN, x, x2, lane);
    } else {
        x = minstd_mulmod(a.rng[t], a.mt.pow[lane + 1]);
    }

    const int W = a.W, half = a.half;
    const int G = 32 / W;
    const int64_t r_begin = t * a.R;
    const int64_t r_end = r_begin + a.R < a.rows ? r_begin + a.R : a.rows;
    int dEsum = 0;
    for (int64_t g0 = r_begin; g0 < r_end; g0 += G) {
        const int nrows = (int)((r_end - g0) < G ? (r_end - g0) : G);
        const int D = nrows * half;
        const int nblk = (D + 31) >> 5;
        for (int b = 0; b < nblk; ++b) {
            const int nvalid = D - 32 * b < 32 ? D - 32 * b : 32;
            uint32_t d;
            if (KIND == ISG_RNG_MT19937) d = mt_warp_step(ring, pos, lane, nvalid);
            else if (KIND == ISG_RNG_PARISI_RAPUANO) d = pr_warp_step(x, x2, lane, nvalid);
            else d = minstd_warp_step(x, a.mt.pow[32], nvalid, lane);
            const uint32_t m4 = __ballot_sync(kFull, d < a.thr1);
            const uint32_t m8 = __ballot_sync(kFull, d < a.thr2);
            const uint32_t m12 = __ballot_sync(kFull, d < a.thr3);
            const uint32_t mv = lane == 0 ? m4 : (lane == 1 ? m8 : m12);
            if (lane < 3) cond[lane * kCondWords + b] = mv;
        }
        __syncwarp();
        if (lane < nrows * W) {
            const int j = lane / W, k = lane - j * W;
            flip_word<Word>(a, (int)(g0 + j), k, j * half + k * w, cond, dEsum);
        }
        __syncwarp();
    }

    if (KIND == ISG_RNG_MT19937) {
        for (int i = lane; i < kMtN; i += 32) a.rng[t * kMtN + i] = ring[i];
        if (lane == 0) a.rng_pos[t] = (uint32_t)pos;
    } else if (KIND == ISG_RNG_PARISI_RAPUANO) {
        pr_store(a.rng + t * kPrN, x, x2, lane);
    } else {
        const uint32_t x0 = __shfl_sync(kFull, x, 0);
        if (lane == 0) a.rng[t] = minstd_mulmod(x0, a.mt.inv);  // state of the last draw used
    }
    for (int sh = 16; sh; sh >>= 1) dEsum += __shfl_xor_sync(kFull, dEsum, sh);
    if (lane == 0 && dEsum != 0) atomicAdd((unsigned long long*)a.dE, (unsigned long long)(long long)dEsum);
}

MinstdTable minstd_table() {
    MinstdTable t;
    t.pow[0] = 1;
    for (int j = 1; j <= 32; ++j) t.pow[j] = minstd_mulmod(t.pow[j - 1], kMinstdA);
    // inverse by Fermat: a^(M-2) mod M
    uint32_t r = 1, b = kMinstdA;
    for (uint32_t e = kMinstdM - 2; e; e >>= 1) {
        if (e & 1) r = minstd_mulmod(r, b);
        b = minstd_mulmod(b, b);
    }
    t.inv = r;
    return t;
}

FlipArgs make_flip_args(isg_sim* h, int colour) {
    FlipArgs a;
    a.planes = h->planes;
    a.plane_bytes = h->plane_bytes;
    a.L = h->L;
    a.half = h->half;
    a.W = h->W;
    a.nt = h->nt;
    a.c = colour;
    a.R = h->R;
    a.S = h->S;
    a.rows = h->rows;
    a.thr1 = h->thr[1];
    a.thr2 = h->thr[2];
    a.thr3 = h->thr[3];
    if (h->kind != ISG_RNG_MINSTD) {
        a.cmp1 = h->thr[1];
        a.cmp2 = h->thr[2];
        a.cmp3 = h->thr[3];
    } else {
        a.cmp1 = (uint32_t)(((uint64_t)h->thr[1] + 1) / 2);
        a.cmp2 = (uint32_t)(((uint64_t)h->thr[2] + 1) / 2);
        a.cmp3 = (uint32_t)(((uint64_t)h->thr[3] + 1) / 2);
    }
    a.rng = h->rng;
    a.rng_pos = h->rng_pos;
    a.dE = h->scal;
    a.mt = minstd_table();
    return a;
}

template <typename Word, int KIND>
static cudaError_t launch_plain_t(isg_sim* h, int colour, cudaStream_t s) {
    const FlipArgs a = make_flip_args(h, colour);
    const int blocks = (int)((h->S + kFlipWarps - 1) / kFlipWarps);
    const size_t smem = (size_t)kFlipWarps * (RingWords<KIND>::value + 3 * kCondWords) * sizeof(uint32_t);
    flip_plain_kernel<Word, KIND><<<blocks, kFlipWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_flip_plain(isg_sim* h, int colour, cudaStream_t s) {
    return with_kind(h->kind, [&](auto kind) {
        constexpr int K = decltype(kind)::value;
        return h->wbits == 64 ? launch_plain_t<uint64_t, K>(h, colour, s) : launch_plain_t<uint32_t, K>(h, colour, s);
    });
}

// ---------------------------------------------------------------------------
// Draws of one stream from its current position, without advancing it.
template <int KIND>
__global__ void peek_kernel(const uint32_t* rng, const uint32_t* rng_pos, int64_t t, int64_t n,
                            uint32_t* out, MinstdTable mt) {
    __shared__ uint32_t ring[kMtN];
    const int lane = threadIdx.x;
    int pos = 0;
    uint32_t x = 0, x2 = 0;
    if (KIND == ISG_RNG_MT19937) {
        for (int i = lane; i < kMtN; i += 32) ring[i] = rng[t * kMtN + i];
        pos = (int)rng_pos[t];
        __syncwarp();
    } else if (KIND == ISG_RNG_PARISI_RAPUANO) {
        pr_load(rng + t * kPrN, x, x2, lane);
    } else {
        x = minstd_mulmod(rng[t], mt.pow[lane + 1]);
    }
    for (int64_t k = 0; k < n; k += 32) {
        const int nvalid = n - k < 32 ? (int)(n - k) : 32;
        uint32_t d;
        if (KIND == ISG_RNG_MT19937) d = mt_warp_step(ring, pos, lane, nvalid);
        else if (KIND == ISG_RNG_PARISI_RAPUANO) d = pr_warp_step(x, x2, lane, nvalid);
        else d = minstd_warp_step(x, mt.pow[32], nvalid, lane);
        if (lane < nvalid) out[k + lane] = d;
    }
}

cudaError_t launch_peek_draws(const isg_sim* h, int64_t t, int64_t n, uint32_t* out, cudaStream_t s) {
    const MinstdTable mt = minstd_table();
    return with_kind(h->kind, [&](auto kind) {
        peek_kernel<decltype(kind)::value><<<1, 32, 0, s>>>(h->rng, h->rng_pos, t, n, out, mt);
        return cudaGetLastError();
    });
}

// ---------------------------------------------------------------------------
// Stencil self-test: 32 stencils per warp, one bit per stencil, run through the
// same Logic<> code as the flip kernel, in 32-bit and in 64-bit words.
__global__ void stencil_kernel(const uint16_t* code, const uint32_t* draw, int64_t n, uint32_t t1,
                               uint32_t t2, uint32_t t3, uint8_t* flip, uint8_t* uout) {
    const int lane = threadIdx.x & 31;
    const int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) - lane;
    if (base >= n) return;
    const int64_t j = base + lane;
    const bool ok = j < n;
    const uint32_t cd = ok ? code[j] : 0u;
    const uint32_t d = ok ? draw[j] : 0xFFFFFFFFu;
    const uint32_t s = __ballot_sync(kFull, cd & 1u);
    uint32_t e[6];
    for (int k = 0; k < 6; ++k) {
        const uint32_t nk = __ballot_sync(kFull, (cd >> (1 + k)) & 1u);
        const uint32_t jk = __ballot_sync(kFull, (cd >> (7 + k)) & 1u);
        e[k] = jk ^ s ^ nk;
    }
    const uint32_t c4 = __ballot_sync(kFull, d < t1), c8 = __ballot_sync(kFull, d < t2),
                   c12 = __ballot_sync(kFull, d < t3);
    uint32_t u0, u1, u2;
    Logic<uint32_t>::count6(e[0], e[1], e[2], e[3], e[4], e[5], u0, u1, u2);
    const uint32_t f = Logic<uint32_t>::flip(u0, u1, u2, c4, c8, c12);
    // 64-bit words: the same 32 stencils in both halves; both halves must agree
    // with the 32-bit result, else u is reported as 0xFF.
    uint64_t E[6];
    for (int k = 0; k < 6; ++k) E[k] = ((uint64_t)e[k] << 32) | e[k];
    uint64_t v0, v1, v2;
    Logic<uint64_t>::count6(E[0], E[1], E[2], E[3], E[4], E[5], v0, v1, v2);
    const uint64_t F = Logic<uint64_t>::flip(v0, v1, v2, ((uint64_t)c4 << 32) | c4, ((uint64_t)c8 << 32) | c8,
                                             ((uint64_t)c12 << 32) | c12);
    const bool agree = ((uint32_t)F == f) && ((uint32_t)(F >> 32) == f) && ((uint32_t)v0 == u0) &&
                       ((uint32_t)(v1 >> 32) == u1) && ((uint32_t)v2 == u2);
    if (ok) {
        flip[j] = (uint8_t)((f >> lane) & 1u);
        uout[j] = agree ? (uint8_t)(((u0 >> lane) & 1u) | (((u1 >> lane) & 1u) << 1) | (((u2 >> lane) & 1u) << 2))
                        : (uint8_t)0xFF;
    }
}

cudaError_t launch_stencil(const uint16_t* code, const uint32_t* draw, int64_t n, uint32_t t1, uint32_t t2,
                           uint32_t t3, uint8_t* flip, uint8_t* u, cudaStream_t s) {
    const int threads = 256;
    const int64_t blocks = (n + threads - 1) / threads;
    stencil_kernel<<<(unsigned)blocks, threads, 0, s>>>(code, draw, n, t1, t2, t3, flip, u);
    return cudaGetLastError();
}

}  // namespace isg
