// isg_stream.cuh -- one warp's colour pass over one RNG stream, shared by the
// single-lattice kernel (isg_flip_fast.cu) and the batched engine (isg_batch.cu).
//
// A stream owns R consecutive rows r = y + L*z of a lattice.  The warp walks
// them in groups of G = 32 / W rows (W words per row and colour), one word of
// the group per lane:
//   1. draw phase: the group's draws are produced 64 at a time in stream order
//      (row by row, ascending x), compared with the three integer thresholds
//      (Sec. 4: R < Rmax exp(-beta dE)) and the three ballots stored as bit
//      streams in shared memory;
//   2. logic phase: each lane loads its word of S_c, its forward couplings and
//      the other colour's neighbour words, counts unsatisfied bonds with a
//      bit-sliced adder, cuts its window out of the ballot bit streams, forms
//      the flip mask, XORs it into S_c and sums dE = 12 - 4u.
//
// Generators (Sec. 3):
//   * MT19937 keeps its 624 words twice in shared memory (slot s and s + 624
//     hold the same word), so x_{k+1} and x_{k+397} sit at fixed offsets from
//     one index; its shifts run as multiplies (MtMul) on the FMA pipe;
//   * MINSTD keeps two lanes' worth of states (positions +1..+32 and +33..+64)
//     and compares the state x with ceil(thr / 2) (d = 2x < thr <=> x <
//     ceil(thr / 2)).
#pragma once

#include "isg_common.cuh"

namespace isg {

// Multipliers that turn the generator's shifts into integer multiplies:
// v >> k == umulhi(v, 2^(32-k)) and v << k == v * 2^k (mod 2^32), exactly.
// They arrive as kernel arguments so that the compiler cannot fold them back
// into shift instructions: the multiplies run on the FMA pipe, leaving only the
// XORs on the (half-rate) logic pipe.
struct MtMul {
    uint32_t hi31;  // 2^31: >> 1
    uint32_t hi21;  // 2^21: >> 11
    uint32_t hi14;  // 2^14: >> 18
    uint32_t lo7;   // 2^7:  << 7
    uint32_t lo15;  // 2^15: << 15
};

// Per-launch generator constants.
struct StreamConst {
    MtMul mul;
    uint32_t a32;   // 16807^32 mod (2^31 - 1)
    uint32_t a64;   // 16807^64 mod (2^31 - 1)
};

inline StreamConst stream_const() {
    const MinstdTable t = minstd_table();
    StreamConst k;
    k.mul.hi31 = 1u << 31;
    k.mul.hi21 = 1u << 21;
    k.mul.hi14 = 1u << 14;
    k.mul.lo7 = 1u << 7;
    k.mul.lo15 = 1u << 15;
    k.a32 = t.pow[32];
    k.a64 = minstd_mulmod(t.pow[32], t.pow[32]);
    return k;
}

// MT19937 twist of one word: x_{k+624} from x_k, x_{k+1}, x_{k+397}.  The odd
// test uses b - 2 (b >> 1) = b & 1.
__device__ __forceinline__ uint32_t mt_twist(uint32_t a, uint32_t b, uint32_t m, const MtMul& k) {
    const uint32_t y = (a & 0x80000000u) | (b & 0x7FFFFFFFu);
    const uint32_t ys = __umulhi(y, k.hi31);
    const uint32_t bh = __umulhi(b, k.hi31);
    const uint32_t odd = b - 2u * bh;
    return m ^ ys ^ (odd * 0x9908B0DFu);
}

// MT19937 tempering with the shifts done as multiplies (see MtMul).
__device__ __forceinline__ uint32_t mt_temper_mul(uint32_t v, const MtMul& k) {
    v ^= __umulhi(v, k.hi21);
    v ^= (v * k.lo7) & 0x9D2C5680u;
    v ^= (v * k.lo15) & 0xEFC60000u;
    v ^= __umulhi(v, k.hi14);
    return v;
}

// Two 32-draw blocks of an MT19937 stream held in a mirrored 1248-word ring.
// iA = (k + lane) mod 624 for the first block's draw k + lane; on return it
// points 64 draws further.  Reads of both blocks precede all writes (one warp
// barrier between): block B's inputs x_{k+32+l+397} were written 195 or more
// draws earlier, and the words both blocks overwrite are read first.
__device__ __forceinline__ void mt_pair(uint32_t* ring, int& iA, uint32_t& dA, uint32_t& dB, const MtMul& k) {
    int iB = iA + 32;
    iB = iB >= kMtN ? iB - kMtN : iB;
    const uint32_t aA = ring[iA], bA = ring[iA + 1], mA = ring[iA + kMtM];
    const uint32_t aB = ring[iB], bB = ring[iB + 1], mB = ring[iB + kMtM];
    __syncwarp();
    const uint32_t vA = mt_twist(aA, bA, mA, k);
    const uint32_t vB = mt_twist(aB, bB, mB, k);
    ring[iA] = vA;
    ring[iA + kMtN] = vA;
    ring[iB] = vB;
    ring[iB + kMtN] = vB;
    __syncwarp();
    iA = iB + 32;
    iA = iA >= kMtN ? iA - kMtN : iA;
    dA = mt_temper_mul(vA, k);
    dB = mt_temper_mul(vB, k);
}

// Four 32-draw blocks (128 draws) at once: block j reads x_{k+32j+l+397}, which
// was written 227 - 32j - l >= 100 draws before this step, and no block reads a
// word another block of the step writes after the barrier.
__device__ __forceinline__ void mt_quad(uint32_t* ring, int& i0, uint32_t d[4], const MtMul& k) {
    int i[4];
    i[0] = i0;
#pragma unroll
    for (int j = 1; j < 4; ++j) {
        const int v = i[j - 1] + 32;
        i[j] = v >= kMtN ? v - kMtN : v;
    }
    uint32_t a[4], b[4], m[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        a[j] = ring[i[j]];
        b[j] = ring[i[j] + 1];
        m[j] = ring[i[j] + kMtM];
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t v = mt_twist(a[j], b[j], m[j], k);
        ring[i[j]] = v;
        ring[i[j] + kMtN] = v;
        d[j] = v;
    }
    __syncwarp();
    const int v = i[3] + 32;
    i0 = v >= kMtN ? v - kMtN : v;
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j] = mt_temper_mul(d[j], k);
}

// One block of up to 32 draws (tail of a row group); lanes >= nvalid consume nothing.
__device__ __forceinline__ uint32_t mt_single(uint32_t* ring, int& iA, int lane, int nvalid, const MtMul& k) {
    const uint32_t a = ring[iA], b = ring[iA + 1], m = ring[iA + kMtM];
    __syncwarp();
    const uint32_t v = mt_twist(a, b, m, k);
    if (lane < nvalid) {
        ring[iA] = v;
        ring[iA + kMtN] = v;
    }
    __syncwarp();
    iA += nvalid;
    iA = iA >= kMtN ? iA - kMtN : iA;
    return mt_temper_mul(v, k);
}

// Logic phase for one word of colour c at row r = y + L z, word k (see the
// layout notes in isg_common.cuh); adds the word's dE to dEsum.
template <typename Word>
__device__ __forceinline__ void word_update(const FlipArgs& a, int c, int r, int y, int z, int k,
                                            const uint32_t* cond, int off, int& dEsum) {
    constexpr int w = 8 * sizeof(Word);
    const int L = a.L, W = a.W, nt = a.nt;
    const size_t pb = (size_t)a.plane_bytes;
    Word* Sc = (Word*)(a.planes + (size_t)(4 * c) * pb);
    const Word* Jxc = (const Word*)(a.planes + (size_t)(4 * c + 1) * pb);
    const Word* Jyc = (const Word*)(a.planes + (size_t)(4 * c + 2) * pb);
    const Word* Jzc = (const Word*)(a.planes + (size_t)(4 * c + 3) * pb);
    const int n = c ^ 1;
    const Word* Sn = (const Word*)(a.planes + (size_t)(4 * n) * pb);
    const Word* Jxn = (const Word*)(a.planes + (size_t)(4 * n + 1) * pb);
    const Word* Jyn = (const Word*)(a.planes + (size_t)(4 * n + 2) * pb);
    const Word* Jzn = (const Word*)(a.planes + (size_t)(4 * n + 3) * pb);

    const int p = (c + y + z) & 1;
    const int rowW = r * W;
    const int dym = (y == 0 ? L - 1 : -1) * W, dyp = (y == L - 1 ? 1 - L : 1) * W;
    const int LW = L * W;
    const int dzm = (z == 0 ? (L - 1) * LW : -LW), dzp = (z == L - 1 ? -(L - 1) * LW : LW);
    const size_t o = (size_t)(rowW + k);

    const Word s = Sc[o];
    const Word na = Sn[o];
    const Word e_yp = Jyc[o] ^ s ^ Sn[o + dyp];
    const Word e_ym = Jyn[o + dym] ^ s ^ Sn[o + dym];
    const Word e_zp = Jzc[o] ^ s ^ Sn[o + dzp];
    const Word e_zm = Jzn[o + dzm] ^ s ^ Sn[o + dzm];
    Word e_xp, e_xm;
    if (p == 0) {
        const size_t onb = (size_t)(rowW + (k == 0 ? W - 1 : k - 1));
        e_xp = Jxc[o] ^ s ^ na;
        e_xm = row_down<Word>(Jxn[o] ^ na, Jxn[onb] ^ Sn[onb], k, nt) ^ s;
    } else {
        const size_t onb = (size_t)(rowW + (k == W - 1 ? 0 : k + 1));
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
}

// Generator state of the stream a warp is working on.
struct StreamRegs {
    int iA;        // MT19937: (next draw + lane) mod 624 in the ring
    uint32_t xA;   // MINSTD: state of draw n + lane + 1
    uint32_t xB;   // MINSTD: state of draw n + lane + 33
};

template <int KIND>
__device__ __forceinline__ void load_stream(const FlipArgs& a, int64_t t, uint32_t* ring, StreamRegs& st,
                                            const StreamConst& k, int lane) {
    if (KIND == ISG_RNG_MT19937) {
        for (int i = lane; i < kMtN; i += 32) {
            const uint32_t v = a.rng[t * kMtN + i];
            ring[i] = v;
            ring[i + kMtN] = v;
        }
        const int i = (int)a.rng_pos[t] + lane;
        st.iA = i >= kMtN ? i - kMtN : i;
        __syncwarp();
    } else {
        st.xA = minstd_mulmod(a.rng[t], a.mt.pow[lane + 1]);
        st.xB = minstd_mulmod(st.xA, k.a32);
    }
}

template <int KIND>
__device__ __forceinline__ void store_stream(const FlipArgs& a, int64_t t, const uint32_t* ring,
                                             const StreamRegs& st, int lane) {
    if (KIND == ISG_RNG_MT19937) {
        __syncwarp();
        for (int i = lane; i < kMtN; i += 32) a.rng[t * kMtN + i] = ring[i];
        const int pos = __shfl_sync(kFull, st.iA, 0);
        if (lane == 0) a.rng_pos[t] = (uint32_t)pos;
        __syncwarp();
    } else {
        const uint32_t x0 = __shfl_sync(kFull, st.xA, 0);
        if (lane == 0) a.rng[t] = minstd_mulmod(x0, a.mt.inv);  // state of the last draw used
    }
}

// One pass of colour c over stream t; the stream state is in ring / st.
template <typename Word, int KIND>
__device__ __forceinline__ void stream_pass(const FlipArgs& a, int c, int64_t t, uint32_t* ring, uint32_t* cond,
                                            StreamRegs& st, const StreamConst& k, int lane, int& dEsum) {
    constexpr int w = 8 * sizeof(Word);
    constexpr bool kMT = KIND == ISG_RNG_MT19937;
    const int W = a.W, half = a.half, L = a.L;
    const int G = 32 / W;
    const int lj = lane / W, lk = lane - lj * W;
    const int loff = lj * half + lk * w;
    const int64_t r_begin = t * a.R;
    const int64_t r_end = r_begin + a.R < a.rows ? r_begin + a.R : a.rows;
    int r = (int)r_begin + lj;
    int y = r % L, z = r / L;
    for (int64_t g0 = r_begin; g0 < r_end; g0 += G) {
        const int nrows = (int)((r_end - g0) < G ? (r_end - g0) : G);
        const int D = nrows * half;
        const int nquads = kMT ? (D >> 7) : 0;
        for (int q = 0; q < nquads; ++q) {
            uint32_t d[4], c4[4], c8[4], c12[4];
            mt_quad(ring, st.iA, d, k.mul);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                c4[j] = __ballot_sync(kFull, d[j] < a.cmp1);
                c8[j] = __ballot_sync(kFull, d[j] < a.cmp2);
                c12[j] = __ballot_sync(kFull, d[j] < a.cmp3);
            }
            if (lane == 0) {
                *(uint4*)(cond + 4 * q) = make_uint4(c4[0], c4[1], c4[2], c4[3]);
                *(uint4*)(cond + kCondWords + 4 * q) = make_uint4(c8[0], c8[1], c8[2], c8[3]);
                *(uint4*)(cond + 2 * kCondWords + 4 * q) = make_uint4(c12[0], c12[1], c12[2], c12[3]);
            }
        }
        uint32_t* cw = cond + 4 * nquads;  // the pair and single steps continue the bit streams here
        const int Dq = D - (nquads << 7);
        const int npairs = Dq >> 6;
        for (int q = 0; q < npairs; ++q) {
            uint32_t dA, dB;
            if (kMT) {
                mt_pair(ring, st.iA, dA, dB, k.mul);
            } else {
                dA = st.xA;
                dB = st.xB;
                st.xA = minstd_mulmod(st.xA, k.a64);
                st.xB = minstd_mulmod(st.xB, k.a64);
            }
            const uint32_t A4 = __ballot_sync(kFull, dA < a.cmp1), B4 = __ballot_sync(kFull, dB < a.cmp1);
            const uint32_t A8 = __ballot_sync(kFull, dA < a.cmp2), B8 = __ballot_sync(kFull, dB < a.cmp2);
            const uint32_t A12 = __ballot_sync(kFull, dA < a.cmp3), B12 = __ballot_sync(kFull, dB < a.cmp3);
            if (lane == 0) {
                *(uint2*)(cw + 2 * q) = make_uint2(A4, B4);
                *(uint2*)(cw + kCondWords + 2 * q) = make_uint2(A8, B8);
                *(uint2*)(cw + 2 * kCondWords + 2 * q) = make_uint2(A12, B12);
            }
        }
        int rem = Dq - (npairs << 6);
        int b = 2 * npairs;
        while (rem > 0) {
            const int nvalid = rem < 32 ? rem : 32;
            uint32_t d;
            if (kMT) {
                d = mt_single(ring, st.iA, lane, nvalid, k.mul);
            } else {
                d = st.xA;
                const int src = lane + nvalid;
                const uint32_t pa = __shfl_sync(kFull, st.xA, src & 31);
                const uint32_t pb = __shfl_sync(kFull, st.xB, src & 31);
                st.xA = src < 32 ? pa : pb;
                st.xB = minstd_mulmod(st.xA, k.a32);
            }
            const uint32_t m4 = __ballot_sync(kFull, d < a.cmp1);
            const uint32_t m8 = __ballot_sync(kFull, d < a.cmp2);
            const uint32_t m12 = __ballot_sync(kFull, d < a.cmp3);
            if (lane == 0) {
                cw[b] = m4;
                cw[kCondWords + b] = m8;
                cw[2 * kCondWords + b] = m12;
            }
            ++b;
            rem -= nvalid;
        }
        __syncwarp();
        if (lane < nrows * W) word_update<Word>(a, c, r, y, z, lk, cond, loff, dEsum);
        __syncwarp();
        r += G;
        y += G;
        while (y >= L) {
            y -= L;
            ++z;
        }
    }
}

}  // namespace isg
