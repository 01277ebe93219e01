// isg_stream.cuh -- one warp's colour pass over one RNG stream, shared by the
// single-lattice kernel (isg_flip_fast.cu) and the batched engine (isg_batch.cu).
//
// A stream owns R consecutive rows r = y + L*z of a lattice.  The warp walks
// them in groups of G = 32 / W rows (W words per row and colour), one word of
// the group per lane:
//   1. draw phase: the group's draws are produced 128 (MT19937 in the latency
//      form: 224) at a time in stream order
//      (row by row, ascending x) and compared with the three integer thresholds
//      thr1 > thr2 > thr3 (Sec. 4: R < Rmax exp(-beta dE)).  Because the three
//      comparisons are nested, a draw's outcome is a level 0..3 (how many
//      thresholds it is below), and two ballots per 32 draws carry it: "lo" =
//      level odd, "hi" = level >= 2; they are stored as bit streams in shared
//      memory;
//   2. logic phase: each lane loads its word of S_c, its forward couplings and
//      the other colour's neighbour words, counts unsatisfied bonds with a
//      bit-sliced adder, cuts its window out of the two bit streams
//      (d < thr1 = lo | hi, d < thr2 = hi, d < thr3 = lo & hi), forms the flip
//      mask, XORs it into S_c and sums dE = 12 - 4u.
//
// Generators (Sec. 3):
//   * MT19937 keeps its words in a linear window of shared memory: B[j] holds
//     x_{base + j}, x_{k+624} is appended at B[k - base + 624], and when the
//     free slots run out the 624 live words move back to the front; the reads
//     x_k, x_{k+1}, x_{k+397} are fixed offsets from one index with no
//     wrap-around arithmetic.  Its shifts run as multiplies (MtMul) on the FMA
//     pipe;
//   * MINSTD keeps two lanes' worth of states (positions +1..+32 and +33..+64)
//     and compares the state x with ceil(thr / 2) (d = 2x < thr <=> x <
//     ceil(thr / 2));
//   * Parisi-Rapuano keeps its 64-word window in two registers per lane
//     (pr_warp_step in isg_common.cuh): no shared memory.
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

// Shared-memory words of one warp's MT19937 window with `slack` free slots.
constexpr int mt_window(int slack) { return kMtN + slack; }

// MT19937 twist of one word: x_{k+624} from x_k, x_{k+1}, x_{k+397}.  y and
// x_{k+1} share their low bit, so the odd test is y - 2 (y >> 1) = y & 1, one
// multiply-add on the shift y >> 1 that the twist needs anyway (testing the
// low bit of x_{k+1} by its own shift cost one more FMA-pipe instruction per
// draw: L = 1024 MT19937 1.169 -> 1.101 ps per attempt without it).
__device__ __forceinline__ uint32_t mt_twist(uint32_t a, uint32_t b, uint32_t m, const MtMul& k) {
    const uint32_t y = (a & 0x80000000u) | (b & 0x7FFFFFFFu);
    const uint32_t ys = __umulhi(y, k.hi31);
    const uint32_t odd = y - 2u * ys;
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

// Make room for `need` more words: if the window is full, move the 624 live
// words B[iA .. iA+623] to the front (all read before any is written).
template <int SLACK>
__device__ __forceinline__ void mt_make_room(uint32_t* B, int& iA, int need, int lane) {
    if (iA + kMtN + need <= mt_window(SLACK)) return;
    __syncwarp();
    if ((iA & 3) == 0) {  // 16-byte aligned: 156 four-word moves (5 per lane)
        uint4 v[5];
#pragma unroll
        for (int q = 0; q < 5; ++q)
            if (lane + 32 * q < kMtN / 4) v[q] = *(const uint4*)(B + iA + 4 * (lane + 32 * q));
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 5; ++q)
            if (lane + 32 * q < kMtN / 4) *(uint4*)(B + 4 * (lane + 32 * q)) = v[q];
    } else {
        uint32_t v[20];
#pragma unroll
        for (int q = 0; q < 20; ++q) v[q] = (lane + 32 * q < kMtN) ? B[iA + lane + 32 * q] : 0u;
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 20; ++q)
            if (lane + 32 * q < kMtN) B[lane + 32 * q] = v[q];
    }
    __syncwarp();
    iA = 0;
}

// Four 32-draw blocks (128 draws) at once.  Block j reads x_{k+32j+l+397},
// which was appended 227 - 32j - l >= 100 draws before this step; the step's
// reads (indices up to k + 524) and writes (from k + 624) never meet, so the
// one warp barrier after the writes, which orders them before the next step's
// reads, is the only one (a second one between the reads and the writes cost
// 0.7 % at L = 1024).
template <int SLACK, bool ROOM = true>
__device__ __forceinline__ void mt_quad(uint32_t* B, int& iA, uint32_t d[4], const MtMul& k, int lane) {
    if (ROOM) mt_make_room<SLACK>(B, iA, 128, lane);
    uint32_t a[4], b[4], m[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int i = iA + 32 * j + lane;
        a[j] = B[i];
        b[j] = B[i + 1];
        m[j] = B[i + kMtM];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t v = mt_twist(a[j], b[j], m[j], k);
        B[iA + 32 * j + lane + kMtN] = v;
        d[j] = v;
    }
    __syncwarp();
    iA += 128;
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j] = mt_temper_mul(d[j], k);
}

// The twist half of a seven-block step (224 draws) for warps too few to hide
// latency: the raw words x_{k+624+32j+l} of blocks j = 0..6, appended to the
// window and returned untempered in v.  Block j reads x_{k+32j+l+397} with
// 32j + l + 397 <= 620 < 624, i.e. words that exist before the step, so no read
// of the step touches a word the step writes and the step needs no barrier of
// its own; the caller puts one warp barrier between consecutive steps.  227
// draws is the most one step of the recurrence allows.
template <int SLACK>
__device__ __forceinline__ void mt_seven_raw(uint32_t* B, int& iA, uint32_t v[7], const MtMul& k, int lane) {
    mt_make_room<SLACK>(B, iA, 224, lane);
    uint32_t a[7], b[7], m[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        const int i = iA + 32 * j + lane;
        a[j] = B[i];
        b[j] = B[i + 1];
        m[j] = B[i + kMtM];
    }
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        v[j] = mt_twist(a[j], b[j], m[j], k);
        B[iA + 32 * j + lane + kMtN] = v[j];
    }
    iA += 224;
}

// One block of up to 32 draws (tail of a row group); lanes >= nvalid consume
// nothing.  Reads reach k + 428 and writes start at k + 624: one barrier, after
// the writes.
template <int SLACK>
__device__ __forceinline__ uint32_t mt_single(uint32_t* B, int& iA, int lane, int nvalid, const MtMul& k) {
    mt_make_room<SLACK>(B, iA, 32, lane);
    const int i = iA + lane;
    const uint32_t a = B[i], b = B[i + 1], m = B[i + kMtM];
    const uint32_t v = mt_twist(a, b, m, k);
    if (lane < nvalid) B[i + kMtN] = v;
    __syncwarp();
    iA += nvalid;
    return mt_temper_mul(v, k);
}

// Logic phase for one word of colour c at row r = y + L z, word k (see the
// layout notes in isg_common.cuh), in two halves: word_load issues the loads of
// the word, its forward couplings and the other colour's neighbour words (and
// of the backward couplings there); word_compute counts the unsatisfied bonds,
// forms the flip mask from the draws' bit streams, writes the word and adds its
// dE to dEsum.  Between the two a warp can make the group's draws, so that the
// loads' latency is hidden behind generator work.
template <typename Word>
struct WordIn {
    size_t o;
    int p;
    Word s, na, jxc, jyc, jzc, syp, jym, sym, szp, jzm, szm, jxn, jxb, sb;
};

template <typename Word>
__device__ __forceinline__ void word_load(const FlipArgs& a, int c, int r, int y, int z, int k, WordIn<Word>& q) {
    const int L = a.L, W = a.W;
    const size_t pb = (size_t)a.plane_bytes;
    const Word* Sc = (const Word*)(a.planes + (size_t)(4 * c) * pb);
    const Word* Jxc = (const Word*)(a.planes + (size_t)(4 * c + 1) * pb);
    const Word* Jyc = (const Word*)(a.planes + (size_t)(4 * c + 2) * pb);
    const Word* Jzc = (const Word*)(a.planes + (size_t)(4 * c + 3) * pb);
    const int n = c ^ 1;
    const Word* Sn = (const Word*)(a.planes + (size_t)(4 * n) * pb);
    const Word* Jxn = (const Word*)(a.planes + (size_t)(4 * n + 1) * pb);
    const Word* Jyn = (const Word*)(a.planes + (size_t)(4 * n + 2) * pb);
    const Word* Jzn = (const Word*)(a.planes + (size_t)(4 * n + 3) * pb);

    q.p = (c + y + z) & 1;
    const int rowW = r * W;
    const int dym = (y == 0 ? L - 1 : -1) * W, dyp = (y == L - 1 ? 1 - L : 1) * W;
    const int LW = L * W;
    const int dzm = (z == 0 ? (L - 1) * LW : -LW), dzp = (z == L - 1 ? -(L - 1) * LW : LW);
    q.o = (size_t)(rowW + k);
    // the x neighbour word across the word boundary: k - 1 for p = 0, k + 1 for p = 1
    const size_t onb = (size_t)(rowW + (q.p == 0 ? (k == 0 ? W - 1 : k - 1) : (k == W - 1 ? 0 : k + 1)));
    const size_t o = q.o;
    q.s = Sc[o];
    q.na = Sn[o];
    q.jxc = Jxc[o];
    q.jyc = Jyc[o];
    q.jzc = Jzc[o];
    q.syp = Sn[o + dyp];
    q.jym = Jyn[o + dym];
    q.sym = Sn[o + dym];
    q.szp = Sn[o + dzp];
    q.jzm = Jzn[o + dzm];
    q.szm = Sn[o + dzm];
    q.jxn = Jxn[o];
    q.jxb = q.p == 0 ? Jxn[onb] : Word(0);
    q.sb = Sn[onb];
}

template <typename Word>
__device__ __forceinline__ void word_compute(const FlipArgs& a, int c, const WordIn<Word>& q, int k,
                                             const uint32_t* cond, int off, int& dEsum, int hi_off = kCondWords,
                                             int* usum = nullptr) {
    constexpr int w = 8 * sizeof(Word);
    const int W = a.W, nt = a.nt;
    Word* Sc = (Word*)(a.planes + (size_t)(4 * c) * (size_t)a.plane_bytes);
    const Word s = q.s, na = q.na;
    const Word e_yp = q.jyc ^ s ^ q.syp;
    const Word e_ym = q.jym ^ s ^ q.sym;
    const Word e_zp = q.jzc ^ s ^ q.szp;
    const Word e_zm = q.jzm ^ s ^ q.szm;
    Word e_xp, e_xm;
    if (q.p == 0) {
        e_xp = q.jxc ^ s ^ na;
        e_xm = row_down<Word>(q.jxn ^ na, q.jxb ^ q.sb, k, nt) ^ s;
    } else {
        e_xp = q.jxc ^ s ^ row_up<Word>(na, q.sb, k, W, nt);
        e_xm = q.jxn ^ s ^ na;
    }
    Word u0, u1, u2;
    Logic<Word>::count6(e_xp, e_xm, e_yp, e_ym, e_zp, e_zm, u0, u1, u2);
    const Word lo = take_bits<Word>(cond, off);
    const Word hi = take_bits<Word>(cond + hi_off, off);
    Word f = Logic<Word>::flip(u0, u1, u2, lo | hi, hi, lo & hi);
    const Word valid = (k == W - 1 && nt < w) ? (Word)((Word(1) << nt) - 1) : ~Word(0);
    f &= valid;
    Sc[q.o] = s ^ f;
    dEsum += Logic<Word>::dE(f, u0, u1, u2);
    // the pass's unsatisfied bonds before any flip: every bond has one site of
    // each colour, so their sum over one colour's sites is U of Eq. 1 (E = 2U - 3N)
    if (usum)
        *usum += Logic<Word>::popc(u0 & valid) + 2 * Logic<Word>::popc(u1 & valid) +
                 4 * Logic<Word>::popc(u2 & valid);
}

template <typename Word>
__device__ __forceinline__ void word_update(const FlipArgs& a, int c, int r, int y, int z, int k,
                                            const uint32_t* cond, int off, int& dEsum, int hi_off = kCondWords,
                                            int* usum = nullptr) {
    WordIn<Word> q;
    word_load<Word>(a, c, r, y, z, k, q);
    word_compute<Word>(a, c, q, k, cond, off, dEsum, hi_off, usum);
}

// Generator state of the stream a warp is working on.
struct StreamRegs {
    int pos;       // MT19937: position (mod 624) of the next draw in the stored ring
    int iA;        // MT19937: window index of x_k for the next draw k
    uint32_t xA;   // MINSTD: state of draw n + lane + 1; Parisi-Rapuano: ira[i-64+lane]
    uint32_t xB;   // MINSTD: state of draw n + lane + 33; Parisi-Rapuano: ira[i-32+lane]
};

// The stored MT19937 state is a 624-word ring with the position of the next
// draw; it is unrolled into the front of the window on load and rolled back on
// store, so the stored format does not depend on the window.
template <int KIND>
__device__ __forceinline__ void load_stream(const FlipArgs& a, int64_t t, uint32_t* B, StreamRegs& st,
                                            const StreamConst& k, int lane) {
    if (KIND == ISG_RNG_MT19937) {
        const int p = (int)a.rng_pos[t];
        for (int j = lane; j < kMtN; j += 32) {
            const int s = p + j >= kMtN ? p + j - kMtN : p + j;
            B[j] = a.rng[t * kMtN + s];
        }
        st.pos = p;
        st.iA = 0;
        __syncwarp();
    } else if (KIND == ISG_RNG_PARISI_RAPUANO) {
        pr_load(a.rng + t * kPrN, st.xA, st.xB, lane);
    } else {
        st.xA = minstd_mulmod(a.rng[t], a.mt.pow[lane + 1]);
        st.xB = minstd_mulmod(st.xA, k.a32);
    }
}

template <int KIND>
__device__ __forceinline__ void store_stream(const FlipArgs& a, int64_t t, const uint32_t* B,
                                             const StreamRegs& st, int lane) {
    if (KIND == ISG_RNG_MT19937) {
        __syncwarp();
        for (int j = lane; j < kMtN; j += 32) {
            const int s = st.pos + j >= kMtN ? st.pos + j - kMtN : st.pos + j;
            a.rng[t * kMtN + s] = B[st.iA + j];
        }
        if (lane == 0) a.rng_pos[t] = (uint32_t)st.pos;
        __syncwarp();
    } else if (KIND == ISG_RNG_PARISI_RAPUANO) {
        pr_store(a.rng + t * kPrN, st.xA, st.xB, lane);
    } else {
        const uint32_t x0 = __shfl_sync(kFull, st.xA, 0);
        if (lane == 0) a.rng[t] = minstd_mulmod(x0, a.mt.inv);  // state of the last draw used
    }
}

// The three compare values of a pass, held in registers: the batched engine
// reads its FlipArgs from global memory, where the compiler could not keep them
// across the shared-memory stores of the draw loop.
struct Cmp {
    uint32_t c1, c2, c3;
};

__device__ __forceinline__ Cmp cmp_of(const FlipArgs& a) { return Cmp{a.cmp1, a.cmp2, a.cmp3}; }

// Level of a draw against the nested thresholds, as the two ballot bits.
__device__ __forceinline__ bool level_lo(uint32_t d, const Cmp& a) {
    return (d < a.c1) ^ (d < a.c2) ^ (d < a.c3);
}

// The two ballots of N consecutive 32-draw blocks.
template <int N>
__device__ __forceinline__ void level_ballots(const uint32_t (&d)[N], const Cmp& a, uint32_t (&lo)[N],
                                              uint32_t (&hi)[N]) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
        lo[j] = __ballot_sync(kFull, level_lo(d[j], a));
        hi[j] = __ballot_sync(kFull, d[j] < a.c2);
    }
}

// Tempering, level ballots and condition-stream words of a seven-block step
// (raw words v, step q of the row group): lane j < 7 stores the ballots of
// block j.
__device__ __forceinline__ void seven_cond(const uint32_t (&v)[7], const Cmp& a, uint32_t* cond, int kCond, int q,
                                           const MtMul& k, int lane) {
    uint32_t d[7], lo[7], hi[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) d[j] = mt_temper_mul(v[j], k);
    level_ballots<7>(d, a, lo, hi);
    uint32_t l = lo[0], h = hi[0];
#pragma unroll
    for (int j = 1; j < 7; ++j)
        if (lane == j) {
            l = lo[j];
            h = hi[j];
        }
    if (lane < 7) {
        cond[7 * q + lane] = l;
        cond[kCond + 7 * q + lane] = h;
    }
}

// The throughput form of the ballots of a quad of blocks.  A draw below cmp2 has
// probability exp(-8 beta) (1.4e-4 at T = 0.9), so the warp first asks whether
// any of its 128 draws is below cmp2.  If none is, none is below cmp3 either,
// every level is 0 or 1, one comparison per draw gives it exactly and the hi
// ballots are all zero.  The extra vote lengthens the dependency chain of a
// step, so kernels whose warps are too few to hide latency do without it.
// 16-byte shared-memory store by lane 0 alone, as one predicated instruction
// (no divergent branch around it); `addr` is a shared-window address.
__device__ __forceinline__ void st_shared_lane0(uint32_t addr, uint32_t x, uint32_t y, uint32_t z, uint32_t w,
                                                int lane) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %5, 0;\n\t@p st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n\t}"
        :
        : "r"(addr), "r"(x), "r"(y), "r"(z), "r"(w), "r"(lane)
        : "memory");
}

// Four ballot words stored by lane 0: with PST as one predicated instruction
// (faster for MT19937, whose step has more shared-memory traffic), otherwise
// under a branch (faster for the register generators).  `p` and `s` are the
// generic and shared-window addresses of the same words.
template <bool PST>
__device__ __forceinline__ void store4_lane0(uint32_t* p, uint32_t s, const uint32_t (&v)[4], int lane) {
    if constexpr (PST) {
        st_shared_lane0(s, v[0], v[1], v[2], v[3], lane);
    } else {
        if (lane == 0) *(uint4*)p = make_uint4(v[0], v[1], v[2], v[3]);
    }
}

// Lane 0 stores the four lo ballots at lo and, only when the hi ballots are
// taken, the four hi ballots at hi (generic pointers, with lo_s and hi_s their
// shared-window addresses); returns whether it stored them.  The hi stream is
// otherwise left as it is (kept all zero by the caller).
template <bool PST>
__device__ __forceinline__ bool quad_ballots(const uint32_t (&d)[4], const Cmp& a, uint32_t* lo, uint32_t* hi,
                                             uint32_t lo_s, uint32_t hi_s, int lane) {
    const uint32_t dmin = min(min(d[0], d[1]), min(d[2], d[3]));
    if (__any_sync(kFull, dmin < a.c2)) {
        uint32_t l[4], h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            l[j] = __ballot_sync(kFull, level_lo(d[j], a));
            h[j] = __ballot_sync(kFull, d[j] < a.c2);
        }
        store4_lane0<PST>(lo, lo_s, l, lane);
        store4_lane0<PST>(hi, hi_s, h, lane);
        return true;
    }
    uint32_t l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) l[j] = __ballot_sync(kFull, d[j] < a.c1);
    store4_lane0<PST>(lo, lo_s, l, lane);
    return false;
}

// Zeroes the hi bit stream of the condition buffer (n words).
__device__ __forceinline__ void clear_hi(uint32_t* hi, int n, int lane) {
    for (int j = lane; j < n; j += 32) hi[j] = 0u;
}

// One pass of colour c over rows [r_begin, r_end) of a stream (all of its rows,
// or a segment that starts at a row group); the generator state, positioned at
// the first of these rows, is in B / st.  SLACK is the free space of the
// MT19937 window (see mt_window); TRIM selects the throughput form of the draw
// phase (quad_ballots; MINSTD four blocks per step) over the latency one
// (MINSTD two blocks per step, MT19937 seven, the word-update loads issued
// before the draws).  WPT is the number of words of a row group each lane
// updates: a group is WPT * 32 / W rows, and cond holds two bit streams of
// WPT * kCondWords words each.
template <typename Word, int KIND, int SLACK, bool TRIM, int WPT = 1>
__device__ __forceinline__ void stream_pass(const FlipArgs& a, int c, int64_t r_begin, int64_t r_end, uint32_t* B,
                                            uint32_t* cond, StreamRegs& st, const StreamConst& k, int lane,
                                            int& dEsum, int* usum = nullptr) {
    constexpr int w = 8 * sizeof(Word);
    constexpr bool kMT = KIND == ISG_RNG_MT19937;
    constexpr int kCond = WPT * kCondWords;
    const int W = a.W, half = a.half, L = a.L;
    const Cmp cm = cmp_of(a);
    const int G = WPT * 32 / W;
    const int lj = lane / W, lk = lane - lj * W;
    const int loff = lj * half + lk * w;
    int r = (int)r_begin + lj;
    int y = r % L, z = r / L;
    bool hiset = false;  // TRIM: the hi stream holds a nonzero word
    const uint32_t cond_s = (uint32_t)__cvta_generic_to_shared(cond);
    if (TRIM) {
        clear_hi(cond + kCond, kCond, lane);
        __syncwarp();
    }
    for (int64_t g0 = r_begin; g0 < r_end; g0 += G) {
        const int nrows = (int)((r_end - g0) < G ? (r_end - g0) : G);
        const int D = nrows * half;
        if (kMT) st.pos = (st.pos + D) % kMtN;  // the ring position after this group's draws
        // latency form: the group's plane words are loaded before its draws are made
        WordIn<Word> win;
        const bool act = lane < nrows * W;
        if (!TRIM && WPT == 1 && act) word_load<Word>(a, c, r, y, z, lk, win);
        // draws four 32-draw blocks per step (MINSTD without TRIM: two), then the
        // remaining blocks one by one
        int b = 0;  // 32-draw blocks of this group done so far
        if (kMT && !TRIM) {
            // software-pipelined: the twist of step q + 1 is made beside the
            // tempering and ballots of step q, two independent chains that one
            // warp per scheduler can interleave
            const int nsev = D / 224;
            if (nsev > 0) {
                uint32_t v[7];
                mt_seven_raw<SLACK>(B, st.iA, v, k.mul, lane);
                __syncwarp();
                for (int q = 0; q + 1 < nsev; ++q) {
                    uint32_t vn[7];
                    mt_seven_raw<SLACK>(B, st.iA, vn, k.mul, lane);
                    seven_cond(v, cm, cond, kCond, q, k.mul, lane);
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < 7; ++j) v[j] = vn[j];
                }
                seven_cond(v, cm, cond, kCond, nsev - 1, k.mul, lane);
            }
            b = 7 * nsev;
        } else if (KIND == ISG_RNG_MINSTD && !TRIM) {
            const int npairs = D >> 6;
            for (int q = 0; q < npairs; ++q) {
                uint32_t d[2] = {st.xA, st.xB}, lo[2], hi[2];
                st.xA = minstd_mulmod(st.xA, k.a64);
                st.xB = minstd_mulmod(st.xB, k.a64);
                level_ballots<2>(d, cm, lo, hi);
                if (lane == 0) {
                    *(uint2*)(cond + 2 * q) = make_uint2(lo[0], lo[1]);
                    *(uint2*)(cond + kCond + 2 * q) = make_uint2(hi[0], hi[1]);
                }
            }
            b = 2 * npairs;
        } else {
            // With TRIM the hi stream is kept all zero between groups and a quad
            // whose hi ballots were skipped stores nothing there.  MT19937 checks
            // its window once per run of quads that fit.
            const int nquads = D >> 7;
            for (int q = 0; q < nquads;) {
                int qe = nquads;
                if (kMT) {
                    mt_make_room<SLACK>(B, st.iA, 128, lane);
                    const int fit = q + ((mt_window(SLACK) - kMtN - st.iA) >> 7);
                    qe = fit < nquads ? fit : nquads;
                }
                for (; q < qe; ++q) {
                    uint32_t d[4];
                    if (kMT) {
                        mt_quad<SLACK, false>(B, st.iA, d, k.mul, lane);
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
                    if constexpr (TRIM) {
                        if (quad_ballots<kMT>(d, cm, cond + 4 * q, cond + kCond + 4 * q, cond_s + 16 * q,
                                              cond_s + 4 * kCond + 16 * q, lane))
                            hiset = true;
                    } else {
                        uint32_t lo[4], hi[4];
                        level_ballots<4>(d, cm, lo, hi);
                        if (lane == 0) {
                            *(uint4*)(cond + 4 * q) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                            *(uint4*)(cond + kCond + 4 * q) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                        }
                    }
                }
            }
            b = 4 * nquads;
        }
        for (int rem = D - 32 * b; rem > 0; rem -= 32, ++b) {
            const int nvalid = rem < 32 ? rem : 32;
            uint32_t d;
            if (kMT) {
                d = mt_single<SLACK>(B, st.iA, lane, nvalid, k.mul);
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
            const uint32_t lo = __ballot_sync(kFull, level_lo(d, cm));
            const uint32_t hi = __ballot_sync(kFull, d < cm.c2);
            hiset |= hi != 0u;
            if (lane == 0) {
                cond[b] = lo;
                cond[kCond + b] = hi;
            }
        }
        __syncwarp();
        if constexpr (WPT == 1) {
            if (act) {
                if (TRIM) word_update<Word>(a, c, r, y, z, lk, cond, loff, dEsum, kCondWords, usum);
                else word_compute<Word>(a, c, win, lk, cond, loff, dEsum, kCondWords, usum);
            }
        } else {
#pragma unroll
            for (int q = 0; q < WPT; ++q) {
                const int wi = lane + 32 * q;  // word of the group: row wi / W, word wi % W
                if (wi < nrows * W) {
                    const int jq = wi / W, kq = wi - jq * W;
                    const int rq = (int)g0 + jq;
                    word_update<Word>(a, c, rq, rq % L, rq / L, kq, cond, jq * half + kq * w, dEsum, kCond, usum);
                }
            }
        }
        __syncwarp();
        if (TRIM && hiset) {
            clear_hi(cond + kCond, kCond, lane);
            hiset = false;
            __syncwarp();
        }
        r += G;
        y += G;
        while (y >= L) {
            y -= L;
            ++z;
        }
    }
}

}  // namespace isg
