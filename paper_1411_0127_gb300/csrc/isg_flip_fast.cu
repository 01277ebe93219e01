// isg_flip_fast.cu -- the production flip kernel behind isg_sweep.
//
// Same site -> (stream, draw) map, same bit logic and same results, bit for bit,
// as the plain kernel of isg_flip.cu; what changes is how the work is issued:
//   * persistent warps: the grid fills the GPU once and every warp takes stream
//     after stream from a monotonically increasing ticket counter, so the last
//     "wave" of streams is spread over all SMs;
//   * draws are produced 64 at a time (two 32-lane blocks with independent
//     dependency chains, one pair of warp barriers per 64 draws);
//   * MT19937 keeps its 624 words twice in shared memory (slot s and s + 624
//     hold the same word), so x_{k+1} and x_{k+397} are read at fixed offsets
//     from one index without wrap-around arithmetic;
//   * MINSTD keeps two lanes' worth of states (positions +1..+32 and +33..+64)
//     and compares the state x itself with ceil(thr / 2) (d = 2x < thr <=> x <
//     ceil(thr / 2)), saving the doubling;
//   * row coordinates advance incrementally instead of by integer division.
#include "isg_common.cuh"

namespace isg {

constexpr int kFastWarps = 4;

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
__device__ __forceinline__ void word_update(const FlipArgs& a, int r, int y, int z, int k, const uint32_t* cond,
                                            int off, int& dEsum) {
    constexpr int w = 8 * sizeof(Word);
    const int c = a.c, L = a.L, W = a.W, nt = a.nt;
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

struct FastExtra {
    unsigned long long* tickets;  // stream-ticket counter (device)
    unsigned long long base;      // its value when this launch starts
    uint32_t c1, c2, c3;          // compared thresholds (MT: thr; MINSTD: ceil(thr/2))
    uint32_t a64;                 // 16807^64 mod (2^31 - 1)
    MtMul mul;
};

template <typename Word, int KIND>
__global__ void __launch_bounds__(kFastWarps * 32, 8) flip_fast_kernel(FlipArgs a, FastExtra x) {
    extern __shared__ uint32_t smem[];
    constexpr int w = 8 * sizeof(Word);
    constexpr bool kMT = KIND == ISG_RNG_MT19937;
    constexpr int kRing = kMT ? 2 * kMtN : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* ring = smem + wid * (kRing + 3 * kCondWords);
    uint32_t* cond = ring + kRing;
    const int W = a.W, half = a.half, L = a.L;
    const int G = 32 / W;
    const int lj = lane / W, lk = lane - lj * W;
    const int loff = lj * half + lk * w;
    const uint32_t a32 = a.mt.pow[32];
    int dEsum = 0;

    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(x.tickets, 1ull);
        tk = __shfl_sync(kFull, tk, 0);
        const int64_t t = (int64_t)(tk - x.base);
        if (t >= a.S) break;

        int iA = 0;
        uint32_t xA = 0, xB = 0;
        if (kMT) {
            for (int i = lane; i < kMtN; i += 32) {
                const uint32_t v = a.rng[t * kMtN + i];
                ring[i] = v;
                ring[i + kMtN] = v;
            }
            iA = (int)a.rng_pos[t] + lane;
            iA = iA >= kMtN ? iA - kMtN : iA;
            __syncwarp();
        } else {
            xA = minstd_mulmod(a.rng[t], a.mt.pow[lane + 1]);
            xB = minstd_mulmod(xA, a32);
        }

        const int64_t r_begin = t * a.R;
        const int64_t r_end = r_begin + a.R < a.rows ? r_begin + a.R : a.rows;
        int r = (int)r_begin + lj;
        int y = r % L, z = r / L;
        for (int64_t g0 = r_begin; g0 < r_end; g0 += G) {
            const int nrows = (int)((r_end - g0) < G ? (r_end - g0) : G);
            const int D = nrows * half;
            const int npairs = D >> 6;
            for (int q = 0; q < npairs; ++q) {
                uint32_t dA, dB;
                if (kMT) {
                    mt_pair(ring, iA, dA, dB, x.mul);
                } else {
                    dA = xA;
                    dB = xB;
                    xA = minstd_mulmod(xA, x.a64);
                    xB = minstd_mulmod(xB, x.a64);
                }
                const uint32_t A4 = __ballot_sync(kFull, dA < x.c1), B4 = __ballot_sync(kFull, dB < x.c1);
                const uint32_t A8 = __ballot_sync(kFull, dA < x.c2), B8 = __ballot_sync(kFull, dB < x.c2);
                const uint32_t A12 = __ballot_sync(kFull, dA < x.c3), B12 = __ballot_sync(kFull, dB < x.c3);
                if (lane == 0) {
                    *(uint2*)(cond + 2 * q) = make_uint2(A4, B4);
                    *(uint2*)(cond + kCondWords + 2 * q) = make_uint2(A8, B8);
                    *(uint2*)(cond + 2 * kCondWords + 2 * q) = make_uint2(A12, B12);
                }
            }
            int rem = D - (npairs << 6);
            int b = 2 * npairs;
            while (rem > 0) {
                const int nvalid = rem < 32 ? rem : 32;
                uint32_t d;
                if (kMT) {
                    d = mt_single(ring, iA, lane, nvalid, x.mul);
                } else {
                    d = xA;
                    const int src = lane + nvalid;
                    const uint32_t pa = __shfl_sync(kFull, xA, src & 31);
                    const uint32_t pb = __shfl_sync(kFull, xB, src & 31);
                    xA = src < 32 ? pa : pb;
                    xB = minstd_mulmod(xA, a32);
                }
                const uint32_t m4 = __ballot_sync(kFull, d < x.c1);
                const uint32_t m8 = __ballot_sync(kFull, d < x.c2);
                const uint32_t m12 = __ballot_sync(kFull, d < x.c3);
                if (lane == 0) {
                    cond[b] = m4;
                    cond[kCondWords + b] = m8;
                    cond[2 * kCondWords + b] = m12;
                }
                ++b;
                rem -= nvalid;
            }
            __syncwarp();
            if (lane < nrows * W) word_update<Word>(a, r, y, z, lk, cond, loff, dEsum);
            __syncwarp();
            r += G;
            y += G;
            while (y >= L) {
                y -= L;
                ++z;
            }
        }

        if (kMT) {
            for (int i = lane; i < kMtN; i += 32) a.rng[t * kMtN + i] = ring[i];
            const int pos = __shfl_sync(kFull, iA, 0);
            if (lane == 0) a.rng_pos[t] = (uint32_t)pos;
            __syncwarp();
        } else {
            const uint32_t x0 = __shfl_sync(kFull, xA, 0);
            if (lane == 0) a.rng[t] = minstd_mulmod(x0, a.mt.inv);  // state of the last draw used
        }
    }
    for (int sh = 16; sh; sh >>= 1) dEsum += __shfl_xor_sync(kFull, dEsum, sh);
    if (lane == 0 && dEsum != 0) atomicAdd((unsigned long long*)a.dE, (unsigned long long)(long long)dEsum);
}

template <typename Word, int KIND>
static cudaError_t launch_fast_t(isg_sim* h, int colour, cudaStream_t s) {
    const FlipArgs a = make_flip_args(h, colour);
    FastExtra x;
    x.tickets = (unsigned long long*)(h->scal + 3);
    x.base = h->tickets;
    if (KIND == ISG_RNG_MT19937) {
        x.c1 = h->thr[1];
        x.c2 = h->thr[2];
        x.c3 = h->thr[3];
    } else {
        x.c1 = (uint32_t)(((uint64_t)h->thr[1] + 1) / 2);
        x.c2 = (uint32_t)(((uint64_t)h->thr[2] + 1) / 2);
        x.c3 = (uint32_t)(((uint64_t)h->thr[3] + 1) / 2);
    }
    x.a64 = minstd_mulmod(a.mt.pow[32], a.mt.pow[32]);
    x.mul.hi31 = 1u << 31;
    x.mul.hi21 = 1u << 21;
    x.mul.hi14 = 1u << 14;
    x.mul.lo7 = 1u << 7;
    x.mul.lo15 = 1u << 15;
    constexpr int kRing = KIND == ISG_RNG_MT19937 ? 2 * kMtN : 0;
    const size_t smem = (size_t)kFastWarps * (kRing + 3 * kCondWords) * sizeof(uint32_t);
    static int sms = 0;
    static int per_sm[2][2] = {{0, 0}, {0, 0}};
    int& occ = per_sm[sizeof(Word) == 8][KIND];
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (occ == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, flip_fast_kernel<Word, KIND>,
                                                                      kFastWarps * 32, smem);
        if (e != cudaSuccess || occ < 1) occ = 1;
    }
    int64_t blocks = (int64_t)sms * occ;
    const int64_t need = (h->S + kFastWarps - 1) / kFastWarps;
    if (blocks > need) blocks = need;
    flip_fast_kernel<Word, KIND><<<(unsigned)blocks, kFastWarps * 32, smem, s>>>(a, x);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) h->tickets += (unsigned long long)h->S + (unsigned long long)blocks * kFastWarps;
    return e;
}

cudaError_t launch_flip_fast(isg_sim* h, int colour, cudaStream_t s) {
    if (h->wbits == 64)
        return h->kind == ISG_RNG_MT19937 ? launch_fast_t<uint64_t, ISG_RNG_MT19937>(h, colour, s)
                                          : launch_fast_t<uint64_t, ISG_RNG_MINSTD>(h, colour, s);
    return h->kind == ISG_RNG_MT19937 ? launch_fast_t<uint32_t, ISG_RNG_MT19937>(h, colour, s)
                                      : launch_fast_t<uint32_t, ISG_RNG_MINSTD>(h, colour, s);
}

}  // namespace isg
