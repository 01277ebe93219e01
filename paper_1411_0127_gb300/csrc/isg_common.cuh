// isg_common.cuh -- internal types and device helpers of the GB300 engine.
//
// Lattice layout (per colour c in {0 = red, 1 = blue}):
//   4 bit planes S_c, Jx_c, Jy_c, Jz_c, each rows = L*L rows of W words of
//   `wbits` bits.  Row r = y + L*z holds the L/2 sites of colour c with
//   x = 2h + p, p = (c + y + z) & 1, at bit h of the row (word h / wbits, bit
//   h % wbits).  Bits past L/2 in the last word are zero.  S bit = 1 means
//   s = +1; J bit = 1 means J = -1 (Sec. 4 bit map).  Jd_c holds the coupling
//   from a colour-c site to its +d neighbour, so the 3N couplings are stored
//   once; a site's -d coupling is the +d coupling of its -d neighbour.
#pragma once

#include <atomic>
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "isg.h"

namespace isg {

constexpr uint64_t kSaltCouplings = 0x6A09E667F3BCC908ull;
constexpr uint64_t kSaltSpins = 0xBB67AE8584CAA73Bull;
constexpr uint64_t kSaltStreams = 0x3C6EF372FE94F82Bull;
constexpr uint64_t kSaltHash = 0xA54FF53A5F1D36F1ull;

constexpr uint32_t kMinstdM = 2147483647u;  // 2^31 - 1
constexpr uint32_t kMinstdA = 16807u;

constexpr int kMtN = 624;   // MT19937 state words
constexpr int kMtM = 397;   // middle offset
constexpr int kPrN = 61;    // Parisi-Rapuano state words (the longest lag)
constexpr int kCondWords = 68;  // per condition plane: 2048 draw bits + padding
constexpr unsigned kFull = 0xFFFFFFFFu;

// SplitMix64 output n (n = 0, 1, ...) of the generator whose state starts at seed.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// x * c mod (2^31 - 1) for x, c in [0, 2^31 - 1): fold the 62-bit product once
// (2^31 = 1 mod M), r = (p mod 2^31) + (p >> 31) < 2^32, then one conditional
// subtraction.  On the device the fold takes three 32-bit multiplies and no
// 64-bit product: f = p >> 31 is the high word of x * 2c (2c < 2^32), and
// r = p mod 2^32 + f (1 - 2^31) mod 2^32, exact because r < 2^32; the
// subtraction is min(r, r - M) (r - M wraps above r when r < M).  L = 1024
// MINSTD 0.661 -> 0.607 ps per attempt, L = 256 1.254 -> 1.133.
__host__ __device__ __forceinline__ uint32_t minstd_mulmod(uint32_t x, uint32_t c) {
#ifdef __CUDA_ARCH__
    const uint32_t lo = x * c;
    const uint32_t f = __umulhi(x, c + c);
    const uint32_t r = lo + f * 0x80000001u;
    return min(r, r - kMinstdM);
#else
    uint64_t p = (uint64_t)x * (uint64_t)c;
    uint32_t r = (uint32_t)(p & kMinstdM) + (uint32_t)(p >> 31);
    return r >= kMinstdM ? r - kMinstdM : r;
#endif
}

// MT19937 tempering (Matsumoto & Nishimura 1998).
__device__ __forceinline__ uint32_t mt_temper(uint32_t v) {
    v ^= v >> 11;
    v ^= (v << 7) & 0x9D2C5680u;
    v ^= (v << 15) & 0xEFC60000u;
    v ^= v >> 18;
    return v;
}

// One warp-wide step of an MT19937 stream kept as a 624-word ring in shared
// memory: lane l produces draw k + l, i.e. x_{k+l+624} =
// x_{k+l+397} ^ twist(x_{k+l}, x_{k+l+1}); pos = k mod 624.  The inputs of a
// step are never outputs of the same step (397 + 31 < 624, 31 < 397), so one
// read phase, a warp barrier and one write phase suffice.  Only the first
// `nvalid` lanes consume (and store) a draw.
__device__ __forceinline__ uint32_t mt_warp_step(uint32_t* ring, int& pos, int lane, int nvalid) {
    int i = pos + lane;
    i = i >= kMtN ? i - kMtN : i;
    int i1 = i + 1;
    i1 = i1 >= kMtN ? i1 - kMtN : i1;
    int im = i + kMtM;
    im = im >= kMtN ? im - kMtN : im;
    const uint32_t a = ring[i], b = ring[i1], m = ring[im];
    __syncwarp();
    const uint32_t y = (a & 0x80000000u) | (b & 0x7FFFFFFFu);
    const uint32_t v = m ^ (y >> 1) ^ ((0u - (b & 1u)) & 0x9908B0DFu);
    if (lane < nvalid) ring[i] = v;
    __syncwarp();
    pos += nvalid;
    pos = pos >= kMtN ? pos - kMtN : pos;
    return mt_temper(v);
}

// MINSTD jump-ahead table: pow[j] = 16807^j mod (2^31 - 1), j = 0..32, plus
// the inverse of 16807.  Filled on the host, passed by value to the kernels.
struct MinstdTable {
    uint32_t pow[33];
    uint32_t inv;
};
MinstdTable minstd_table();

// Arguments of one colour pass of the flip kernels.
struct FlipArgs {
    unsigned char* planes;
    int64_t plane_bytes;
    int L, half, W, nt, c;
    int64_t R, S, rows;
    uint32_t thr1, thr2, thr3;
    uint32_t cmp1, cmp2, cmp3;   // compared with the generator value: thr_k, for MINSTD ceil(thr_k / 2)
    uint32_t* rng;
    uint32_t* rng_pos;
    long long* dE;
    MinstdTable mt;
};

// One warp-wide step of a MINSTD stream: lane j holds x_{n+j+1}; returns the
// draw 2*x and moves every lane forward by nvalid positions (a32 = 16807^32).
__device__ __forceinline__ uint32_t minstd_warp_step(uint32_t& x, uint32_t a32, int nvalid, int lane) {
    const uint32_t d = x << 1;
    const uint32_t y = minstd_mulmod(x, a32);
    if (nvalid == 32) {
        x = y;
    } else {
        const int src = lane + nvalid;
        const uint32_t xa = __shfl_sync(kFull, x, src & 31);
        const uint32_t ya = __shfl_sync(kFull, y, src & 31);
        x = src < 32 ? xa : ya;
    }
    return d;
}

// Parisi-Rapuano (Sec. 3): ira[i] = ira[i-24] + ira[i-55] (mod 2^32), draw
// R = ira[i] ^ ira[i-61].  A warp keeps ira[i-64 .. i-1] in two registers per
// lane, a = ira[i-64+l] and b = ira[i-32+l]; lane l makes draw i + l.  Lanes
// 0..23 find both lags in the registers; lanes 24..31 need ira[i+l-24], made
// by lane l-24 in the same step.  Moves every lane forward by nvalid draws.
__device__ __forceinline__ uint32_t pr_warp_step(uint32_t& a, uint32_t& b, int lane, int nvalid) {
    const int s3 = (lane + 3) & 31, s8 = (lane + 8) & 31, s9 = (lane + 9) & 31;
    const uint32_t lag24 = __shfl_sync(kFull, b, s8);
    const uint32_t a9 = __shfl_sync(kFull, a, s9), b9 = __shfl_sync(kFull, b, s9);
    const uint32_t a3 = __shfl_sync(kFull, a, s3), b3 = __shfl_sync(kFull, b, s3);
    const uint32_t lag55 = lane < 23 ? a9 : b9;   // ira[i+l-55]
    const uint32_t lag61 = lane < 29 ? a3 : b3;   // ira[i+l-61]
    const uint32_t v0 = lag24 + lag55;
    const uint32_t v1 = __shfl_sync(kFull, v0, s8) + lag55;
    const uint32_t v = lane < 24 ? v0 : v1;       // ira[i+l]
    if (nvalid == 32) {
        a = b;
        b = v;
    } else {
        const int src = (lane + nvalid) & 31;
        const bool up = lane + nvalid >= 32;
        const uint32_t as = __shfl_sync(kFull, a, src), bs = __shfl_sync(kFull, b, src);
        const uint32_t vs = __shfl_sync(kFull, v, src);
        a = up ? bs : as;
        b = up ? vs : bs;
    }
    return v ^ lag61;
}

// The stored Parisi-Rapuano state of a stream is ira[i-61 .. i-1], oldest
// first (61 words); lanes 0..2 of `a` hold words that are never read.
__device__ __forceinline__ void pr_load(const uint32_t* st, uint32_t& a, uint32_t& b, int lane) {
    a = lane >= 3 ? st[lane - 3] : 0u;
    b = st[29 + lane];
}

__device__ __forceinline__ void pr_store(uint32_t* st, uint32_t a, uint32_t b, int lane) {
    if (lane >= 3) st[lane - 3] = a;
    st[29 + lane] = b;
}

// Words of stored state per stream.
__host__ __device__ constexpr int rng_state_words(int kind) {
    return kind == ISG_RNG_MT19937 ? kMtN : (kind == ISG_RNG_PARISI_RAPUANO ? kPrN : 1);
}

inline bool rng_kind_valid(int kind) {
    return kind == ISG_RNG_MINSTD || kind == ISG_RNG_MT19937 || kind == ISG_RNG_PARISI_RAPUANO;
}

// Host dispatch on the generator kind: f(std::integral_constant<int, KIND>).
template <class F>
inline auto with_kind(int kind, F&& f) {
    if (kind == ISG_RNG_MT19937) return f(std::integral_constant<int, ISG_RNG_MT19937>{});
    if (kind == ISG_RNG_PARISI_RAPUANO) return f(std::integral_constant<int, ISG_RNG_PARISI_RAPUANO>{});
    return f(std::integral_constant<int, ISG_RNG_MINSTD>{});
}

// ---------------------------------------------------------------------------
// Bit-sliced stencil logic (Sec. 4, with the reading dE = 12 - 4u): e_k = 1 marks
// an unsatisfied bond; u = sum of the six e bits as three bit planes.
template <typename Word>
struct Logic {
    __device__ __forceinline__ static void count6(Word e1, Word e2, Word e3, Word e4, Word e5, Word e6,
                                                  Word& u0, Word& u1, Word& u2) {
        const Word s1 = e1 ^ e2 ^ e3;
        const Word c1 = (e1 & e2) | (e3 & (e1 ^ e2));
        const Word s2 = e4 ^ e5 ^ e6;
        const Word c2 = (e4 & e5) | (e6 & (e4 ^ e5));
        u0 = s1 ^ s2;
        const Word c3 = s1 & s2;
        u1 = c1 ^ c2 ^ c3;
        u2 = (c1 & c2) | (c3 & (c1 ^ c2));
    }
    // flip when u >= 3 (dE <= 0), or u = 2 and d < thr[1], u = 1 and d < thr[2],
    // u = 0 and d < thr[3]; c4, c8, c12 are those three comparisons.
    __device__ __forceinline__ static Word flip(Word u0, Word u1, Word u2, Word c4, Word c8, Word c12) {
        const Word low = (u0 & c8) | (~u0 & c12);
        return u2 | (u1 & (u0 | c4)) | (~u1 & low);
    }
    // sum of dE = 12 - 4u over the flipped bits
    __device__ __forceinline__ static int dE(Word f, Word u0, Word u1, Word u2) {
        return 12 * popc(f) - 4 * (popc(f & u0) + 2 * popc(f & u1) + 4 * popc(f & u2));
    }
    __device__ __forceinline__ static int popc(Word v);
};
template <>
__device__ __forceinline__ int Logic<uint32_t>::popc(uint32_t v) { return __popc(v); }
template <>
__device__ __forceinline__ int Logic<uint64_t>::popc(uint64_t v) { return __popcll(v); }

// Take `bits`-wide window starting at bit `off` of a packed 32-bit bit array.
__device__ __forceinline__ uint32_t take_bits32(const uint32_t* pl, int off) {
    const int q = off >> 5, sh = off & 31;
    return __funnelshift_r(pl[q], pl[q + 1], sh);
}
template <typename Word>
__device__ __forceinline__ Word take_bits(const uint32_t* pl, int off);
template <>
__device__ __forceinline__ uint32_t take_bits<uint32_t>(const uint32_t* pl, int off) {
    return take_bits32(pl, off);
}
template <>
__device__ __forceinline__ uint64_t take_bits<uint64_t>(const uint32_t* pl, int off) {
    return (uint64_t)take_bits32(pl, off) | ((uint64_t)take_bits32(pl, off + 32) << 32);
}

// Row neighbours along x.  up(): bit h of the result is bit h+1 of the row (the
// last valid bit wraps to bit 0 of word 0); down(): bit h is bit h-1 (bit 0
// wraps to the last valid bit).  `nb` is word k+1 (k-1) of the same row, or
// word 0 (W-1) at the wrap; nt = valid bits of the last word.
template <typename Word>
__device__ __forceinline__ Word row_up(Word cur, Word nb, int k, int W, int nt) {
    constexpr int w = 8 * sizeof(Word);
    const Word in = (k < W - 1) ? (Word)(nb << (w - 1)) : (Word)((nb & (Word)1) << (nt - 1));
    return (cur >> 1) | in;
}
template <typename Word>
__device__ __forceinline__ Word row_down(Word cur, Word nb, int k, int nt) {
    constexpr int w = 8 * sizeof(Word);
    const Word in = (k > 0) ? (Word)(nb >> (w - 1)) : (Word)((nb >> (nt - 1)) & (Word)1);
    return (Word)(cur << 1) | in;
}

}  // namespace isg

// ---------------------------------------------------------------------------
// The opaque handle.
struct isg_sim {
    int L = 0, half = 0, wbits = 0, W = 0, nt = 0;
    bool member = false;                // batch member or batched server job: 64-bit words whatever L,
                                        // no segmented streams
    int kind = 0;
    double beta = 0.0;
    uint32_t thr[4] = {0, 0, 0, 0};
    uint64_t seed_J = 0, seed_spin = 0, seed_rng = 0;  // seed_rng seeds the RNG streams
    int64_t rows = 0, R = 0, S = 0;
    int64_t plane_bytes = 0;            // one plane: rows * W * wbits / 8
    unsigned char* planes = nullptr;    // 8 planes: index 4*c + q, q = S, Jx, Jy, Jz
    uint32_t* rng = nullptr;            // MT: S * 624 ring words; MINSTD: S states
    uint32_t* rng_pos = nullptr;        // MT: S ring positions
    uint32_t* rng_alt = nullptr;        // MINSTD: the other state buffer of segmented passes (see isg_flip_fast.cu)
    long long* scal = nullptr;          // [0] tracked dE, [1] scratch sum, [2] hash, [3] stream tickets,
                                        // [4] energy word of isg_exchange_async, [5] error word (a bounded
                                        // wait of a multi-pass launch gave up)
    unsigned long long* done = nullptr; // per stream: colour passes completed by multi-pass launches (not
                                        // for batch members)
    unsigned long long passes = 0;      // colour passes of all multi-pass launches so far
    bool stall_next = false;            // testing: the next multi-pass launch's pass-1 waits never end
    uint32_t* stage = nullptr;          // packed-spin staging buffer of isg_exchange_async (made on first use)
    unsigned long long tickets = 0;     // value of the stream-ticket counter before the next launch
    int64_t E0 = 0;                     // energy when tracking (re)started
    int64_t sweeps = 0;
    cudaStream_t last_stream = nullptr;
    void* (*alloc)(size_t, void*) = nullptr;
    void (*free_fn)(void*, void*) = nullptr;
    void* alloc_ctx = nullptr;

    unsigned char* plane(int c, int q) const { return planes + (size_t)(4 * c + q) * (size_t)plane_bytes; }
};

namespace isg {
// Per-device launch facts.  A process may drive several devices, so SM counts
// and occupancies are cached per device ordinal (up to kDeviceSlots devices;
// beyond that they are queried on every call).
constexpr int kDeviceSlots = 64;
int current_device();   // cudaGetDevice, 0 if it fails
int sm_count();         // SMs of the current device

// Resident blocks per SM of `kernel` with the given block shape on the current
// device, looked up once per device in `cache` (one array per instantiation).
template <class Kernel>
int occupancy_cached(std::atomic<int> (&cache)[kDeviceSlots], Kernel kernel, int threads, size_t smem) {
    const int dev = current_device();
    if (dev < kDeviceSlots) {
        const int v = cache[dev].load(std::memory_order_relaxed);
        if (v > 0) return v;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    if (dev < kDeviceSlots) cache[dev].store(occ, std::memory_order_relaxed);
    return occ;
}

// Host-side helpers shared by the .cu files of the library.
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
void* dev_alloc(isg_sim* h, size_t n);
void dev_free(isg_sim* h, void* p);
int create_sim(int L, uint64_t seed_J, uint64_t seed_spin, uint64_t seed_rng, double beta, int rng_kind, bool member,
               isg_sim** out);
void destroy_sim(isg_sim* h);
size_t sim_device_bytes(int L, int rng_kind, bool member);
// floor(2^32 exp(-4 k beta)) for k = 1..3, thr[0] = 0 (Sec. 4)
void thresholds(double beta, uint32_t thr[4]);

// kernels (launchers) implemented in the .cu files
cudaError_t launch_init_planes(isg_sim* h, cudaStream_t s);
cudaError_t launch_init_rng(isg_sim* h, cudaStream_t s);
FlipArgs make_flip_args(isg_sim* h, int colour);
cudaError_t launch_flip_plain(isg_sim* h, int colour, cudaStream_t s);
// usum (may be NULL): a device word that receives the pass's count of
// unsatisfied bonds before its flips (U of Eq. 1, E = 2U - 3N)
cudaError_t launch_flip_fast(isg_sim* h, int colour, cudaStream_t s, unsigned long long* usum = nullptr);
// n full sweeps as persistent launches of up to 64 sweeps each (isg_flip_fast.cu):
// only where sweeps_in_one_launch(h, n) holds (enough streams, n >= 8)
bool sweeps_in_one_launch(const isg_sim* h, int64_t n);
cudaError_t launch_sweeps(isg_sim* h, int64_t n, cudaStream_t s);
cudaError_t launch_energy(const isg_sim* h, long long* out, cudaStream_t s);
cudaError_t launch_overlap(const isg_sim* a, const isg_sim* b, long long* out, cudaStream_t s);
cudaError_t launch_hash(const isg_sim* h, unsigned long long* out, cudaStream_t s);
// spin I/O (isg_spinio.cu): int8 +-1 and packed bits in site order
cudaError_t launch_unpack_spins_fast(const isg_sim* h, int8_t* dev_out, cudaStream_t s);
cudaError_t launch_pack_spins_checked(const isg_sim* h, const int8_t* dev_in, unsigned char* dev_scratch, int* dev_bad,
                                      cudaStream_t s);
cudaError_t launch_unpack_spins_bits(const isg_sim* h, uint32_t* dev_out, cudaStream_t s);
cudaError_t launch_pack_spins_bits(isg_sim* h, const uint32_t* dev_in, cudaStream_t s);
cudaError_t launch_unpack_couplings(const isg_sim* h, int8_t* dev_out, cudaStream_t s);
cudaError_t launch_pack_couplings(isg_sim* h, const int8_t* dev_in, cudaStream_t s);
cudaError_t launch_check_pm1(const int8_t* dev_in, int64_t n, int* dev_bad, cudaStream_t s);
cudaError_t launch_peek_draws(const isg_sim* h, int64_t t, int64_t n, uint32_t* dev_out, cudaStream_t s);
cudaError_t launch_stencil(const uint16_t* code, const uint32_t* draw, int64_t n, uint32_t t1,
                           uint32_t t2, uint32_t t3, uint8_t* flip, uint8_t* u, cudaStream_t s);
}  // namespace isg
