// isg_flip_fast.cu -- the production flip kernel behind isg_sweep.
//
// Same site -> (stream, draw) map, same bit logic and the same results, bit for
// bit, as the plain kernel of isg_flip.cu; the per-stream work is the shared
// stream_pass of isg_stream.cuh.  What changes is how the work is issued: the
// grid fills the GPU once and every warp takes stream after stream from a
// monotonically increasing ticket counter, so the last "wave" of streams is
// spread over all SMs instead of leaving most of them idle.
#include "isg_stream.cuh"

namespace isg {

constexpr int kFastWarps = 4;
constexpr int kFastSlack = 1024;  // MT19937 window: 624 live words + 1024 free (6.6 KiB per warp)

struct Tickets {
    unsigned long long* counter;  // device word, only ever incremented
    unsigned long long base;      // its value when this launch starts
};

template <typename Word, int KIND, bool TRIM>
__global__ void __launch_bounds__(kFastWarps * 32, KIND == ISG_RNG_MT19937 ? 7 : 8)
    flip_fast_kernel(FlipArgs a, StreamConst k, Tickets tk) {
    extern __shared__ uint32_t smem[];
    constexpr int kRing = KIND == ISG_RNG_MT19937 ? mt_window(kFastSlack) : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* ring = smem + wid * (kRing + 2 * kCondWords);
    uint32_t* cond = ring + kRing;
    int dEsum = 0;
    for (;;) {
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(tk.counter, 1ull);
        v = __shfl_sync(kFull, v, 0);
        const int64_t t = (int64_t)(v - tk.base);
        if (t >= a.S) break;
        StreamRegs st;
        load_stream<KIND>(a, t, ring, st, k, lane);
        stream_pass<Word, KIND, kFastSlack, TRIM>(a, a.c, t, ring, cond, st, k, lane, dEsum);
        store_stream<KIND>(a, t, ring, st, lane);
    }
    for (int sh = 16; sh; sh >>= 1) dEsum += __shfl_xor_sync(kFull, dEsum, sh);
    if (lane == 0 && dEsum != 0) atomicAdd((unsigned long long*)a.dE, (unsigned long long)(long long)dEsum);
}

// Streams per SM from which the throughput form of the draw phase (TRIM) is used:
// below it too few warps are resident to hide the longer dependency chain.
constexpr int64_t kTrimStreamsPerSM = 16;

template <typename Word, int KIND, bool TRIM>
static cudaError_t launch_fast_t(isg_sim* h, int colour, cudaStream_t s, int sms) {
    const FlipArgs a = make_flip_args(h, colour);
    const StreamConst k = stream_const();
    Tickets tk;
    tk.counter = (unsigned long long*)(h->scal + 3);
    tk.base = h->tickets;
    constexpr int kRing = KIND == ISG_RNG_MT19937 ? mt_window(kFastSlack) : 0;
    const size_t smem = (size_t)kFastWarps * (kRing + 2 * kCondWords) * sizeof(uint32_t);
    static int occ = 0;  // resident blocks per SM of this instantiation
    if (occ == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, flip_fast_kernel<Word, KIND, TRIM>,
                                                                      kFastWarps * 32, smem);
        if (e != cudaSuccess || occ < 1) occ = 1;
    }
    int64_t blocks = (int64_t)sms * occ;
    const int64_t need = (h->S + kFastWarps - 1) / kFastWarps;
    if (blocks > need) blocks = need;
    flip_fast_kernel<Word, KIND, TRIM><<<(unsigned)blocks, kFastWarps * 32, smem, s>>>(a, k, tk);
    const cudaError_t e = cudaGetLastError();
    // every warp takes one ticket past the last stream before it stops
    if (e == cudaSuccess) h->tickets += (unsigned long long)h->S + (unsigned long long)blocks * kFastWarps;
    return e;
}

cudaError_t launch_flip_fast(isg_sim* h, int colour, cudaStream_t s) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const bool trim = h->S >= kTrimStreamsPerSM * sms;
    return with_kind(h->kind, [&](auto kind) {
        constexpr int K = decltype(kind)::value;
        if (h->wbits == 64)
            return trim ? launch_fast_t<uint64_t, K, true>(h, colour, s, sms)
                        : launch_fast_t<uint64_t, K, false>(h, colour, s, sms);
        return trim ? launch_fast_t<uint32_t, K, true>(h, colour, s, sms)
                    : launch_fast_t<uint32_t, K, false>(h, colour, s, sms);
    });
}

}  // namespace isg
