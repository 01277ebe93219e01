// isg_rngbench.cu -- device-API benchmark of the generator engines (Sec. 3,
// Table MYTEST: generate many numbers on the device and count the odd ones).
//
// `streams` streams of one kind are seeded exactly like the streams of a lattice
// (v_t = SplitMix64(seed ^ K_R, t); MT19937 init_genrand((uint32) v_t), MINSTD
// x_0 = 1 + v_t mod (2^31 - 2); Parisi-Rapuano ira[j] = SplitMix64(v_t, j) >> 32).
// Each warp then produces n consecutive raw outputs of its stream with the same
// engines the flip kernels use (MT19937: tempered word; MINSTD: the state x
// itself; Parisi-Rapuano: ira[i] ^ ira[i-61]) and counts the odd ones.
#include "isg_stream.cuh"

namespace isg {

constexpr int kBenchWarps = 4;
constexpr int kBenchSlack = 1024;

template <int KIND>
__global__ void __launch_bounds__(kBenchWarps * 32) rng_odd_kernel(const uint32_t* state, int64_t streams, int64_t n,
                                                                   MinstdTable mt, StreamConst k,
                                                                   unsigned long long* odd) {
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* B = smem + wid * mt_window(kBenchSlack);
    unsigned long long cnt = 0;
    for (int64_t t = (int64_t)blockIdx.x * kBenchWarps + wid; t < streams; t += (int64_t)gridDim.x * kBenchWarps) {
        int iA = 0;
        uint32_t xA = 0, xB = 0;
        if (KIND == ISG_RNG_MT19937) {
            for (int j = lane; j < kMtN; j += 32) B[j] = state[t * kMtN + j];
            __syncwarp();
        } else if (KIND == ISG_RNG_PARISI_RAPUANO) {
            pr_load(state + t * kPrN, xA, xB, lane);
        } else {
            xA = minstd_mulmod(state[t], mt.pow[lane + 1]);
            xB = minstd_mulmod(xA, k.a32);
        }
        int64_t done = 0;
        if (KIND == ISG_RNG_MT19937) {
            for (; done + 128 <= n; done += 128) {
                uint32_t d[4];
                mt_quad<kBenchSlack>(B, iA, d, k.mul, lane);
#pragma unroll
                for (int j = 0; j < 4; ++j) cnt += __popc(__ballot_sync(kFull, d[j] & 1u));
            }
            for (; done < n; done += 32) {
                const int nvalid = n - done < 32 ? (int)(n - done) : 32;
                const uint32_t d = mt_single<kBenchSlack>(B, iA, lane, nvalid, k.mul);
                cnt += __popc(__ballot_sync(kFull, (d & 1u) && lane < nvalid));
            }
        } else if (KIND == ISG_RNG_PARISI_RAPUANO) {
            for (; done + 128 <= n; done += 128) {
#pragma unroll
                for (int j = 0; j < 4; ++j) cnt += __popc(__ballot_sync(kFull, pr_warp_step(xA, xB, lane, 32) & 1u));
            }
            for (; done < n; done += 32) {
                const int nvalid = n - done < 32 ? (int)(n - done) : 32;
                const uint32_t d = pr_warp_step(xA, xB, lane, nvalid);
                cnt += __popc(__ballot_sync(kFull, (d & 1u) && lane < nvalid));
            }
        } else {
            for (; done + 64 <= n; done += 64) {
                cnt += __popc(__ballot_sync(kFull, xA & 1u)) + __popc(__ballot_sync(kFull, xB & 1u));
                xA = minstd_mulmod(xA, k.a64);
                xB = minstd_mulmod(xB, k.a64);
            }
            for (; done < n; done += 32) {
                const int nvalid = n - done < 32 ? (int)(n - done) : 32;
                cnt += __popc(__ballot_sync(kFull, (xA & 1u) && lane < nvalid));
                xA = xB;
                xB = minstd_mulmod(xA, k.a32);
            }
        }
        __syncwarp();
    }
    if (lane == 0 && cnt) atomicAdd(odd, cnt);
}

}  // namespace isg

using namespace isg;

extern "C" int isg_rng_count_odd(int rng_kind, uint64_t seed, int64_t streams, int64_t n, uint64_t* odd,
                                 double* gen_ms) {
    if (!odd || streams < 1 || n < 0 || !rng_kind_valid(rng_kind)) {
        set_error("isg_rng_count_odd: bad argument");
        return ISG_ERR_ARG;
    }
    const size_t words = (size_t)streams * rng_state_words(rng_kind);
    uint32_t *state = nullptr, *pos = nullptr;
    unsigned long long* dodd = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&state, words * 4);
    if (e == cudaSuccess) e = cudaMalloc(&pos, (size_t)streams * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dodd, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(dodd, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        isg_sim tmp;  // only the fields the seeding kernel reads
        tmp.kind = rng_kind;
        tmp.seed_rng = seed;
        tmp.S = streams;
        tmp.rng = state;
        tmp.rng_pos = pos;
        e = launch_init_rng(&tmp, 0);
        tmp.rng = nullptr;
        tmp.rng_pos = nullptr;
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
        const MinstdTable mt = minstd_table();
        const StreamConst k = stream_const();
        const size_t smem = rng_kind == ISG_RNG_MT19937 ? (size_t)kBenchWarps * mt_window(kBenchSlack) * 4 : 0;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t need = (streams + kBenchWarps - 1) / kBenchWarps;
        const unsigned grid = (unsigned)(need < (int64_t)sms * 16 ? need : (int64_t)sms * 16);
        cudaEventRecord(e0, 0);
        e = with_kind(rng_kind, [&](auto kc) {
            rng_odd_kernel<decltype(kc)::value><<<grid, kBenchWarps * 32, smem, 0>>>(state, streams, n, mt, k, dodd);
            return cudaGetLastError();
        });
        cudaEventRecord(e1, 0);
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, dodd, sizeof h, cudaMemcpyDeviceToHost);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaFree(state);
    cudaFree(pos);
    cudaFree(dodd);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "isg_rng_count_odd");
    *odd = h;
    if (gen_ms) *gen_ms = ms;
    return ISG_OK;
}

// ---------------------------------------------------------------------------
// Integer issue-rate microbenchmark (the denominators of the flip kernel's
// roofline): every thread runs 8 independent chains for `iters` steps; a step
// of a chain is one three-input logic operation (LOP3), one integer
// multiply-add (IMAD), or one of each.  The chains feed each other's operands
// so that nothing folds, and their XOR is written out so that nothing is
// dropped.  Ops counted: chains x steps x (1 or 2) per thread.
namespace isg {

template <int MODE>
__global__ void __launch_bounds__(256) int_rate_kernel(uint32_t seed, int iters, uint32_t* out) {
    uint32_t a[8], b[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        a[j] = seed ^ (threadIdx.x * 0x9E3779B9u + j);
        b[j] = seed + (blockIdx.x * 0x85EBCA6Bu) + 3 * j;
    }
    const uint32_t m = seed | 0x01000193u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (MODE != 2) a[j] = (a[j] & b[(j + 1) & 7]) ^ b[j];    // one LOP3
            if (MODE != 1) b[j] = b[j] * m + a[(j + 3) & 7];         // one IMAD
            if (MODE == 1) b[j] = (b[j] | a[(j + 5) & 7]) ^ a[j];    // LOP3 only: a second LOP3
            if (MODE == 2) a[j] = a[j] * m + b[(j + 5) & 7];         // IMAD only: a second IMAD
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) r ^= a[j] ^ b[j];
    if (r == 0x5A5A5A5Au) out[0] = r;  // practically never: keeps the chains live
}

}  // namespace isg

extern "C" int isg_int_rate(int mode, double* ops_per_s) {
    if (!ops_per_s || mode < 0 || mode > 2) {
        set_error("isg_int_rate: bad argument");
        return ISG_ERR_ARG;
    }
    uint32_t* d = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256, iters = 4096;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
        e = cudaEventRecord(e0, 0);
        if (e == cudaSuccess) {
            if (mode == 0) int_rate_kernel<0><<<blocks, threads>>>(0x12345u + rep, iters, d);
            else if (mode == 1) int_rate_kernel<1><<<blocks, threads>>>(0x12345u + rep, iters, d);
            else int_rate_kernel<2><<<blocks, threads>>>(0x12345u + rep, iters, d);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaFree(d);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "isg_int_rate");
    const double ops = (double)blocks * threads * iters * 8 * 2;
    *ops_per_s = ops / (ms * 1e-3);
    return ISG_OK;
}
