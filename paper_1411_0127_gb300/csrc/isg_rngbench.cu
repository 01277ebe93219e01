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
