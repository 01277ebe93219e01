// isg_noalloc.cu -- isg_energy_static_scratch: the energy of a handle computed
// without allocating any memory.
//
// Some callers must not allocate device memory at the moment they ask for the
// energy: real-time loops that cannot afford the device-wide synchronisation
// an allocation may cause, and processes or embedding runtimes that hand out
// their device memory from a budget fixed up front, where any allocation
// outside it is an error.  isg_energy reduces into a word owned by the handle;
// this variant keeps its per-block partial sums in a fixed array compiled into
// the library instead, so the call only launches kernels and never calls
// cudaMalloc, cudaFree or any allocating routine.
//
// Limits and sharing rules:
//   * the array holds kStaticPartials = 8192 partial sums (64 KiB per device);
//     one partial covers 512 rows of one colour, so lattices with
//     2 L^2 / 512 > 8192, i.e. L > 1448, are rejected with ISG_ERR_ARG;
//   * every device that loads the library holds the array until the process
//     exits;
//   * every call writes all the partials it later reads, so nothing has to be
//     cleared between calls, but all calls share the one array: calls whose
//     kernels overlap on the GPU (for instance on two streams) race and give
//     wrong results;
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (once per device, with that device current) and
//     keeps it; make that first call before any stream capture begins.  The
//     kept address assumes that the device's context lives until the process
//     exits (no cudaDeviceReset in between).
#include <mutex>

#include "isg_common.cuh"

namespace isg {

constexpr int kStaticPartials = 8192;
constexpr int kRowsPerPartial = 512;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned long long g_energy_partials[kStaticPartials];

struct StaticGeom {
    const unsigned char* planes;
    int64_t plane_bytes;
    int L, half, W, nt;
    int64_t rows;
};

// Block b counts the unsatisfied forward bonds of rows [512 b, 512 b + 512) of
// the 2 * rows rows of both colours (the count isg_energy makes) and writes the
// count to partials[b].
template <typename Word>
__global__ void static_unsat_kernel(StaticGeom g, unsigned long long* partials) {
    constexpr int w = 8 * sizeof(Word);
    __shared__ unsigned long long warp_sum[8];
    const int64_t q0 = (int64_t)blockIdx.x * kRowsPerPartial;
    const int64_t q1 = q0 + kRowsPerPartial < 2 * g.rows ? q0 + kRowsPerPartial : 2 * g.rows;
    const int nwords = (int)((q1 - q0) * g.W);  // a few rows' words: 32-bit index arithmetic
    unsigned long long acc = 0;
    for (int e = threadIdx.x; e < nwords; e += blockDim.x) {
        const int eq = e / g.W;
        const int64_t q = q0 + eq;
        const int k = e - eq * g.W;
        const int c = q >= g.rows ? 1 : 0;
        const int r = (int)(q - (int64_t)c * g.rows);
        const int L = g.L, W = g.W;
        const int y = r % L, z = r / L;
        const int p = (c + y + z) & 1;
        const int yp = y == L - 1 ? 0 : y + 1, zp = z == L - 1 ? 0 : z + 1;
        const size_t o = (size_t)r * W + k;
        const Word* Sn = (const Word*)(g.planes + (size_t)(4 * (c ^ 1)) * g.plane_bytes);
        const Word s = ((const Word*)(g.planes + (size_t)(4 * c) * g.plane_bytes))[o];
        Word nxp = Sn[o];
        if (p == 1) nxp = row_up<Word>(nxp, Sn[(size_t)r * W + (k == W - 1 ? 0 : k + 1)], k, W, g.nt);
        const Word ex = ((const Word*)(g.planes + (size_t)(4 * c + 1) * g.plane_bytes))[o] ^ s ^ nxp;
        const Word ey = ((const Word*)(g.planes + (size_t)(4 * c + 2) * g.plane_bytes))[o] ^ s ^
                        Sn[(size_t)(yp + L * z) * W + k];
        const Word ez = ((const Word*)(g.planes + (size_t)(4 * c + 3) * g.plane_bytes))[o] ^ s ^
                        Sn[(size_t)(y + L * zp) * W + k];
        const Word m = (k == W - 1 && g.nt < w) ? (Word)((Word(1) << g.nt) - 1) : ~Word(0);
        acc += (unsigned long long)(Logic<Word>::popc(ex & m) + Logic<Word>::popc(ey & m) +
                                    Logic<Word>::popc(ez & m));
    }
    for (int sh = 16; sh; sh >>= 1) acc += __shfl_xor_sync(kFull, acc, sh);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += warp_sum[i];
        partials[blockIdx.x] = t;
    }
}

// One block: E = 2 * (sum of the n partials) - 3 N, written to *out.
__global__ void static_sum_kernel(const unsigned long long* partials, int n, long long threeN, long long* out) {
    __shared__ unsigned long long warp_sum[8];
    unsigned long long acc = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
    for (int sh = 16; sh; sh >>= 1) acc += __shfl_xor_sync(kFull, acc, sh);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += warp_sum[i];
        *out = 2 * (long long)t - threeN;
    }
}

// Device address of g_energy_partials for each device, looked up once.
static std::mutex g_static_mu;
static void* g_static_ptr[kMaxDevices] = {nullptr};

static int static_partials(unsigned long long** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("isg_energy_static_scratch: device %d beyond the %d supported", dev, kMaxDevices);
        return ISG_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_energy_partials);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(g_energy_partials)");
        g_static_ptr[dev] = p;
    }
    *out = (unsigned long long*)g_static_ptr[dev];
    return ISG_OK;
}

}  // namespace isg

using namespace isg;

extern "C" int isg_energy_static_scratch(const isg_sim* h, long long* dev_E, void* cuda_stream) {
    if (!h || !dev_E) {
        set_error("isg_energy_static_scratch: NULL argument");
        return ISG_ERR_ARG;
    }
    const int64_t blocks = (2 * h->rows + kRowsPerPartial - 1) / kRowsPerPartial;
    if (blocks > kStaticPartials) {
        set_error("isg_energy_static_scratch: L=%d needs %lld partial sums, the static array holds %d "
                  "(L <= 1448)", h->L, (long long)blocks, kStaticPartials);
        return ISG_ERR_ARG;
    }
    unsigned long long* partials = nullptr;
    int rc = static_partials(&partials);
    if (rc) return rc;
    StaticGeom g;
    g.planes = h->planes;
    g.plane_bytes = h->plane_bytes;
    g.L = h->L;
    g.half = h->half;
    g.W = h->W;
    g.nt = h->nt;
    g.rows = h->rows;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (h->wbits == 64) static_unsat_kernel<uint64_t><<<(unsigned)blocks, 256, 0, s>>>(g, partials);
    else static_unsat_kernel<uint32_t><<<(unsigned)blocks, 256, 0, s>>>(g, partials);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        static_sum_kernel<<<1, 256, 0, s>>>(partials, (int)blocks, 3LL * h->L * h->L * h->L, dev_E);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? ISG_OK : cuda_fail(e, "isg_energy_static_scratch launch");
}
