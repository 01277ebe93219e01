// isg_init.cu -- lattice and RNG-stream initialisation kernels (not timed).
//
// Couplings (Eq. 2): J_d(i) = -1 when bit 63 of SplitMix64(seed_J ^ K_J, 3i + d)
// is set; spins: s_i = -1 when bit 63 of SplitMix64(seed_spin ^ K_S, i) is set.
// Streams: v_t = SplitMix64(seed_rng ^ K_R, t) (seed_rng = seed_spin unless the
// handle was made with isg_create2); MT19937 starts from
// init_genrand((uint32) v_t), MINSTD from x_0 = 1 + v_t mod (2^31 - 2), and
// Parisi-Rapuano from ira[j] = SplitMix64(v_t, j) >> 32, j < 61, with ira[60]
// made odd (Sec. 3).
#include "isg_common.cuh"

namespace isg {

struct PlaneGeom {
    unsigned char* planes;
    int64_t plane_bytes;
    int L, half, W;
    int64_t rows;
};

static PlaneGeom geom(const isg_sim* h) {
    PlaneGeom g;
    g.planes = h->planes;
    g.plane_bytes = h->plane_bytes;
    g.L = h->L;
    g.half = h->half;
    g.W = h->W;
    g.rows = h->rows;
    return g;
}

// One thread per word of one colour: the four words S, Jx, Jy, Jz at (c, r, k).
template <typename Word>
__global__ void init_planes_kernel(PlaneGeom g, uint64_t seed_J, uint64_t seed_spin) {
    constexpr int w = 8 * sizeof(Word);
    const int64_t nw = 2 * g.rows * g.W;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nw; q += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(q / (g.rows * g.W));
        const int64_t rem = q - (int64_t)c * g.rows * g.W;
        const int64_t r = rem / g.W;
        const int k = (int)(rem - r * g.W);
        const int L = g.L;
        const int y = (int)(r % L), z = (int)(r / L);
        const int p = (c + y + z) & 1;
        Word ws = 0, wx = 0, wy = 0, wz = 0;
        for (int b = 0; b < w; ++b) {
            const int h = k * w + b;
            if (h >= g.half) break;
            const int x = 2 * h + p;
            const uint64_t i = (uint64_t)x + (uint64_t)L * y + (uint64_t)L * L * z;
            const Word bit = (Word)1 << b;
            if (!(splitmix64(seed_spin ^ kSaltSpins, i) >> 63)) ws |= bit;
            if (splitmix64(seed_J ^ kSaltCouplings, 3 * i + 0) >> 63) wx |= bit;
            if (splitmix64(seed_J ^ kSaltCouplings, 3 * i + 1) >> 63) wy |= bit;
            if (splitmix64(seed_J ^ kSaltCouplings, 3 * i + 2) >> 63) wz |= bit;
        }
        const int64_t o = r * g.W + k;
        ((Word*)(g.planes + (size_t)(4 * c + 0) * g.plane_bytes))[o] = ws;
        ((Word*)(g.planes + (size_t)(4 * c + 1) * g.plane_bytes))[o] = wx;
        ((Word*)(g.planes + (size_t)(4 * c + 2) * g.plane_bytes))[o] = wy;
        ((Word*)(g.planes + (size_t)(4 * c + 3) * g.plane_bytes))[o] = wz;
    }
}

static unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return (unsigned)b;
}

cudaError_t launch_init_planes(isg_sim* h, cudaStream_t s) {
    const PlaneGeom g = geom(h);
    const int64_t nw = 2 * h->rows * h->W;
    if (h->wbits == 64)
        init_planes_kernel<uint64_t><<<grid_for(nw, 256), 256, 0, s>>>(g, h->seed_J, h->seed_spin);
    else
        init_planes_kernel<uint32_t><<<grid_for(nw, 256), 256, 0, s>>>(g, h->seed_J, h->seed_spin);
    return cudaGetLastError();
}

// One thread per stream.
__global__ void init_rng_kernel(int kind, uint64_t seed_rng, int64_t S, uint32_t* rng, uint32_t* pos) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S) return;
    const uint64_t v = splitmix64(seed_rng ^ kSaltStreams, (uint64_t)t);
    if (kind == ISG_RNG_MT19937) {
        uint32_t* x = rng + t * kMtN;
        uint32_t prev = (uint32_t)v;
        x[0] = prev;
        for (int k = 1; k < kMtN; ++k) {
            prev = 1812433253u * (prev ^ (prev >> 30)) + (uint32_t)k;
            x[k] = prev;
        }
        pos[t] = 0;
    } else if (kind == ISG_RNG_PARISI_RAPUANO) {
        uint32_t* w = rng + t * kPrN;
        for (int j = 0; j < kPrN; ++j) w[j] = (uint32_t)(splitmix64(v, (uint64_t)j) >> 32);
        w[kPrN - 1] |= 1u;
    } else {
        rng[t] = 1u + (uint32_t)(v % 2147483646ull);
    }
}

cudaError_t launch_init_rng(isg_sim* h, cudaStream_t s) {
    const int threads = 128;
    const unsigned blocks = (unsigned)((h->S + threads - 1) / threads);
    init_rng_kernel<<<blocks, threads, 0, s>>>(h->kind, h->seed_rng, h->S, h->rng, h->rng_pos);
    return cudaGetLastError();
}

}  // namespace isg
