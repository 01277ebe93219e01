// isg_measure.cu -- popcount kernels for the energy (Eq. 1), the replica
// overlap and the Zobrist hash, and the kernels that convert the coupling planes
// to and from int8 +-1 arrays in site order i = x + L*y + L*L*z (the spins'
// conversions are in isg_spinio.cu).
//
// Energy: every coupling is the forward (+x, +y or +z) coupling of exactly one
// site, so U = number of unsatisfied bonds = sum over both colours and all words
// of popc(e_+x) + popc(e_+y) + popc(e_+z), with e = J ^ s ^ s' (Sec. 4 bit map),
// and E = 2U - 3N.
#include "isg_common.cuh"

namespace isg {

struct MeasGeom {
    const unsigned char* planes;
    int64_t plane_bytes;
    int L, half, W, nt;
    int64_t rows;
};

static MeasGeom mgeom(const isg_sim* h) {
    MeasGeom g;
    g.planes = h->planes;
    g.plane_bytes = h->plane_bytes;
    g.L = h->L;
    g.half = h->half;
    g.W = h->W;
    g.nt = h->nt;
    g.rows = h->rows;
    return g;
}

template <typename Word>
__device__ __forceinline__ const Word* plane(const MeasGeom& g, int c, int q) {
    return (const Word*)(g.planes + (size_t)(4 * c + q) * g.plane_bytes);
}

template <typename Word>
__device__ __forceinline__ Word valid_mask(const MeasGeom& g, int k) {
    constexpr int w = 8 * sizeof(Word);
    return (k == g.W - 1 && g.nt < w) ? (Word)((Word(1) << g.nt) - 1) : ~Word(0);
}

__device__ __forceinline__ int popcw(uint32_t v) { return __popc(v); }
__device__ __forceinline__ int popcw(uint64_t v) { return __popcll(v); }

static unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// ---------------------------------------------------------------- energy ---
// Thread t of a block owns word k = t % W of rows r = t / W + rows_per_block * j
// (blocks striding over rows) and counts the forward bonds of that word in BOTH
// colours, so every plane is read from memory once: the neighbour words of one
// colour's word (rows y+1 and z+1 of the other colour, and the next word of the
// row for the site whose +x neighbour is shifted) are words another thread of
// the same pass reads as its own, found in L1 or L2.
template <typename Word>
struct UnsatPair {
    Word s0, s1, jx0, jy0, jz0, jx1, jy1, jz1, n1y, n1z, n0y, n0z, nb;
    int p0;
};

template <typename Word>
__device__ __forceinline__ void unsat_pair_load(const MeasGeom& g, int r, int y, int z, int k, UnsatPair<Word>& u) {
    const int L = g.L, W = g.W;
    const size_t o = (size_t)r * W + k;
    const int ryp = y == L - 1 ? r - (L - 1) : r + 1;
    const int rzp = z == L - 1 ? r - (L - 1) * L : r + L;
    const Word* S0 = plane<Word>(g, 0, 0);
    const Word* S1 = plane<Word>(g, 1, 0);
    u.p0 = (y + z) & 1;  // colour 0's row parity; colour 1's is the other
    u.s0 = S0[o];
    u.s1 = S1[o];
    u.jx0 = plane<Word>(g, 0, 1)[o];
    u.jy0 = plane<Word>(g, 0, 2)[o];
    u.jz0 = plane<Word>(g, 0, 3)[o];
    u.jx1 = plane<Word>(g, 1, 1)[o];
    u.jy1 = plane<Word>(g, 1, 2)[o];
    u.jz1 = plane<Word>(g, 1, 3)[o];
    u.n1y = S1[(size_t)ryp * W + k];
    u.n1z = S1[(size_t)rzp * W + k];
    u.n0y = S0[(size_t)ryp * W + k];
    u.n0z = S0[(size_t)rzp * W + k];
    // the colour whose row parity is 1 has its +x neighbours shifted by one site
    const size_t onb = (size_t)r * W + (k == W - 1 ? 0 : k + 1);
    u.nb = (u.p0 == 1 ? S1 : S0)[onb];
}

template <typename Word>
__device__ __forceinline__ int unsat_pair_count(const MeasGeom& g, int k, const UnsatPair<Word>& u) {
    const Word m = valid_mask<Word>(g, k);
    const Word nx0 = u.p0 == 1 ? row_up<Word>(u.s1, u.nb, k, g.W, g.nt) : u.s1;
    const Word nx1 = u.p0 == 1 ? u.s0 : row_up<Word>(u.s0, u.nb, k, g.W, g.nt);
    return popcw((u.jx0 ^ u.s0 ^ nx0) & m) + popcw((u.jy0 ^ u.s0 ^ u.n1y) & m) +
           popcw((u.jz0 ^ u.s0 ^ u.n1z) & m) + popcw((u.jx1 ^ u.s1 ^ nx1) & m) +
           popcw((u.jy1 ^ u.s1 ^ u.n0y) & m) + popcw((u.jz1 ^ u.s1 ^ u.n0z) & m);
}

// Rows advance by `step` per iteration: (y, z) follow with the precomputed
// step % L and step / L and one carry.
__device__ __forceinline__ void row_advance(int& r, int& y, int& z, int step, int sy, int sz, int L) {
    r += step;
    y += sy;
    z += sz;
    if (y >= L) {
        y -= L;
        ++z;
    }
}

template <typename Word>
__global__ void unsat_kernel(MeasGeom g, long long* out) {
    const int L = g.L, W = g.W, rows = (int)g.rows;
    const int rpb = blockDim.x / W;  // rows per block and iteration
    const int t = threadIdx.x;
    const int rl = t / W, k = t - rl * W;
    long long acc = 0;
    if (rl < rpb) {
        const int step = gridDim.x * rpb;
        const int sy = step % L, sz = step / L;
        int r = blockIdx.x * rpb + rl;
        int y = r % L, z = r / L;
        // two rows in flight: all their loads are issued before either is counted
        while (r < rows) {
            int r2 = r, y2 = y, z2 = z;
            row_advance(r2, y2, z2, step, sy, sz, L);
            UnsatPair<Word> a, b;
            unsat_pair_load<Word>(g, r, y, z, k, a);
            const bool two = r2 < rows;
            if (two) unsat_pair_load<Word>(g, r2, y2, z2, k, b);
            acc += unsat_pair_count<Word>(g, k, a);
            if (two) acc += unsat_pair_count<Word>(g, k, b);
            r = r2;
            y = y2;
            z = z2;
            row_advance(r, y, z, step, sy, sz, L);
        }
    }
    for (int sh = 16; sh; sh >>= 1) acc += __shfl_xor_sync(kFull, acc, sh);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd((unsigned long long*)out, (unsigned long long)acc);
}

cudaError_t launch_energy(const isg_sim* h, long long* out, cudaStream_t s) {
    const MeasGeom g = mgeom(h);
    const int threads = 256;
    const int64_t rpb = threads / h->W;
    int64_t blocks = (h->rows + rpb - 1) / rpb;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    if (h->wbits == 64) unsat_kernel<uint64_t><<<(unsigned)blocks, threads, 0, s>>>(g, out);
    else unsat_kernel<uint32_t><<<(unsigned)blocks, threads, 0, s>>>(g, out);
    return cudaGetLastError();
}

// --------------------------------------------------------------- overlap ---
// Number of sites where the two replicas differ (tail bits are zero in both).
__global__ void differ_kernel(const unsigned long long* a0, const unsigned long long* a1,
                              const unsigned long long* b0, const unsigned long long* b1, int64_t n64,
                              long long* out) {
    long long acc = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n64; q += (int64_t)gridDim.x * blockDim.x)
        acc += __popcll(a0[q] ^ b0[q]) + __popcll(a1[q] ^ b1[q]);
    for (int sh = 16; sh; sh >>= 1) acc += __shfl_xor_sync(kFull, acc, sh);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd((unsigned long long*)out, (unsigned long long)acc);
}

cudaError_t launch_overlap(const isg_sim* a, const isg_sim* b, long long* out, cudaStream_t s) {
    // a plane holds rows * W * wbits bits; with wbits = 32 and an odd word count
    // the byte size is still a multiple of 4; pad handling: count in 32-bit words
    const int64_t n64 = a->plane_bytes / 8;
    const bool odd = (a->plane_bytes % 8) != 0;
    if (odd) return cudaErrorInvalidValue;  // plane_bytes is always padded to 8 bytes
    differ_kernel<<<grid_for(n64, 256), 256, 0, s>>>(
        (const unsigned long long*)a->plane(0, 0), (const unsigned long long*)a->plane(1, 0),
        (const unsigned long long*)b->plane(0, 0), (const unsigned long long*)b->plane(1, 0), n64, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ hash ---
template <typename Word>
__global__ void hash_kernel(MeasGeom g, unsigned long long* out) {
    constexpr int w = 8 * sizeof(Word);
    const int64_t nw = 2 * g.rows * g.W;
    unsigned long long acc = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nw; q += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(q / (g.rows * g.W));
        const int64_t rem = q - (int64_t)c * g.rows * g.W;
        const int r = (int)(rem / g.W);
        const int k = (int)(rem - (int64_t)r * g.W);
        const int L = g.L;
        const int y = r % L, z = r / L;
        const int p = (c + y + z) & 1;
        Word v = plane<Word>(g, c, 0)[(size_t)r * g.W + k] & valid_mask<Word>(g, k);
        const uint64_t rowbase = (uint64_t)L * y + (uint64_t)L * L * z;
        while (v) {
            const int b = (w == 64) ? (__ffsll((long long)v) - 1) : (__ffs((int)v) - 1);
            v &= v - 1;
            const uint64_t i = rowbase + (uint64_t)(2 * (k * w + b) + p);
            acc ^= splitmix64(kSaltHash, i);
        }
    }
    for (int sh = 16; sh; sh >>= 1) acc ^= __shfl_xor_sync(kFull, acc, sh);
    if ((threadIdx.x & 31) == 0 && acc) atomicXor(out, acc);
}

cudaError_t launch_hash(const isg_sim* h, unsigned long long* out, cudaStream_t s) {
    const MeasGeom g = mgeom(h);
    const int64_t nw = 2 * h->rows * h->W;
    if (h->wbits == 64) hash_kernel<uint64_t><<<grid_for(nw, 256), 256, 0, s>>>(g, out);
    else hash_kernel<uint32_t><<<grid_for(nw, 256), 256, 0, s>>>(g, out);
    return cudaGetLastError();
}

// ------------------------------------------------------ unpack / pack ---
// q = 0: spins (bit 1 -> +1); q = 1..3: couplings (bit 1 -> -1).
template <typename Word>
__global__ void unpack_kernel(MeasGeom g, int q, int8_t* out) {
    constexpr int w = 8 * sizeof(Word);
    const int64_t L = g.L, N = L * L * L;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % L), y = (int)((i / L) % L), z = (int)(i / (L * L));
        const int c = (x + y + z) & 1;
        const int h = x >> 1, k = h / w, b = h % w;
        const Word word = plane<Word>(g, c, q)[((size_t)y + (size_t)L * z) * g.W + k];
        const int bit = (int)((word >> b) & 1);
        out[i] = q == 0 ? (bit ? 1 : -1) : (bit ? -1 : 1);
    }
}

template <typename Word>
__global__ void pack_kernel(MeasGeom g, int q, const int8_t* in) {
    constexpr int w = 8 * sizeof(Word);
    const int64_t nw = 2 * g.rows * g.W;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nw; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / (g.rows * g.W));
        const int64_t rem = t - (int64_t)c * g.rows * g.W;
        const int r = (int)(rem / g.W);
        const int k = (int)(rem - (int64_t)r * g.W);
        const int L = g.L;
        const int y = r % L, z = r / L;
        const int p = (c + y + z) & 1;
        Word word = 0;
        for (int b = 0; b < w; ++b) {
            const int h = k * w + b;
            if (h >= g.half) break;
            const int64_t i = (int64_t)(2 * h + p) + (int64_t)L * y + (int64_t)L * L * z;
            const int v = in[i];
            const bool one = (q == 0) ? (v == 1) : (v == -1);
            if (one) word |= (Word)1 << b;
        }
        ((Word*)(g.planes + (size_t)(4 * c + q) * g.plane_bytes))[(size_t)r * g.W + k] = word;
    }
}

cudaError_t launch_unpack_couplings(const isg_sim* h, int8_t* out, cudaStream_t s) {
    const MeasGeom g = mgeom(h);
    const int64_t N = (int64_t)h->L * h->L * h->L;
    for (int d = 0; d < 3; ++d) {
        if (h->wbits == 64) unpack_kernel<uint64_t><<<grid_for(N, 256), 256, 0, s>>>(g, 1 + d, out + d * N);
        else unpack_kernel<uint32_t><<<grid_for(N, 256), 256, 0, s>>>(g, 1 + d, out + d * N);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_couplings(isg_sim* h, const int8_t* in, cudaStream_t s) {
    const MeasGeom g = mgeom(h);
    const int64_t N = (int64_t)h->L * h->L * h->L;
    const int64_t nw = 2 * h->rows * h->W;
    for (int d = 0; d < 3; ++d) {
        if (h->wbits == 64) pack_kernel<uint64_t><<<grid_for(nw, 256), 256, 0, s>>>(g, 1 + d, in + d * N);
        else pack_kernel<uint32_t><<<grid_for(nw, 256), 256, 0, s>>>(g, 1 + d, in + d * N);
    }
    return cudaGetLastError();
}

__global__ void check_pm1_kernel(const int8_t* in, int64_t n, int* bad) {
    int b = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b |= (in[i] != 1 && in[i] != -1);
    if (__any_sync(kFull, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

cudaError_t launch_check_pm1(const int8_t* in, int64_t n, int* bad, cudaStream_t s) {
    check_pm1_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, n, bad);
    return cudaGetLastError();
}

}  // namespace isg
