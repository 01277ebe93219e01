// isg_spinio.cu -- spin configurations between the bit planes and host formats
// in site order i = x + L*y + L*L*z: int8 +-1 (one byte per spin) and packed
// bits (bit i of the array is site i; 1 means s = +1, the Sec. 4 bit map).
//
// The plane layout stores colour c's sites of row r = y + L*z at bits
// h = x >> 1 (x = 2h + ((c+y+z) & 1)); a run of consecutive sites therefore
// alternates between the two colour planes and advances one bit in each every
// two sites.  The site-order kernels (planes -> host format) give each thread a
// run of 16 or 32 sites and keep the current word of each colour in registers;
// the plane-order kernels (host format -> planes) give each thread one plane
// word and gather its sites, two bytes (or bits) apart.
#include "isg_common.cuh"

namespace isg {

struct IoGeom {
    unsigned char* planes;
    int64_t plane_bytes;
    int L, half, W;
    int64_t rows, N;
};

static IoGeom iogeom(const isg_sim* h) {
    IoGeom g;
    g.planes = h->planes;
    g.plane_bytes = h->plane_bytes;
    g.L = h->L;
    g.half = h->half;
    g.W = h->W;
    g.rows = h->rows;
    g.N = (int64_t)h->L * h->L * h->L;
    return g;
}

// Walks sites i, i + 1, ... keeping (x, y, z, r) and the last plane word read
// for each colour.
template <typename Word>
struct SiteWalk {
    int x, y, z;
    int64_t r;
    int64_t idx[2];
    Word word[2];

    __device__ __forceinline__ void start(const IoGeom& g, int64_t i) {
        r = i / g.L;
        x = (int)(i - r * g.L);
        y = (int)(r % g.L);
        z = (int)(r / g.L);
        idx[0] = idx[1] = -1;
    }
    // spin bit of the current site
    __device__ __forceinline__ unsigned bit(const IoGeom& g) {
        constexpr int w = 8 * sizeof(Word);
        const int c = (x + y + z) & 1, h = x >> 1;
        const int64_t k = r * g.W + h / w;
        if (k != idx[c]) {
            idx[c] = k;
            word[c] = ((const Word*)(g.planes + (size_t)(4 * c) * g.plane_bytes))[k];
        }
        return (unsigned)(word[c] >> (h % w)) & 1u;
    }
    __device__ __forceinline__ void next(const IoGeom& g) {
        if (++x == g.L) {
            x = 0;
            ++r;
            if (++y == g.L) {
                y = 0;
                ++z;
            }
        }
    }
};

// planes -> int8 +-1: 16 sites per thread, one 16-byte store.
template <typename Word>
__global__ void unpack_spins16_kernel(IoGeom g, int8_t* out) {
    const int64_t nt = (g.N + 15) / 16;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = 16 * t;
        SiteWalk<Word> s;
        s.start(g, i0);
        if (i0 + 16 <= g.N) {
            uint32_t v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t u = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    u |= (s.bit(g) ? 0x01u : 0xFFu) << (8 * j);
                    s.next(g);
                }
                v[q] = u;
            }
            *(uint4*)(out + i0) = make_uint4(v[0], v[1], v[2], v[3]);
        } else {
            for (int64_t i = i0; i < g.N; ++i) {
                out[i] = s.bit(g) ? 1 : -1;
                s.next(g);
            }
        }
    }
}

// planes -> packed bits: 32 sites per thread, one word.
template <typename Word>
__global__ void unpack_spins_bits_kernel(IoGeom g, uint32_t* out) {
    const int64_t nt = (g.N + 31) / 32;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = 32 * t;
        const int n = g.N - i0 < 32 ? (int)(g.N - i0) : 32;
        SiteWalk<Word> s;
        s.start(g, i0);
        uint32_t u = 0;
        for (int j = 0; j < n; ++j) {
            u |= s.bit(g) << j;
            s.next(g);
        }
        out[t] = u;
    }
}

// Plane word t = (c, r, k) and its parity p.
struct WordPos {
    int c, k, p;
    int64_t r;
};

__device__ __forceinline__ WordPos word_pos(const IoGeom& g, int64_t t) {
    WordPos q;
    const int64_t per = g.rows * g.W;
    q.c = (int)(t / per);
    const int64_t rem = t - q.c * per;
    q.r = rem / g.W;
    q.k = (int)(rem - q.r * g.W);
    const int y = (int)(q.r % g.L), z = (int)(q.r / g.L);
    q.p = (q.c + y + z) & 1;
    return q;
}

// int8 +-1 -> planes, checked: every byte must be 1 or -1 (else *bad = 1).
// Writes colour c's word into dst + c * plane_bytes (a scratch copy of the two
// spin planes), so that a rejected array changes nothing.  With L a multiple of
// 2w a word's 2w bytes are one aligned run, read as 16-byte vectors.
template <typename Word>
__global__ void pack_spins_checked_kernel(IoGeom g, const int8_t* in, unsigned char* dst, int* bad) {
    constexpr int w = 8 * sizeof(Word);
    const int64_t nw = 2 * g.rows * g.W;
    const bool vec = g.L % (2 * w) == 0;
    int badl = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nw; t += (int64_t)gridDim.x * blockDim.x) {
        const WordPos q = word_pos(g, t);
        Word word = 0;
        const int64_t base = q.r * g.L + 2 * (int64_t)q.k * w;  // byte of x = 2 k w
        if (vec) {
            const uint4* src = (const uint4*)(in + base);
#pragma unroll
            for (int v4 = 0; v4 < 2 * w / 16; ++v4) {
                const uint4 m = src[v4];
                const uint32_t part[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t one = __vcmpeq4(part[j], 0x01010101u);
                    const uint32_t neg = __vcmpeq4(part[j], 0xFFFFFFFFu);
                    badl |= (one | neg) != 0xFFFFFFFFu;
                    // bytes 2s + p of this 4-byte group are sites h = 2 (4 v4 + j) + s
                    const int h0 = 2 * (4 * v4 + j);
                    const uint32_t b0 = (one >> (8 * q.p)) & 1u, b1 = (one >> (16 + 8 * q.p)) & 1u;
                    word |= ((Word)b0 << h0) | ((Word)b1 << (h0 + 1));
                }
            }
        } else {
            for (int b = 0; b < w; ++b) {
                const int h = q.k * w + b;
                if (h >= g.half) break;
                const int v = in[q.r * g.L + 2 * h + q.p];
                badl |= v != 1 && v != -1;
                if (v == 1) word |= (Word)1 << b;
            }
        }
        ((Word*)(dst + (size_t)q.c * g.plane_bytes))[q.r * g.W + q.k] = word;
    }
    if (__any_sync(kFull, badl) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

// packed bits -> planes (every bit pattern is a valid configuration).
template <typename Word>
__global__ void pack_spins_bits_kernel(IoGeom g, const uint32_t* in) {
    constexpr int w = 8 * sizeof(Word);
    const int64_t nw = 2 * g.rows * g.W;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nw; t += (int64_t)gridDim.x * blockDim.x) {
        const WordPos q = word_pos(g, t);
        Word word = 0;
        int64_t cur = -1;
        uint32_t bits = 0;
        for (int b = 0; b < w; ++b) {
            const int h = q.k * w + b;
            if (h >= g.half) break;
            const int64_t i = q.r * g.L + 2 * h + q.p;
            if ((i >> 5) != cur) {
                cur = i >> 5;
                bits = in[cur];
            }
            word |= (Word)((bits >> (i & 31)) & 1u) << b;
        }
        ((Word*)(g.planes + (size_t)(4 * q.c) * g.plane_bytes))[q.r * g.W + q.k] = word;
    }
}

// Bit interleaving for rows whose site runs align with plane words (L a
// multiple of 64): the 64 sites x = 64m .. 64m + 63 of a row are the 32 bits
// h = 32m .. 32m + 31 of each colour, red at x = 2h + pr, blue at 2h + 1 - pr
// (pr = (y + z) & 1).  spread() puts bit j at 2j; compact() is its inverse.
__device__ __forceinline__ uint64_t spread32(uint64_t v) {
    v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
    v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

__device__ __forceinline__ uint64_t compact32(uint64_t v) {
    v &= 0x5555555555555555ull;
    v = (v | (v >> 1)) & 0x3333333333333333ull;
    v = (v | (v >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v >> 4)) & 0x00FF00FF00FF00FFull;
    v = (v | (v >> 8)) & 0x0000FFFF0000FFFFull;
    v = (v | (v >> 16)) & 0x00000000FFFFFFFFull;
    return v;
}

// planes -> packed bits, L % 64 == 0: one thread per plane word slot (row r,
// word k) of both colours, i.e. w / 32 runs of 64 sites of the row; a last word
// with fewer valid sites (64-bit words when L / 2 is an odd multiple of 32)
// writes only its valid runs.  Indices fit in 32 bits (rows * W < 2^27).
template <typename Word>
__global__ void unpack_spins_bits64_kernel(IoGeom g, uint64_t* out) {
    constexpr int w = 8 * sizeof(Word);
    const unsigned W = (unsigned)g.W, L = (unsigned)g.L, half = (unsigned)g.half;
    const unsigned n = (unsigned)g.rows * W;
    const Word* P0 = (const Word*)g.planes;
    const Word* P1 = (const Word*)(g.planes + (size_t)4 * g.plane_bytes);
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
        const unsigned r = t / W, k = t - r * W;
        const unsigned pr = (r % L + r / L) & 1u;
        const Word red = P0[t], blue = P1[t];
        uint64_t* o = out + (size_t)r * (L / 64) + (size_t)k * (w / 32);
#pragma unroll
        for (int q = 0; q < w / 32; ++q)
            if (k * w + 32 * q < half)
                o[q] = (spread32((uint32_t)(red >> (32 * q))) << pr) |
                       (spread32((uint32_t)(blue >> (32 * q))) << (1 - pr));
    }
}

// packed bits -> planes, L % 64 == 0: one thread per plane word slot of both
// colours; the bits of a last word past the row's valid sites stay zero.
template <typename Word>
__global__ void pack_spins_bits64_kernel(IoGeom g, const uint64_t* in) {
    constexpr int w = 8 * sizeof(Word);
    const unsigned W = (unsigned)g.W, L = (unsigned)g.L, half = (unsigned)g.half;
    const unsigned n = (unsigned)g.rows * W;
    Word* P0 = (Word*)g.planes;
    Word* P1 = (Word*)(g.planes + (size_t)4 * g.plane_bytes);
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
        const unsigned r = t / W, k = t - r * W;
        const unsigned pr = (r % L + r / L) & 1u;
        const uint64_t* ip = in + (size_t)r * (L / 64) + (size_t)k * (w / 32);
        Word red = 0, blue = 0;
#pragma unroll
        for (int q = 0; q < w / 32; ++q)
            if (k * w + 32 * q < half) {
                const uint64_t v = ip[q];
                red |= (Word)compact32(v >> pr) << (32 * q);
                blue |= (Word)compact32(v >> (1 - pr)) << (32 * q);
            }
        P0[t] = red;
        P1[t] = blue;
    }
}

static unsigned io_grid(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_unpack_spins_fast(const isg_sim* h, int8_t* out, cudaStream_t s) {
    const IoGeom g = iogeom(h);
    const unsigned grid = io_grid((g.N + 15) / 16, 256);
    if (h->wbits == 64) unpack_spins16_kernel<uint64_t><<<grid, 256, 0, s>>>(g, out);
    else unpack_spins16_kernel<uint32_t><<<grid, 256, 0, s>>>(g, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_spins_checked(const isg_sim* h, const int8_t* in, unsigned char* dst, int* bad,
                                      cudaStream_t s) {
    const IoGeom g = iogeom(h);
    const unsigned grid = io_grid(2 * g.rows * g.W, 256);
    if (h->wbits == 64) pack_spins_checked_kernel<uint64_t><<<grid, 256, 0, s>>>(g, in, dst, bad);
    else pack_spins_checked_kernel<uint32_t><<<grid, 256, 0, s>>>(g, in, dst, bad);
    return cudaGetLastError();
}

cudaError_t launch_unpack_spins_bits(const isg_sim* h, uint32_t* out, cudaStream_t s) {
    const IoGeom g = iogeom(h);
    if (g.L % 64 == 0) {
        const unsigned grid = io_grid(g.rows * g.W, 256);
        if (h->wbits == 64) unpack_spins_bits64_kernel<uint64_t><<<grid, 256, 0, s>>>(g, (uint64_t*)out);
        else unpack_spins_bits64_kernel<uint32_t><<<grid, 256, 0, s>>>(g, (uint64_t*)out);
        return cudaGetLastError();
    }
    const unsigned grid = io_grid((g.N + 31) / 32, 256);
    if (h->wbits == 64) unpack_spins_bits_kernel<uint64_t><<<grid, 256, 0, s>>>(g, out);
    else unpack_spins_bits_kernel<uint32_t><<<grid, 256, 0, s>>>(g, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_spins_bits(isg_sim* h, const uint32_t* in, cudaStream_t s) {
    const IoGeom g = iogeom(h);
    if (g.L % 64 == 0) {
        const unsigned grid = io_grid(g.rows * g.W, 256);
        if (h->wbits == 64) pack_spins_bits64_kernel<uint64_t><<<grid, 256, 0, s>>>(g, (const uint64_t*)in);
        else pack_spins_bits64_kernel<uint32_t><<<grid, 256, 0, s>>>(g, (const uint64_t*)in);
        return cudaGetLastError();
    }
    const unsigned grid = io_grid(2 * g.rows * g.W, 256);
    if (h->wbits == 64) pack_spins_bits_kernel<uint64_t><<<grid, 256, 0, s>>>(g, in);
    else pack_spins_bits_kernel<uint32_t><<<grid, 256, 0, s>>>(g, in);
    return cudaGetLastError();
}

}  // namespace isg
