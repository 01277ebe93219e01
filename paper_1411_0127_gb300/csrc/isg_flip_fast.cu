// isg_flip_fast.cu -- the production flip kernel behind isg_sweep.
//
// Same site -> (stream, draw) map, same bit logic and the same results, bit for
// bit, as the plain kernel of isg_flip.cu; the per-stream work is the shared
// stream_pass of isg_stream.cuh.  What changes is how the work is issued: the
// grid fills the GPU once and every warp takes stream after stream from a
// monotonically increasing ticket counter, so the last "wave" of streams is
// spread over all SMs instead of leaving most of them idle.
//
// Segments (MINSTD, lattices with few streams): the draws of a stream are
// x_j = x 16807^(j+1) mod (2^31 - 1), so a warp can start anywhere in the
// stream by one multiplication.  When the lattice has too few streams to fill
// the GPU, every stream is cut into nseg segments of whole row groups, each a
// work item of its own, started from x 16807^(first draw index).  The stream's
// end state x 16807^D is written by its last segment into the handle's other
// state buffer (rng_alt), so no item can overwrite a state another item has
// still to read; the host swaps the two buffers after the launch.
//
// Consecutive passes are launched with programmatic dependent launch: a warp
// with no items left signals griddepcontrol.launch_dependents, so the next
// pass's CTAs can be placed on the SM slots this grid frees, and every CTA
// starts with griddepcontrol.wait, which returns once the previous grid has
// completed and its writes are visible.  Small lattices, whose passes last a
// few microseconds, spend much less of each sweep between launches.
#include <cstring>
#include <utility>

#include "isg_stream.cuh"

namespace isg {

constexpr int kFastWarps = 4;
constexpr int kFastSlack = 1024;  // MT19937 window: 624 live words + 1024 free (6.6 KiB per warp)

struct Tickets {
    unsigned long long* counter;  // device word, only ever incremented
    unsigned long long base;      // its value when this launch starts
};

constexpr int kMaxSegments = 64;

// Segmented launch (MINSTD only; nseg = 1 otherwise).
struct Segments {
    int nseg;                     // segments per stream
    int64_t segrows;              // rows per segment, a multiple of the row-group height
    uint32_t jump[kMaxSegments];  // 16807^(k segrows L/2) mod (2^31 - 1): start of segment k
    uint32_t jend, jend_last;     // 16807^D for a full stream and for the last stream
    uint32_t* rng_out;            // the other state buffer
};

// The throughput form keeps 7 (MT19937: shared memory) or 8 blocks of 4 warps
// per SM; the latency form runs with few warps and may use more registers.
template <typename Word, int KIND, bool TRIM, bool USUM>
__global__ void __launch_bounds__(kFastWarps * 32, TRIM ? (KIND == ISG_RNG_MT19937 ? 7 : 8) : 2)
    flip_fast_kernel(FlipArgs a, StreamConst k, Tickets tk, Segments sg, unsigned long long* usum) {
    // Programmatic dependent launch: wait for the previous pass (its spins,
    // generator states and ticket count) before touching any of them.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    extern __shared__ uint32_t smem[];
    constexpr int kRing = KIND == ISG_RNG_MT19937 ? mt_window(kFastSlack) : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* ring = smem + wid * (kRing + 2 * kCondWords);
    uint32_t* cond = ring + kRing;
    const int64_t items = a.S * sg.nseg;
    int dEsum = 0;
    int ulocal = 0;  // USUM: unsatisfied bonds counted before the pass's flips
    int* up = USUM ? &ulocal : nullptr;
    // Items come from the ticket counter, except in the MINSTD latency form
    // (segmented launches), which takes them statically, item u by CTA u mod
    // grid, so that every SM gets work (L = 256 MINSTD 1.34 -> 1.25 ps, L = 32
    // 169 -> 163 ps).  The choice is made at compile time: in the MT19937 and
    // Parisi-Rapuano latency forms even an unused static branch changed the
    // code enough to cost 6-40 %.
    constexpr bool kStatic = KIND == ISG_RNG_MINSTD && !TRIM;
    int64_t u_next = (int64_t)wid * gridDim.x + blockIdx.x;
    for (;;) {
        int64_t u;
        if constexpr (kStatic) {
            u = u_next;
            u_next += (int64_t)gridDim.x * kFastWarps;
        } else {
            unsigned long long v = 0;
            if (lane == 0) v = atomicAdd(tk.counter, 1ull);
            v = __shfl_sync(kFull, v, 0);
            u = (int64_t)(v - tk.base);
        }
        if (u >= items) break;
        StreamRegs st;
        if (KIND == ISG_RNG_MINSTD && !TRIM && sg.nseg > 1) {  // segments: latency form only
            const int64_t t = u / sg.nseg;
            const int ks = (int)(u - t * sg.nseg);
            const int64_t r0 = t * a.R, r1 = r0 + a.R < a.rows ? r0 + a.R : a.rows;
            const int64_t rb = r0 + ks * sg.segrows;
            const int64_t re = rb + sg.segrows < r1 ? rb + sg.segrows : r1;
            const uint32_t x0 = a.rng[t];
            if (rb < re) {
                st.xA = minstd_mulmod(minstd_mulmod(x0, sg.jump[ks]), a.mt.pow[lane + 1]);
                st.xB = minstd_mulmod(st.xA, k.a32);
                stream_pass<Word, KIND, kFastSlack, TRIM>(a, a.c, rb, re, ring, cond, st, k, lane, dEsum, up);
            }
            if (ks == sg.nseg - 1 && lane == 0)
                sg.rng_out[t] = minstd_mulmod(x0, t == a.S - 1 ? sg.jend_last : sg.jend);
        } else {
            const int64_t t = u;
            load_stream<KIND>(a, t, ring, st, k, lane);
            const int64_t rb = t * a.R, re = rb + a.R < a.rows ? rb + a.R : a.rows;
            stream_pass<Word, KIND, kFastSlack, TRIM>(a, a.c, rb, re, ring, cond, st, k, lane, dEsum, up);
            store_stream<KIND>(a, t, ring, st, lane);
        }
    }
    // this warp has no more items: the next pass's CTAs may take the SM slots
    // that this grid's CTAs free (they wait above until this grid completes)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    for (int sh = 16; sh; sh >>= 1) dEsum += __shfl_xor_sync(kFull, dEsum, sh);
    if (lane == 0 && dEsum != 0) atomicAdd((unsigned long long*)a.dE, (unsigned long long)(long long)dEsum);
    if (USUM) {
        for (int sh = 16; sh; sh >>= 1) ulocal += __shfl_xor_sync(kFull, ulocal, sh);
        if (lane == 0 && ulocal != 0) atomicAdd(usum, (unsigned long long)ulocal);
    }
}

// Streams per SM from which the throughput form of the draw phase (TRIM) is used:
// below it too few warps are resident to hide the longer dependency chain.
constexpr int64_t kTrimStreamsPerSM = 16;

// a^e mod (2^31 - 1) by square and multiply (host).
static uint32_t minstd_pow(uint32_t a, uint64_t e) {
    uint32_t r = 1;
    while (e) {
        if (e & 1) r = minstd_mulmod(r, a);
        a = minstd_mulmod(a, a);
        e >>= 1;
    }
    return r;
}

// Segments of a MINSTD launch with fewer streams than the resident warps can
// take (nseg = 1 otherwise): about two items per resident warp, each at least
// one row group.  Not for batch members and batched server jobs (member): their
// state pointers are also held in device descriptors and captured graphs, which
// the buffer swap would leave behind.
static Segments plan_segments(const isg_sim* h, int64_t resident_warps, bool latency_form) {
    Segments sg;
    memset(&sg, 0, sizeof sg);
    sg.nseg = 1;
    if (h->kind != ISG_RNG_MINSTD || !latency_form || !h->rng_alt || h->member) return sg;
    const int64_t G = 32 / h->W;
    const int64_t groups = (h->R + G - 1) / G;
    int64_t nseg = (2 * resident_warps + h->S - 1) / h->S;
    if (nseg > groups) nseg = groups;
    if (nseg > kMaxSegments) nseg = kMaxSegments;
    if (nseg < 2) return sg;
    const int64_t gps = (groups + nseg - 1) / nseg;  // row groups per segment
    sg.nseg = (int)((groups + gps - 1) / gps);
    sg.segrows = gps * G;
    for (int k = 0; k < sg.nseg; ++k) sg.jump[k] = minstd_pow(kMinstdA, (uint64_t)(k * sg.segrows * h->half));
    const int64_t last_rows = h->rows - (h->S - 1) * h->R;
    sg.jend = minstd_pow(kMinstdA, (uint64_t)(h->R * h->half));
    sg.jend_last = minstd_pow(kMinstdA, (uint64_t)(last_rows * h->half));
    sg.rng_out = h->rng_alt;
    return sg;
}

template <typename Word, int KIND, bool TRIM>
static cudaError_t launch_fast_t(isg_sim* h, int colour, cudaStream_t s, int sms, unsigned long long* usum) {
    const FlipArgs a = make_flip_args(h, colour);
    const StreamConst k = stream_const();
    Tickets tk;
    tk.counter = (unsigned long long*)(h->scal + 3);
    tk.base = h->tickets;
    constexpr int kRing = KIND == ISG_RNG_MT19937 ? mt_window(kFastSlack) : 0;
    const size_t smem = (size_t)kFastWarps * (kRing + 2 * kCondWords) * sizeof(uint32_t);
    static std::atomic<int> occ_cache[kDeviceSlots];  // resident blocks per SM of this instantiation
    const int occ = occupancy_cached(occ_cache, flip_fast_kernel<Word, KIND, TRIM, false>, kFastWarps * 32, smem);
    const Segments sg = plan_segments(h, (int64_t)sms * occ * kFastWarps, !TRIM);
    const int64_t items = h->S * sg.nseg;
    int64_t blocks = (int64_t)sms * occ;
    const int64_t need = (items + kFastWarps - 1) / kFastWarps;
    if (blocks > need) blocks = need > sms ? need : (sms < blocks ? sms : blocks);  // at least one block per SM
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)blocks);
    lc.blockDim = dim3(kFastWarps * 32);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    // Programmatic dependent launch, except for the unsegmented latency form
    // (MT19937 and Parisi-Rapuano below 16 streams per SM), where the next
    // pass's CTAs, placed while this grid still runs, made L = 256 MT19937 14 %
    // slower; it takes L = 32 / 48 / 256 MINSTD from 250 / 104 / 1.62 to
    // 168 / 54 / 1.34 ps.
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = (TRIM || sg.nseg > 1) ? 1 : 0;
    // with usum, the instantiation that also counts the pass's unsatisfied bonds
    cudaError_t e = usum ? cudaLaunchKernelEx(&lc, flip_fast_kernel<Word, KIND, TRIM, true>, a, k, tk, sg, usum)
                         : cudaLaunchKernelEx(&lc, flip_fast_kernel<Word, KIND, TRIM, false>, a, k, tk, sg, usum);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // with tickets, every warp takes one ticket past the last item before it stops
    if (KIND != ISG_RNG_MINSTD || TRIM)
        h->tickets += (unsigned long long)items + (unsigned long long)blocks * kFastWarps;
    if (sg.nseg > 1) std::swap(h->rng, h->rng_alt);  // the end states are in the other buffer
    return e;
}

cudaError_t launch_flip_fast(isg_sim* h, int colour, cudaStream_t s, unsigned long long* usum) {
    const int sms = sm_count();
    const bool trim = h->S >= kTrimStreamsPerSM * sms;
    return with_kind(h->kind, [&](auto kind) {
        constexpr int K = decltype(kind)::value;
        if (h->wbits == 64)
            return trim ? launch_fast_t<uint64_t, K, true>(h, colour, s, sms, usum)
                        : launch_fast_t<uint64_t, K, false>(h, colour, s, sms, usum);
        return trim ? launch_fast_t<uint32_t, K, true>(h, colour, s, sms, usum)
                    : launch_fast_t<uint32_t, K, false>(h, colour, s, sms, usum);
    });
}

}  // namespace isg
