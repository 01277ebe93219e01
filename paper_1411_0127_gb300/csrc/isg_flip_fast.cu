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

// ---------------------------------------------------------------------------
// Several colour passes in one launch (isg_sweep calls of at least 8 sweeps on
// MINSTD and MT19937 lattices with more streams than the launch has warps, in
// the throughput form of the draw phase).  A launch of one pass per colour ends
// with a last wave in which most warps have run out of streams, and the next
// pass cannot start before the whole grid has finished.  Here one persistent
// launch runs npass passes (red, blue, red, ...): an item is (pass p, stream t),
// taken from the ticket counter in pass order, and before it starts it waits
// (bounded) only for the streams whose rows its rows neighbour: the rows of
// stream t read the other colour's spins of rows r +- 1 and r +- L (periodic),
// which streams t_lo .. t_hi (cyclic) wrote in pass p - 1, and they overwrite
// their own colour's words, which those streams read in pass p - 1.  A stream
// also continues its own draws, so t is among them.  Within a pass the streams
// update disjoint rows of one colour and read only the other colour, so the
// order of a pass's items does not change the trajectory.  Pass p takes its
// streams in the order p d, p d + 1, ... (mod S), where d bounds how far (in
// streams) a stream's neighbouring rows reach: item j of pass p then needs only
// items j .. j + 2d of pass p - 1, dispatched S - 2d tickets earlier.  With at
// least W + 2d streams for the W warps of the launch, those have finished by
// the time a warp takes item j, so warps go on from one pass to the next
// without a last wave in which most of them idle.  (Lattices with fewer
// streams keep one launch per pass.)
//
// done[t] counts the passes stream t has completed, over the life of the handle
// (base = the passes of all earlier launches of this kind): an item of pass p
// waits until done[t'] >= base + p for every neighbour t', and when its stores
// are visible sets done[t] = base + p + 1.  Every item waited for has an earlier
// ticket, already taken by a running warp, so the waits end.  A wait that gives
// up sets the error word; every later item sees it and skips its work, so the
// launch ends quickly and the next energy read reports ISG_ERR_TIMEOUT.  The
// flag protocol is what makes the spins and generator states of other SMs
// visible: a finished item fences its lanes' stores and then releases its
// count, a waiting item acquires the counts and fences before any load, so its
// loads see every store of the items it waited for (and, through them, of the
// earlier passes).
constexpr int64_t kSweepPassesPerLaunch = 128;   // 64 sweeps
// Fewest sweeps per call for the multi-pass launches: a launch of a few passes
// has as many waves as the same passes launched one by one (two passes of
// 8192 streams on 4256 warps are 3.85 waves, four either way), and its waits
// at the pass boundaries then cost more than they save.
constexpr int64_t kSweepsMin = 8;
constexpr unsigned kSweepWaitPolls = 1u << 21;   // about a second with the sleeps

struct SweepPlan {
    unsigned long long* done;  // per stream: passes completed
    unsigned long long base;   // passes of the earlier launches
    int64_t npass;             // passes of this launch
    unsigned long long* err;   // error word
    unsigned long long stall;  // testing: pass 1 waits for this many passes too many (0 normally)
    int64_t shift;             // d: pass p starts at stream p d (mod S)
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Whether item (pass p, rows [rb, re)) may start: false if the error word is set
// or a wait gave up (which sets it).  The same answer in every lane.  Not
// inlined, so that its registers do not weigh on the draw loop's (with 32-bit
// item indices: MINSTD 0.5525 -> 0.5266 ps at L = 1024, MT19937 unchanged).
__device__ __noinline__ bool pass_ready(const FlipArgs& a, const SweepPlan& sp, int64_t p, int64_t rb, int64_t re,
                                        int lane) {
    if (*(volatile const unsigned long long*)sp.err != 0ull) return false;
    if (p == 0) return true;  // the previous pass belongs to an earlier, completed launch
    const unsigned long long target = sp.base + (unsigned long long)p + (p == 1 ? sp.stall : 0ull);
    const int64_t rows = a.rows, R = a.R, S = a.S, L = a.L;
    // the streams holding rows rb - L .. re - 1 + L (cyclic): s0, s0 + 1, ... (mod S)
    int64_t lo = rb - L, hi = re - 1 + L;
    if (lo < 0) lo += rows;
    if (hi >= rows) hi -= rows;
    const int64_t s0 = lo / R;
    const int64_t cnt = (re - rb + 2 * L >= rows) ? S : ((hi / R - s0 + S) % S + 1);
    bool ok = true;
    for (int64_t k0 = 0; k0 < cnt && ok; k0 += 32) {
        bool mine = true;
        if (k0 + lane < cnt) {
            int64_t t2 = s0 + k0 + lane;
            if (t2 >= S) t2 -= S;
            mine = false;
            for (unsigned it = 0; it < kSweepWaitPolls; ++it) {
                if (ld_acquire_u64(sp.done + t2) >= target) {
                    mine = true;
                    break;
                }
                if (*(volatile const unsigned long long*)sp.err != 0ull) break;
                __nanosleep(128);
            }
        }
        ok = __all_sync(kFull, mine);
    }
    if (!ok && lane == 0) atomicExch(sp.err, 1ull);
    __syncwarp();
    __threadfence();  // every lane's later loads after the counts acquired above
    return ok;
}

template <typename Word, int KIND>
__global__ void __launch_bounds__(kFastWarps * 32, KIND == ISG_RNG_MT19937 ? 7 : 8)
    flip_sweeps_kernel(FlipArgs a, StreamConst k, Tickets tk, SweepPlan sp) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    extern __shared__ uint32_t smem[];
    constexpr int kRing = KIND == ISG_RNG_MT19937 ? mt_window(kFastSlack) : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* ring = smem + wid * (kRing + 2 * kCondWords);
    uint32_t* cond = ring + kRing;
    // 32-bit item indices: items <= 128 passes x 8192 streams, rows <= 2048^2
    const int S = (int)a.S, items = (int)(sp.npass * a.S), R = (int)a.R, rows = (int)a.rows;
    const int shift = (int)sp.shift;
    int dEsum = 0;
    for (;;) {
        unsigned long long v = 0;
        if (lane == 0) v = atomicAdd(tk.counter, 1ull);
        v = __shfl_sync(kFull, v, 0);
        const int u = (int)(v - tk.base);  // at most items + the launch's warps
        if (u >= items) break;
        const int p = u / S;
        const int t = (u - p * S + (p * shift) % S) % S;
        const int rb = t * R, re = rb + R < rows ? rb + R : rows;
        if (!pass_ready(a, sp, p, rb, re, lane)) continue;
        StreamRegs st;
        load_stream<KIND>(a, t, ring, st, k, lane);
        stream_pass<Word, KIND, kFastSlack, true>(a, (int)(p & 1), rb, re, ring, cond, st, k, lane, dEsum);
        store_stream<KIND>(a, t, ring, st, lane);
        // publish the item: every lane's spin and state stores before the count
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_u64(sp.done + t, sp.base + (unsigned long long)p + 1ull);
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    for (int sh = 16; sh; sh >>= 1) dEsum += __shfl_xor_sync(kFull, dEsum, sh);
    if (lane == 0 && dEsum != 0) atomicAdd((unsigned long long*)a.dE, (unsigned long long)(long long)dEsum);
}

// d: the streams holding the rows r - L .. r + L of a stream's rows r lie within
// d streams of it.
static int64_t sweep_reach(const isg_sim* h) { return (h->L + h->R - 1) / h->R + 1; }

template <typename Word, int KIND>
static int sweep_occupancy() {
    constexpr int kRing = KIND == ISG_RNG_MT19937 ? mt_window(kFastSlack) : 0;
    const size_t smem = (size_t)kFastWarps * (kRing + 2 * kCondWords) * sizeof(uint32_t);
    static std::atomic<int> occ_cache[kDeviceSlots];
    return occupancy_cached(occ_cache, flip_sweeps_kernel<Word, KIND>, kFastWarps * 32, smem);
}

template <typename Word, int KIND>
static cudaError_t launch_sweeps_t(isg_sim* h, int64_t npass, cudaStream_t s, int sms) {
    const FlipArgs a = make_flip_args(h, 0);
    const StreamConst k = stream_const();
    Tickets tk;
    tk.counter = (unsigned long long*)(h->scal + 3);
    tk.base = h->tickets;
    SweepPlan sp;
    sp.done = h->done;
    sp.base = h->passes;
    sp.npass = npass;
    sp.err = (unsigned long long*)(h->scal + 5);
    sp.stall = h->stall_next ? 1ull : 0ull;
    sp.shift = sweep_reach(h);
    constexpr int kRing = KIND == ISG_RNG_MT19937 ? mt_window(kFastSlack) : 0;
    const size_t smem = (size_t)kFastWarps * (kRing + 2 * kCondWords) * sizeof(uint32_t);
    const int64_t blocks = (int64_t)sms * sweep_occupancy<Word, KIND>();  // more streams than warps: fill the GPU
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)blocks);
    lc.blockDim = dim3(kFastWarps * 32);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&lc, flip_sweeps_kernel<Word, KIND>, a, k, tk, sp);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    h->tickets += (unsigned long long)(npass * h->S) + (unsigned long long)blocks * kFastWarps;
    h->passes += (unsigned long long)npass;
    h->stall_next = false;
    return e;
}

bool sweeps_in_one_launch(const isg_sim* h, int64_t n) {
    // Parisi-Rapuano keeps one launch per pass: with 8 CTAs per SM the last wave
    // of its passes still holds enough warps to keep issuing, and the multi-pass
    // form measured 0.839 against 0.832 ps at L = 1024 (MT19937 1.052 against
    // 1.094, MINSTD 0.552 against 0.607)
    if (!h->done || n < kSweepsMin || h->kind == ISG_RNG_PARISI_RAPUANO) return false;
    const int sms = sm_count();
    if (h->S < kTrimStreamsPerSM * sms) return false;
    const int occ = with_kind(h->kind, [&](auto kind) {
        constexpr int K = decltype(kind)::value;
        return h->wbits == 64 ? sweep_occupancy<uint64_t, K>() : sweep_occupancy<uint32_t, K>();
    });
    const int64_t warps = (int64_t)sms * occ * kFastWarps;
    return h->S >= warps + 2 * sweep_reach(h);
}

cudaError_t launch_sweeps(isg_sim* h, int64_t n, cudaStream_t s) {
    const int sms = sm_count();
    for (int64_t left = 2 * n; left > 0;) {
        const int64_t np = left < kSweepPassesPerLaunch ? left : kSweepPassesPerLaunch;
        const cudaError_t e = with_kind(h->kind, [&](auto kind) {
            constexpr int K = decltype(kind)::value;
            return h->wbits == 64 ? launch_sweeps_t<uint64_t, K>(h, np, s, sms)
                                  : launch_sweeps_t<uint32_t, K>(h, np, s, sms);
        });
        if (e != cudaSuccess) return e;
        left -= np;
    }
    return cudaSuccess;
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
