// isg_batch.cu -- batched persistent engine: many disorder samples of uneven L,
// two replicas each, swept by one persistent launch per group of sweeps.
//
// The paper fills the GPU with many samples at once (Sec. 2, coded samples k;
// Sec. 4 results, psFlip against k).  Here a batch is a set of ordinary
// lattices (64-bit words whatever L, so one kernel template serves every L), two
// per sample with the same couplings and different spin seeds, and:
//   * on the host their RNG streams are packed into bundles: a lattice with more
//     than `capacity` streams is one bundle; smaller lattices are packed
//     together, at most `capacity` streams per bundle;
//   * CTAs of WARPS warps (one or two per SM) take task after task from a
//     counter: a task is a bundle for all sweeps of the launch or, for a bundle
//     much longer than the average work per CTA, one of up to 8 consecutive
//     parts of its sweeps (split_tasks), which waits, bounded, for the previous
//     part; warp w sweeps entries w, w + WARPS, ... of the bundle, and a block
//     barrier separates the colour passes; no lattice spans two CTAs at once,
//     so no grid-wide barrier is needed;
//   * when a bundle has at most WARPS streams each warp can keep its stream's
//     generator state (MT19937 words in shared memory) for the whole task;
//   * the shape, the capacity, that residency and the words per lane form the
//     execution configuration (isg_batch_set_config), chosen by the autotuner;
//   * the task counter and flags return to zero when the last CTA leaves, so
//     the launch is captured once into a CUDA graph and replayed.
// Every lattice follows exactly the trajectory it has alone (same map from
// site to stream and draw), which the tests check against isg_sweep and the
// CPU oracle.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstring>
#include <new>
#include <vector>

#include "isg_bundles.cuh"
#include "isg_stream.cuh"

struct isg_batch {
    int n = 0;                          // samples
    int kind = 0;
    std::vector<isg_sim*> reps;         // 2n lattices, replica-major
    isg::FlipArgs* d_reps = nullptr;    // per-lattice descriptors
    int2* d_entries = nullptr;          // (lattice, stream) grouped by bundle
    int* d_boff = nullptr;              // bundle offsets into d_entries
    unsigned* d_ctr = nullptr;          // [0] next task, [1] CTAs done, [2] dependency-wait error
    isg::BundleTasks tasks;             // launch order of the bundles, long ones split in two
    int nbundles = 0;                   // bundles, or (pass engine) items
    int2* d_items = nullptr;            // pass engine: (lattice, stream), longest streams first
    unsigned* d_done = nullptr;         // pass engine: per lattice, items completed in the running launch
    int stall = -1;                     // pass engine test hook (isg_batch_test_stall)
    int64_t attempts_per_sweep = 0;
    isg::BundleConfig cfg;              // execution configuration (isg_batch_set_config)
    cudaStream_t cap = nullptr;         // private stream used for graph capture
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    int graph_group = 0;
};

namespace isg {

constexpr int kBatchSlack = 512;  // MT19937 window per warp: 624 + 512 words (32 warps fit in 227 KiB)

struct BatchArgs {
    const FlipArgs* reps;
    const int2* entries;
    const int* boff;
    const int* bsweeps;   // sweeps of each bundle in this launch, or NULL: `sweeps` for all
    int nbundles;
    int sweeps;
    int resident;         // keep the generator state of bundles that fit in the CTA for the whole launch
    unsigned* ctr;        // [0] next task, [1] CTAs done, [2] sticky error: a dependency wait gave up
    const int4* tasks;    // NULL: task i is bundle i, all its sweeps; else see BundleTasks
    int ntasks;
    unsigned* done;       // per task: its sweeps are done (set by parts that have a next part); zeroed at launch end
};

// Iterations of the wait for a previous part (each about 0.25 us of sleep): seconds
// beyond any real wait, after which the kernel sets ctr[2] and skips the task.
constexpr int kDepWaitLimit = 1 << 24;

// CTA shapes of the bundle kernel (warps per CTA, CTAs per SM); see BundleConfig.
struct BundleShape {
    int warps, per_sm;
};
constexpr BundleShape kBundleShapes[kBundleShapeCount] = {{32, 1}, {24, 1}, {16, 1}, {16, 2}};

template <int KIND, int WARPS, int PER_SM, int WPT>
__global__ void __launch_bounds__(WARPS * 32, PER_SM) batch_kernel(BatchArgs b, StreamConst k) {
    constexpr int kBatchWarps = WARPS;
    extern __shared__ uint32_t smem[];
    __shared__ int s_task, s_ok;
    constexpr int kRing = KIND == ISG_RNG_MT19937 ? mt_window(kBatchSlack) : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* ring = smem + wid * (kRing + 2 * WPT * kCondWords);
    uint32_t* cond = ring + kRing;
    const int ntasks = b.tasks ? b.ntasks : b.nbundles;
    for (;;) {
        if (threadIdx.x == 0) s_task = (int)atomicAdd(&b.ctr[0], 1u);
        __syncthreads();
        const int tid = s_task;
        __syncthreads();
        if (tid >= ntasks) break;
        const int4 tk = b.tasks ? b.tasks[tid] : make_int4(tid, 0, -1, 0);
        const int bid = tk.x;
        int sweeps = b.bsweeps ? b.bsweeps[bid] : b.sweeps;
        if (tk.y > 0) sweeps = sweeps * tk.y / tk.w - sweeps * (tk.y - 1) / tk.w;  // part y of w
        if (tk.z >= 0) {
            // the previous part of this bundle's sweeps is task tk.z, taken
            // earlier by a running CTA: wait (bounded) until it has finished
            if (threadIdx.x == 0) {
                int ok = 0;
                for (int it = 0; it < kDepWaitLimit; ++it) {
                    if (*(volatile const unsigned*)(b.done + tk.z) != 0u) {
                        ok = 1;
                        break;
                    }
                    __nanosleep(256);
                }
                __threadfence();
                if (!ok) atomicExch(&b.ctr[2], 1u);
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) continue;
        }
        const int e0 = b.boff[bid], n = b.boff[bid + 1] - e0;
        const bool resident = b.resident && n <= kBatchWarps;
        StreamRegs st;
        if (resident && wid < n) {
            const int2 e = b.entries[e0 + wid];
            load_stream<KIND>(b.reps[e.x], e.y, ring, st, k, lane);
        }
        for (int pass = 0; pass < 2 * sweeps; ++pass) {
            for (int j = wid; j < n; j += kBatchWarps) {
                const int2 e = b.entries[e0 + j];
                const FlipArgs& g = b.reps[e.x];
                if (!resident) load_stream<KIND>(g, e.y, ring, st, k, lane);
                // The fields the pass reads, held in registers: read through the
                // descriptor in global memory they would be re-read after every
                // store to the spin planes.
                FlipArgs a;
                a.planes = g.planes;
                a.plane_bytes = g.plane_bytes;
                a.L = g.L;
                a.half = g.half;
                a.W = g.W;
                a.nt = g.nt;
                a.cmp1 = g.cmp1;
                a.cmp2 = g.cmp2;
                a.cmp3 = g.cmp3;
                int dE = 0;
                const int64_t rb = (int64_t)e.y * g.R, re = rb + g.R < g.rows ? rb + g.R : g.rows;
                stream_pass<uint64_t, KIND, kBatchSlack, true, WPT>(a, pass & 1, rb, re, ring, cond, st, k, lane, dE);
                if (!resident) store_stream<KIND>(g, e.y, ring, st, lane);
                for (int sh = 16; sh; sh >>= 1) dE += __shfl_xor_sync(kFull, dE, sh);
                if (lane == 0 && dE != 0) atomicAdd((unsigned long long*)g.dE, (unsigned long long)(long long)dE);
            }
            __syncthreads();
        }
        if (resident && wid < n) {
            const int2 e = b.entries[e0 + wid];
            store_stream<KIND>(b.reps[e.x], e.y, ring, st, lane);
        }
        if (tk.y > 0 && tk.y < tk.w) {  // publish this part to the one that waits for it
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicExch(b.done + tid, 1u);
            }
        }
    }
    // the last CTA to leave returns the counters and flags to zero for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(&b.ctr[1], 1u);
        if (done == gridDim.x - 1) {
            for (int t = 0; b.tasks && t < b.ntasks; ++t) b.done[t] = 0u;
            atomicExch(&b.ctr[0], 0u);
            atomicExch(&b.ctr[1], 0u);
            __threadfence();
        }
    }
}

static size_t batch_smem(int kind, int warps, int wpt) {
    const int ring = kind == ISG_RNG_MT19937 ? mt_window(kBatchSlack) : 0;
    return (size_t)warps * (ring + 2 * wpt * kCondWords) * sizeof(uint32_t);
}

// f(std::integral_constant<int, shape index>) for a runtime shape index.
template <class F>
static auto with_shape(int shape, F&& f) {
    switch (shape) {
        case 1: return f(std::integral_constant<int, 1>{});
        case 2: return f(std::integral_constant<int, 2>{});
        case 3: return f(std::integral_constant<int, 3>{});
        default: return f(std::integral_constant<int, 0>{});
    }
}

// f(std::integral_constant<int, words per lane>) for a runtime value of 1 or 2.
template <class F>
static auto with_wpt(int wpt, F&& f) {
    if (wpt == 2) return f(std::integral_constant<int, 2>{});
    return f(std::integral_constant<int, 1>{});
}

cudaError_t prepare_bundle_kernel(int kind, const BundleConfig& cfg) {
    return with_kind(kind, [&](auto kc) {
        return with_shape(cfg.shape, [&](auto sc) {
            return with_wpt(cfg.wpt, [&](auto wc) {
                constexpr BundleShape sh = kBundleShapes[decltype(sc)::value];
                return cudaFuncSetAttribute(
                    batch_kernel<decltype(kc)::value, sh.warps, sh.per_sm, decltype(wc)::value>,
                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem(kind, sh.warps, decltype(wc)::value));
            });
        });
    });
}

cudaError_t launch_bundle_kernel(int kind, const BundleConfig& cfg, const FlipArgs* reps, const int2* entries,
                                 const int* boff, const int* bsweeps, int nbundles, int sweeps, unsigned* ctr,
                                 cudaStream_t s, const BundleTasks* tasks) {
    if (nbundles <= 0) return cudaSuccess;
    BatchArgs a;
    a.reps = reps;
    a.entries = entries;
    a.boff = boff;
    a.bsweeps = bsweeps;
    a.nbundles = nbundles;
    a.sweeps = sweeps;
    a.resident = cfg.resident;
    a.ctr = ctr;
    a.tasks = tasks ? tasks->d_tasks : nullptr;
    a.ntasks = tasks ? tasks->ntasks : nbundles;
    a.done = tasks ? tasks->d_done : nullptr;
    const StreamConst k = stream_const();
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return with_kind(kind, [&](auto kc) {
        return with_shape(cfg.shape, [&](auto sc) {
            return with_wpt(cfg.wpt, [&](auto wc) {
                constexpr BundleShape sh = kBundleShapes[decltype(sc)::value];
                constexpr int wpt = decltype(wc)::value;
                const int grid = std::max(1, std::min(sms * sh.per_sm, a.ntasks));
                batch_kernel<decltype(kc)::value, sh.warps, sh.per_sm, wpt>
                    <<<grid, sh.warps * 32, batch_smem(kind, sh.warps, wpt), s>>>(a, k);
                return cudaGetLastError();
            });
        });
    });
}

int bundle_warps(const BundleConfig& cfg) { return cfg.shape >= kPassShape ? 4 : kBundleShapes[cfg.shape].warps; }

// ---------------------------------------------------------------------------
// Pass engines (shapes kPassShape and kGroupShape): no bundles and no block
// barriers.  Persistent 4-warp CTAs take items by ticket, longest streams
// first; an item is one stream of one lattice in one colour pass: a warp loads
// the stream's generator state, sweeps the stream's rows with the same
// stream_pass as the single-lattice kernel (throughput form) and stores the
// state back.  With kPassShape every colour pass is one launch.  With
// kGroupShape one launch runs all the passes of a sweep group, items taken pass
// by pass: a lattice's pass p reads the spins and continues the generator
// states its pass p - 1 left, so an item of pass p first waits (bounded) until
// its lattice has completed all items of the earlier passes (a per-lattice
// count); other lattices need not wait, so passes overlap across lattices.
// Items are taken in pass order, so every item waited for is already held by a
// running warp: the waits always end.  The last CTA to leave returns the
// ticket counter (and the lattice counts) to zero, so the launches are
// captured once into a CUDA graph and replayed.
constexpr int kPassWarps = 4;
constexpr int kPassSlack = 1024;

struct PassArgs {
    const FlipArgs* reps;
    const int2* items;   // (lattice, stream), longest streams first
    int nitems;
    int npasses;         // passes of this launch (1 for a launch per pass)
    int pass0;           // index of its first pass (colour = index & 1)
    const int* limit;    // per lattice: passes to run, or NULL for all (a lattice
                         // with fewer skips the items of its later passes)
    int nlat;
    int stall;           // test hook: this lattice's pass-1 items wait for one item too many (-1: none)
    unsigned* ctr;       // [0] next ticket, [1] CTAs done, [2] sticky error: a wait gave up
    unsigned* done;      // per lattice: items completed in this launch
};

template <int KIND, int WPT, bool GROUP>
__global__ void __launch_bounds__(kPassWarps * 32, 7) pass_kernel(PassArgs pa, StreamConst k) {
    extern __shared__ uint32_t smem[];
    constexpr int kRing = KIND == ISG_RNG_MT19937 ? mt_window(kPassSlack) : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* ring = smem + wid * (kRing + 2 * WPT * kCondWords);
    uint32_t* cond = ring + kRing;
    const unsigned total = (unsigned)pa.npasses * (unsigned)pa.nitems;
    for (;;) {
        unsigned v = 0;
        if (lane == 0) v = atomicAdd(&pa.ctr[0], 1u);
        v = __shfl_sync(kFull, v, 0);
        if (v >= total) break;
        const int p = GROUP ? (int)(v / (unsigned)pa.nitems) : 0;
        const int2 e = pa.items[v - (unsigned)p * (unsigned)pa.nitems];
        if (pa.limit && pa.pass0 + p >= pa.limit[e.x]) continue;  // this lattice is done for the launch
        const FlipArgs& g = pa.reps[e.x];
        if (GROUP && p > 0) {
            const unsigned need = (unsigned)p * (unsigned)g.S + (e.x == pa.stall && p == 1 ? 1u : 0u);
            int ok = 1;
            if (lane == 0) {
                ok = 0;
                for (int it = 0; it < kDepWaitLimit; ++it) {
                    if (*(volatile const unsigned*)(pa.done + e.x) >= need) {
                        ok = 1;
                        break;
                    }
                    __nanosleep(256);
                }
                if (!ok) atomicExch(&pa.ctr[2], 1u);
            }
            ok = __shfl_sync(kFull, ok, 0);
            __threadfence();
            if (!ok) {  // counted but not swept: the error is reported, and nothing waits on it forever
                if (lane == 0) atomicAdd(pa.done + e.x, 1u);
                continue;
            }
        }
        FlipArgs a;  // the fields stream_pass reads, in registers
        a.planes = g.planes;
        a.plane_bytes = g.plane_bytes;
        a.L = g.L;
        a.half = g.half;
        a.W = g.W;
        a.nt = g.nt;
        a.cmp1 = g.cmp1;
        a.cmp2 = g.cmp2;
        a.cmp3 = g.cmp3;
        StreamRegs st;
        load_stream<KIND>(g, e.y, ring, st, k, lane);
        int dE = 0;
        const int64_t rb = (int64_t)e.y * g.R, re = rb + g.R < g.rows ? rb + g.R : g.rows;
        stream_pass<uint64_t, KIND, kPassSlack, true, WPT>(a, (pa.pass0 + p) & 1, rb, re, ring, cond, st, k, lane, dE);
        store_stream<KIND>(g, e.y, ring, st, lane);
        for (int sh = 16; sh; sh >>= 1) dE += __shfl_xor_sync(kFull, dE, sh);
        if (lane == 0 && dE != 0) atomicAdd((unsigned long long*)g.dE, (unsigned long long)(long long)dE);
        if (GROUP) {  // publish the item: every lane's spin and state stores before the count
            __threadfence();
            __syncwarp();
            if (lane == 0) atomicAdd(pa.done + e.x, 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned fin = atomicAdd(&pa.ctr[1], 1u);
        if (fin == gridDim.x - 1) {
            for (int l = 0; GROUP && l < pa.nlat; ++l) pa.done[l] = 0u;
            atomicExch(&pa.ctr[0], 0u);
            atomicExch(&pa.ctr[1], 0u);
            __threadfence();
        }
    }
}

static size_t pass_smem(int kind, int wpt) {
    const int ring = kind == ISG_RNG_MT19937 ? mt_window(kPassSlack) : 0;
    return (size_t)kPassWarps * (ring + 2 * wpt * kCondWords) * sizeof(uint32_t);
}

// `sweeps` sweeps of every lattice of the item list: one launch per colour
// pass (group = false) or one launch for all of them (group = true).
static cudaError_t launch_passes(int kind, int wpt, bool group, PassArgs pa, int sweeps, cudaStream_t s);

cudaError_t launch_pass_items(int kind, const FlipArgs* reps, const int2* items, int nitems, const int* limit,
                              int sweeps, unsigned* ctr, cudaStream_t s) {
    PassArgs pa;
    pa.reps = reps;
    pa.items = items;
    pa.nitems = nitems;
    pa.npasses = 0;
    pa.pass0 = 0;
    pa.limit = limit;
    pa.nlat = 0;
    pa.stall = -1;
    pa.ctr = ctr;
    pa.done = nullptr;
    return launch_passes(kind, 1, false, pa, sweeps, s);
}

static cudaError_t launch_passes(int kind, int wpt, bool group, PassArgs pa, int sweeps, cudaStream_t s) {
    if (pa.nitems <= 0 || sweeps <= 0) return cudaSuccess;
    const StreamConst k = stream_const();
    const size_t smem = pass_smem(kind, wpt);
    auto run = [&](auto kern, std::atomic<int> (&occ_cache)[kDeviceSlots]) {
        const int occ = occupancy_cached(occ_cache, kern, kPassWarps * 32, smem);
        int64_t grid = (int64_t)sm_count() * occ;
        const int64_t need = (pa.nitems + kPassWarps - 1) / kPassWarps;
        if (grid > need) grid = need;
        const int launches = group ? 1 : 2 * sweeps;
        pa.npasses = group ? 2 * sweeps : 1;
        for (int l = 0; l < launches; ++l) {
            pa.pass0 = l;
            kern<<<(unsigned)grid, kPassWarps * 32, smem, s>>>(pa, k);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    return with_kind(kind, [&](auto kc) {
        return with_wpt(wpt, [&](auto wc) {
            constexpr int K = decltype(kc)::value, WPT = decltype(wc)::value;
            static std::atomic<int> occ_pass[kDeviceSlots], occ_group[kDeviceSlots];
            return group ? run(pass_kernel<K, WPT, true>, occ_group) : run(pass_kernel<K, WPT, false>, occ_pass);
        });
    });
}

void plan_bundles(const std::vector<isg_sim*>& reps, std::vector<int2>& entries, std::vector<int>& boff,
                  std::vector<int>* order, int capacity) {
    const int cap = capacity;  // streams per packed bundle
    struct Bundle {
        std::vector<int2> e;
        std::vector<int> members;
        double work;
    };
    std::vector<Bundle> bundles;
    std::vector<int> small;
    const int nrep = (int)reps.size();
    for (int r = 0; r < nrep; ++r) {
        const isg_sim* h = reps[r];
        if (h->S > cap) {
            Bundle bd;
            for (int64_t t = 0; t < h->S; ++t) bd.e.push_back(make_int2(r, (int)t));
            bd.members.push_back(r);
            bd.work = (double)((h->S + cap - 1) / cap) * (double)h->R * h->half;
            bundles.push_back(bd);
        } else {
            small.push_back(r);
        }
    }
    std::stable_sort(small.begin(), small.end(), [&](int x, int y) {
        const isg_sim *a = reps[x], *c = reps[y];
        if (a->S != c->S) return a->S > c->S;
        return a->L > c->L;
    });
    std::vector<Bundle> packs;
    for (int r : small) {
        const isg_sim* h = reps[r];
        Bundle* fit = nullptr;
        for (Bundle& p : packs)
            if ((int64_t)p.e.size() + h->S <= cap) { fit = &p; break; }
        if (!fit) { packs.push_back(Bundle{{}, {}, 0.0}); fit = &packs.back(); }
        for (int64_t t = 0; t < h->S; ++t) fit->e.push_back(make_int2(r, (int)t));
        fit->members.push_back(r);
        fit->work = std::max(fit->work, (double)h->R * h->half);
    }
    bundles.insert(bundles.end(), packs.begin(), packs.end());
    std::stable_sort(bundles.begin(), bundles.end(), [](const Bundle& x, const Bundle& y) { return x.work > y.work; });
    entries.clear();
    boff.assign(1, 0);
    if (order) order->clear();
    for (const Bundle& bd : bundles) {
        entries.insert(entries.end(), bd.e.begin(), bd.e.end());
        boff.push_back((int)entries.size());
        if (order) {  // members of each bundle, -1 terminated
            order->insert(order->end(), bd.members.begin(), bd.members.end());
            order->push_back(-1);
        }
    }
}

static cudaError_t batch_launch(isg_batch* b, int sweeps, cudaStream_t s) {
    if (b->cfg.shape >= kPassShape) {
        PassArgs pa;
        pa.reps = b->d_reps;
        pa.items = b->d_items;
        pa.nitems = b->nbundles;
        pa.npasses = 0;
        pa.pass0 = 0;
        pa.limit = nullptr;
        pa.nlat = (int)b->reps.size();
        pa.stall = b->stall;
        pa.ctr = b->d_ctr;
        pa.done = b->d_done;
        return launch_passes(b->kind, b->cfg.wpt, b->cfg.shape == kGroupShape, pa, sweeps, s);
    }
    return launch_bundle_kernel(b->kind, b->cfg, b->d_reps, b->d_entries, b->d_boff, nullptr, b->nbundles, sweeps,
                                b->d_ctr, s, &b->tasks);
}

// Task order of a launch.  A persistent CTA takes whole bundles, so a bundle far
// longer than the average work per CTA decides when the launch ends (e.g. 162
// lattices of L = 192, one bundle each, on 152 CTAs: ten CTAs run two).  A
// bundle with more than kSplitDiv-th of that average is split into up to
// kSplitMax consecutive parts of its sweeps: all first parts go first, then all
// second parts in the same order (each waiting for its own previous part, which
// a running CTA took earlier), and so on, then the other bundles, longest first.
constexpr int kSplitMax = 8, kSplitDiv = 6;
static std::vector<int4> split_tasks(const isg_batch* b, const std::vector<int2>& entries,
                                     const std::vector<int>& boff, int ctas) {
    const int nb = (int)boff.size() - 1, warps = bundle_warps(b->cfg);
    std::vector<double> work(nb, 0.0);
    double total = 0.0;
    for (int i = 0; i < nb; ++i) {
        double per_round = 0.0;
        for (int j = boff[i]; j < boff[i + 1]; ++j) {
            const isg_sim* h = b->reps[entries[j].x];
            per_round = std::max(per_round, (double)h->R * h->half);
        }
        const int n = boff[i + 1] - boff[i];
        work[i] = (double)((n + warps - 1) / warps) * per_round;
        total += work[i];
    }
    const double piece = total / std::max(1, ctas) / kSplitDiv;
    std::vector<int> parts(nb, 1);
    int maxparts = 1;
    for (int i = 0; i < nb; ++i) {
        parts[i] = (int)std::min<double>(kSplitMax, std::ceil(work[i] / piece));
        if (parts[i] < 1) parts[i] = 1;
        maxparts = std::max(maxparts, parts[i]);
    }
    std::vector<int4> out;
    std::vector<int> prev(nb, -1);
    for (int p = 1; p <= maxparts; ++p)
        for (int i = 0; i < nb; ++i)
            if (parts[i] > 1 && p <= parts[i]) {
                out.push_back(make_int4(i, p, prev[i], parts[i]));
                prev[i] = (int)out.size() - 1;
            }
    for (int i = 0; i < nb; ++i)
        if (parts[i] == 1) out.push_back(make_int4(i, 0, -1, 1));
    return out;
}

// Bundles for the configuration's capacity, uploaded (the entries keep their
// number; the offsets are reallocated); the captured graph is dropped.
static int batch_plan(isg_batch* b) {
    isg_sim* h0 = b->reps[0];
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->graph_group = 0;
    if (b->cfg.shape >= kPassShape) {
        // every stream of every lattice is an item; the longest go first
        std::vector<int2> items;
        std::vector<int64_t> len;
        for (int r = 0; r < (int)b->reps.size(); ++r) {
            const isg_sim* h = b->reps[r];
            for (int64_t t = 0; t < h->S; ++t) items.push_back(make_int2(r, (int)t));
        }
        auto draws = [&](const int2& it) {
            const isg_sim* h = b->reps[it.x];
            const int64_t r0 = (int64_t)it.y * h->R, r1 = std::min(r0 + h->R, h->rows);
            return (r1 - r0) * h->half;
        };
        std::stable_sort(items.begin(), items.end(), [&](const int2& x, const int2& y) { return draws(x) > draws(y); });
        if (!b->d_items) b->d_items = (int2*)dev_alloc(h0, items.size() * sizeof(int2));
        if (!b->d_done) {
            b->d_done = (unsigned*)dev_alloc(h0, b->reps.size() * sizeof(unsigned));
            if (b->d_done && cudaMemset(b->d_done, 0, b->reps.size() * sizeof(unsigned)) != cudaSuccess) {
                set_error("isg_batch: clearing the lattice counts failed");
                return ISG_ERR_CUDA;
            }
        }
        b->stall = -1;
        if (!b->d_items || !b->d_done) {
            set_error("isg_batch: device allocation failed");
            return ISG_ERR_NOMEM;
        }
        b->nbundles = (int)items.size();
        const cudaError_t e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice);
        return e == cudaSuccess ? ISG_OK : cuda_fail(e, "isg_batch: pass plan");
    }
    std::vector<int2> entries;
    std::vector<int> boff;
    plan_bundles(b->reps, entries, boff, nullptr, b->cfg.capacity);
    dev_free(h0, b->d_boff);
    b->d_boff = (int*)dev_alloc(h0, boff.size() * sizeof(int));
    if (!b->d_entries) b->d_entries = (int2*)dev_alloc(h0, entries.size() * sizeof(int2));
    if (!b->d_boff || !b->d_entries) {
        set_error("isg_batch: device allocation failed");
        return ISG_ERR_NOMEM;
    }
    b->nbundles = (int)boff.size() - 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const std::vector<int4> tasks = split_tasks(b, entries, boff, sms * kBundleShapes[b->cfg.shape].per_sm);
    dev_free(h0, b->tasks.d_tasks);
    dev_free(h0, b->tasks.d_done);
    b->tasks.ntasks = (int)tasks.size();
    b->tasks.d_tasks = (int4*)dev_alloc(h0, tasks.size() * sizeof(int4));
    b->tasks.d_done = (unsigned*)dev_alloc(h0, tasks.size() * sizeof(unsigned));
    if (!b->tasks.d_tasks || !b->tasks.d_done) {
        set_error("isg_batch: device allocation failed");
        return ISG_ERR_NOMEM;
    }
    cudaError_t e = cudaMemcpy(b->d_entries, entries.data(), entries.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_boff, boff.data(), boff.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->tasks.d_tasks, tasks.data(), tasks.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->tasks.d_done, 0, tasks.size() * sizeof(unsigned));
    if (e == cudaSuccess) e = prepare_bundle_kernel(b->kind, b->cfg);
    return e == cudaSuccess ? ISG_OK : cuda_fail(e, "isg_batch: bundle plan");
}

static void batch_free(isg_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (!b->reps.empty() && b->reps[0]) {
        dev_free(b->reps[0], b->d_reps);
        dev_free(b->reps[0], b->d_entries);
        dev_free(b->reps[0], b->d_boff);
        dev_free(b->reps[0], b->d_ctr);
        dev_free(b->reps[0], b->tasks.d_tasks);
        dev_free(b->reps[0], b->tasks.d_done);
        dev_free(b->reps[0], b->d_items);
        dev_free(b->reps[0], b->d_done);
    }
    for (isg_sim* h : b->reps) destroy_sim(h);
    delete b;
}

}  // namespace isg

using namespace isg;

extern "C" {

int isg_batch_create(int n, const int* L, const uint64_t* seed_J, const uint64_t* seed_spin, const double* beta,
                     int rng_kind, isg_batch** out) {
    if (!out) { set_error("isg_batch_create: out is NULL"); return ISG_ERR_ARG; }
    *out = nullptr;
    if (n < 1 || !L || !seed_J || !seed_spin || !beta) { set_error("isg_batch_create: bad argument"); return ISG_ERR_ARG; }
    if (!rng_kind_valid(rng_kind)) {
        set_error("isg_batch_create: unknown rng_kind %d", rng_kind);
        return ISG_ERR_ARG;
    }
    for (int s = 0; s < n; ++s)
        if (L[s] < 4 || L[s] > 2048 || (L[s] & 1) || !(beta[s] > 0.0)) {
            set_error("isg_batch_create: sample %d has L=%d beta=%g", s, L[s], beta[s]);
            return ISG_ERR_ARG;
        }
    isg_batch* b = new (std::nothrow) isg_batch();
    if (!b) { set_error("isg_batch_create: out of host memory"); return ISG_ERR_NOMEM; }
    b->n = n;
    b->kind = rng_kind;
    b->reps.assign(2 * n, nullptr);
    for (int r = 0; r < 2 * n; ++r) {
        const int s = r / 2;
        const int rc = create_sim(L[s], seed_J[s], seed_spin[r], seed_spin[r], beta[s], rng_kind, true, &b->reps[r]);
        if (rc) { batch_free(b); return rc; }
        b->attempts_per_sweep += (int64_t)L[s] * L[s] * L[s];
    }

    // bundles: big lattices alone, small ones first-fit into `capacity` entries
    std::vector<FlipArgs> desc(2 * n);
    for (int r = 0; r < 2 * n; ++r) desc[r] = make_flip_args(b->reps[r], 0);
    isg_sim* h0 = b->reps[0];
    b->d_reps = (FlipArgs*)dev_alloc(h0, desc.size() * sizeof(FlipArgs));
    b->d_ctr = (unsigned*)dev_alloc(h0, 3 * sizeof(unsigned));
    if (!b->d_reps || !b->d_ctr) {
        batch_free(b);
        set_error("isg_batch_create: device allocation failed");
        return ISG_ERR_NOMEM;
    }
    if (const int rc = batch_plan(b)) {
        batch_free(b);
        return rc;
    }
    cudaError_t e = cudaMemcpy(b->d_reps, desc.data(), desc.size() * sizeof(FlipArgs), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_ctr, 0, 3 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "isg_batch_create");
    }
    *out = b;
    return ISG_OK;
}

void isg_batch_destroy(isg_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    batch_free(b);
}

int isg_batch_info(const isg_batch* b, int* samples, int* bundles, int64_t* attempts_per_sweep) {
    if (!b) { set_error("isg_batch_info: NULL batch"); return ISG_ERR_ARG; }
    if (samples) *samples = b->n;
    if (bundles) *bundles = b->nbundles;
    if (attempts_per_sweep) *attempts_per_sweep = b->attempts_per_sweep;
    return ISG_OK;
}

int isg_batch_set_config(isg_batch* b, int shape, int capacity, int resident, int words_per_lane) {
    if (!b || shape < 0 || shape > kGroupShape || capacity < 0 || (resident != 0 && resident != 1) ||
        (words_per_lane != 1 && words_per_lane != 2)) {
        set_error("isg_batch_set_config: bad argument");
        return ISG_ERR_ARG;
    }
    BundleConfig cfg;
    cfg.shape = shape;
    cfg.wpt = words_per_lane;
    const int warps = bundle_warps(cfg);
    cfg.capacity = capacity == 0 ? warps : capacity;
    cfg.resident = resident;
    if (cfg.capacity > warps) {
        set_error("isg_batch_set_config: capacity %d exceeds the %d warps of shape %d", capacity, warps, shape);
        return ISG_ERR_ARG;
    }
    const cudaError_t e = cudaDeviceSynchronize();  // no launch of the old plan may be in flight
    if (e != cudaSuccess) return cuda_fail(e, "isg_batch_set_config");
    b->cfg = cfg;
    return batch_plan(b);
}

int isg_batch_get_config(const isg_batch* b, int* shape, int* capacity, int* resident, int* words_per_lane) {
    if (!b) { set_error("isg_batch_get_config: NULL batch"); return ISG_ERR_ARG; }
    if (shape) *shape = b->cfg.shape;
    if (capacity) *capacity = b->cfg.capacity;
    if (resident) *resident = b->cfg.resident;
    if (words_per_lane) *words_per_lane = b->cfg.wpt;
    return ISG_OK;
}

int isg_batch_test_stall(isg_batch* b) {
    if (!b) { set_error("isg_batch_test_stall: NULL batch"); return ISG_ERR_ARG; }
    if (b->cfg.shape == kPassShape) {
        set_error("isg_batch_test_stall: the pass launches have no waits");
        return ISG_ERR_STATE;
    }
    if (b->cfg.shape == kGroupShape) {  // the smallest lattice's pass-1 items wait for one item too many
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        b->graph_group = 0;
        int best = 0;
        for (int r = 1; r < (int)b->reps.size(); ++r)
            if (b->reps[r]->S < b->reps[best]->S) best = r;
        b->stall = best;
        return ISG_OK;
    }
    const int n = b->tasks.ntasks;
    if (n < 2) { set_error("isg_batch_test_stall: fewer than two tasks"); return ISG_ERR_STATE; }
    int4 t;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&t, b->tasks.d_tasks + (n - 1), sizeof(int4), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "isg_batch_test_stall");
    t.z = n - 1;  // its own flag: a part-0 or last part never sets it
    if (t.y == 0) {
        t.y = 1;
        t.w = 1;
    }
    e = cudaMemcpy(b->tasks.d_tasks + (n - 1), &t, sizeof(int4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "isg_batch_test_stall");
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->graph_group = 0;
    return ISG_OK;
}

int isg_batch_member(isg_batch* b, int i, isg_sim** out) {
    if (!b || !out || i < 0 || i >= 2 * b->n) { set_error("isg_batch_member: bad argument"); return ISG_ERR_ARG; }
    *out = b->reps[i];
    return ISG_OK;
}

int isg_batch_run(isg_batch* b, int64_t sweeps, int group_sweeps, void* cuda_stream) {
    if (!b || sweeps < 0) { set_error("isg_batch_run: bad argument"); return ISG_ERR_ARG; }
    if (group_sweeps <= 0) group_sweeps = 64;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t full = sweeps / group_sweeps;
    const int rem = (int)(sweeps % group_sweeps);
    cudaError_t e = cudaSuccess;
    if (full > 0 && (!b->exec || b->graph_group != group_sweeps)) {
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t le = batch_launch(b, group_sweeps, b->cap);
            e = cudaStreamEndCapture(b->cap, &b->graph);
            if (e == cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) return cuda_fail(e, "isg_batch_run: graph capture");
        b->graph_group = group_sweeps;
    }
    for (int64_t g = 0; g < full && e == cudaSuccess; ++g) e = cudaGraphLaunch(b->exec, s);
    if (e == cudaSuccess && rem > 0) e = batch_launch(b, rem, s);
    if (e != cudaSuccess) return cuda_fail(e, "isg_batch_run");
    for (isg_sim* h : b->reps) {
        h->sweeps += sweeps;
        h->last_stream = s;
    }
    return ISG_OK;
}

// ISG_ERR_TIMEOUT (once) if a launch gave up waiting for the previous part of a
// split bundle: that bundle's lattices then missed sweeps.
static int batch_check(isg_batch* b, cudaStream_t s) {
    unsigned err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, b->d_ctr + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "isg_batch: error check");
    if (err) {
        cudaMemsetAsync(b->d_ctr + 2, 0, sizeof(unsigned), s);
        set_error("isg_batch: a part of a split bundle gave up waiting for the previous part");
        return ISG_ERR_TIMEOUT;
    }
    return ISG_OK;
}

int isg_batch_measure(isg_batch* b, int64_t* E, int64_t* Q, void* cuda_stream) {
    if (!b) { set_error("isg_batch_measure: NULL batch"); return ISG_ERR_ARG; }
    if (const int rc = batch_check(b, (cudaStream_t)cuda_stream)) return rc;
    for (int r = 0; E && r < 2 * b->n; ++r) {
        const int rc = isg_energy(b->reps[r], &E[r], cuda_stream);
        if (rc) return rc;
    }
    for (int s = 0; Q && s < b->n; ++s) {
        const int rc = isg_overlap(b->reps[2 * s], b->reps[2 * s + 1], &Q[s], cuda_stream);
        if (rc) return rc;
    }
    return ISG_OK;
}

int isg_batch_tracked(isg_batch* b, int64_t* E, uint64_t* H, void* cuda_stream) {
    if (!b) { set_error("isg_batch_tracked: NULL batch"); return ISG_ERR_ARG; }
    if (const int rc = batch_check(b, (cudaStream_t)cuda_stream)) return rc;
    for (int r = 0; r < 2 * b->n; ++r) {
        if (E) {
            const int rc = isg_tracked_energy(b->reps[r], &E[r]);
            if (rc) return rc;
        }
        if (H) {
            const int rc = isg_hash(b->reps[r], &H[r], cuda_stream);
            if (rc) return rc;
        }
    }
    return ISG_OK;
}

}  // extern "C"
