// isg_bundles.cuh -- the multi-lattice engines of the batched engine
// (isg_batch.cu): bundle planning and the persistent bundle kernel, and the
// per-pass launches over (lattice, stream) items that the request server
// (isg_serve.cu) also uses.
#pragma once

#include <vector>

#include "isg_common.cuh"

namespace isg {

// Execution configuration of the persistent bundle kernel.  None of it changes
// a result: every lattice follows its own trajectory whatever the bundles.
//   shape     0: one CTA of 32 warps per SM, 1: one of 24, 2: one of 16,
//             3: two of 16; batches only, no bundles: kPassShape, every colour
//             pass of all lattices is one launch whose warps take (lattice,
//             stream) items by ticket; kGroupShape, one launch runs all passes
//             of a sweep group, items of pass p waiting (bounded) for their own
//             lattice's pass p - 1 only (capacity and resident do not apply)
//   capacity  streams per packed bundle of small lattices (1 .. warps of the shape)
//   resident  1: the generator state of a bundle that fits in the CTA stays in
//             shared memory / registers for the whole launch; 0: it is loaded
//             and stored around every colour pass
//   wpt       words of a row group each lane updates (1 or 2): a row group is
//             wpt * 32 words, so 2 halves the groups per pass
constexpr int kBundleShapeCount = 4;
constexpr int kPassShape = 4;
constexpr int kGroupShape = 5;
struct BundleConfig {
    int shape = 0;
    int capacity = 32;
    int resident = 1;
    int wpt = 1;
};

// Warps per CTA of the configuration's shape.
int bundle_warps(const BundleConfig& cfg);

// Pack the RNG streams of the lattices `reps` into bundles: a lattice with more
// than `capacity` streams is one bundle; smaller lattices are packed first-fit,
// at most `capacity` streams per bundle.  Bundles come out largest first.  entries holds
// (lattice index, stream) pairs, boff the bundle offsets (size bundles + 1);
// if order is given it receives the lattice indices of each bundle, each
// bundle's list terminated by -1.
void plan_bundles(const std::vector<isg_sim*>& reps, std::vector<int2>& entries, std::vector<int>& boff,
                  std::vector<int>* order, int capacity = 32);

// Launch order of the bundles (device arrays): task i is (bundle, part, dep,
// parts): part 0 = all of the launch's sweeps, else part p of `parts`
// consecutive shares of them, which waits for task dep (the same bundle's part
// p - 1; -1 for the first) to finish.
struct BundleTasks {
    int4* d_tasks = nullptr;
    unsigned* d_done = nullptr;  // one flag per task, zero between launches
    int ntasks = 0;
};

// One-time attribute set-up of the bundle kernel (large dynamic shared memory).
cudaError_t prepare_bundle_kernel(int kind, const BundleConfig& cfg);

// Launch the persistent bundle kernel: the shape's CTAs per SM (at most one per
// task) sweep task after task; bundle b runs bsweeps[b] sweeps (or `sweeps` for
// all when bsweeps is NULL), split as `tasks` says (NULL: one task per bundle,
// in bundle order).  ctr must hold three zeroed words; the kernel returns the
// first two, and the task flags, to zero when it ends; ctr[2] becomes 1 if a
// wait for a previous part gave up (the waiting part is then skipped).
cudaError_t launch_bundle_kernel(int kind, const BundleConfig& cfg, const FlipArgs* reps, const int2* entries,
                                 const int* boff, const int* bsweeps, int nbundles, int sweeps, unsigned* ctr,
                                 cudaStream_t s, const BundleTasks* tasks = nullptr);

// Per-pass launches of the pass engine over an item list (lattice, stream),
// longest streams first: 2 * sweeps launches, launch p sweeping colour p & 1 of
// the items whose lattice has limit[lattice] > p (limit NULL: every lattice
// runs all passes).  ctr must hold two zeroed words; each launch returns them
// to zero when it ends.
cudaError_t launch_pass_items(int kind, const FlipArgs* reps, const int2* items, int nitems, const int* limit,
                              int sweeps, unsigned* ctr, cudaStream_t s);

}  // namespace isg
