// isg_bundles.cuh -- bundle planning and the persistent bundle kernel, shared by
// the batched engine (isg_batch.cu) and the request server (isg_serve.cu).
#pragma once

#include <vector>

#include "isg_common.cuh"

namespace isg {

// Pack the RNG streams of the lattices `reps` into bundles: a lattice with more
// than 32 streams is one bundle; smaller lattices are packed first-fit, at most
// 32 streams per bundle.  Bundles come out largest first.  entries holds
// (lattice index, stream) pairs, boff the bundle offsets (size bundles + 1);
// if order is given it receives the lattice indices of each bundle, each
// bundle's list terminated by -1.
void plan_bundles(const std::vector<isg_sim*>& reps, std::vector<int2>& entries, std::vector<int>& boff,
                  std::vector<int>* order);

// One-time attribute set-up of the bundle kernel (large dynamic shared memory).
cudaError_t prepare_bundle_kernel(int kind);

// Launch the persistent bundle kernel: one CTA per SM (at most one per bundle)
// sweeps bundle after bundle; bundle b runs bsweeps[b] sweeps (or `sweeps` for
// all when bsweeps is NULL).  ctr must hold two zeroed words; the kernel
// returns them to zero when it ends.
cudaError_t launch_bundle_kernel(int kind, const FlipArgs* reps, const int2* entries, const int* boff,
                                 const int* bsweeps, int nbundles, int sweeps, unsigned* ctr, cudaStream_t s);

}  // namespace isg
