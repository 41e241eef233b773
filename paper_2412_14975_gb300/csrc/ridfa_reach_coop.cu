// Reach-kernel instantiations of one text path (kPathCoop): every table layout and interface
// register count it supports.
#include "ridfa_reach.cuh"

namespace ridfa {
cudaError_t reach_path_coop(const ReachArgs &a, const ReachPlan &pl, cudaStream_t st, int *per_sm) {
    return reach_m<kPathCoop>(a, pl, st, per_sm);
}
}  // namespace ridfa
