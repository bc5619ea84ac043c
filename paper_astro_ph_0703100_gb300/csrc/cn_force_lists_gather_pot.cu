// Gathering interaction-list kernels with the potential.
#include "cn_force_lists_gather.cuh"

namespace cn {

const void* select_gather_pot(int k, bool guard, int j_lanes) { return gather::select<true>(k, guard, j_lanes); }

}  // namespace cn
