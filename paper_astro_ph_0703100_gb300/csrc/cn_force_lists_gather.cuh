// Gathering interaction-list kernels: pair_kernel with GATHER = true, for
// list plans whose j records are addressed through an index array (each
// list entry the index of a record of the source array, as a tree code
// hands over particles and tree nodes). The same policies and tile shapes
// as the contiguous list kernels; only the staging of a j-tile differs.
// Included by the two translation units that instantiate them without and
// with the potential, so that the two halves compile in parallel.
#pragma once

#include "cn_pair.cuh"

namespace cn {
namespace gather {

template <int K, bool POT, bool GUARD, bool SPLITJ>
const void* fn() {
  if constexpr (K >= 2)
    return reinterpret_cast<const void*>(&pair_kernel<F32x2Policy<K, POT, GUARD, SPLITJ, false>, K, true, true>);
  else
    return reinterpret_cast<const void*>(&pair_kernel<F32Policy<K, POT, GUARD, SPLITJ, false>, K, true, true>);
}

// k i-particles per thread (per lane group with j_lanes > 1); the guarded
// kernel (a group with eps2 = 0) holds one particle per thread, no split-j
template <bool POT>
const void* select(int k, bool guard, int j_lanes) {
  if (guard) return (k == 1 && j_lanes <= 1) ? fn<1, POT, true, false>() : nullptr;
  if (j_lanes > 1) {
    switch (k) {
      case 2: return fn<2, POT, false, true>();
      case 4: return fn<4, POT, false, true>();
      case 8: return fn<8, POT, false, true>();
      default: return nullptr;
    }
  }
  switch (k) {
    case 1: return fn<1, POT, false, false>();
    case 2: return fn<2, POT, false, false>();
    case 4: return fn<4, POT, false, false>();
    case 8: return fn<8, POT, false, false>();
    default: return nullptr;
  }
}

}  // namespace gather
}  // namespace cn
