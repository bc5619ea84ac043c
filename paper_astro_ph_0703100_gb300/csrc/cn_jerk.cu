// Force-jerk-potential pair-kernel instantiations (single system).
#include "cn_pair.cuh"

namespace cn {
namespace {

// K >= 2 runs the packed (f32x2) policy: the same results, fewer issued
// instructions per pair.
template <int K, bool POT, bool GUARD, bool SPLITJ = false>
const void* fn() {
  if constexpr (K >= 2)
    return reinterpret_cast<const void*>(&pair_kernel<JerkX2Policy<K, POT, GUARD, SPLITJ>, K, false>);
  else
    return reinterpret_cast<const void*>(&pair_kernel<JerkPolicy<K, POT, GUARD>, K, false>);
}

template <bool POT, bool GUARD>
const void* by_k(int k) {
  if constexpr (GUARD) {
    return k == 1 ? fn<1, POT, true>() : nullptr;
  } else {
    switch (k) {
      case 1: return fn<1, POT, false>();
      case 2: return fn<2, POT, false>();
      case 4: return fn<4, POT, false>();
      default: return nullptr;
    }
  }
}

// j_lanes > 1 (small systems): the packed form with two i-particles per lane group
const void* select(int k, bool pot, bool guard, int j_lanes) {
  if (j_lanes > 1) {
    if (k != 2 || guard) return nullptr;
    return pot ? fn<2, true, false, true>() : fn<2, false, false, true>();
  }
  if (pot) return guard ? by_k<true, true>(k) : by_k<true, false>(k);
  return guard ? by_k<false, true>(k) : by_k<false, false>(k);
}

}  // namespace

cudaError_t occupancy_jerk(const Plan& p, bool pot, bool guard, size_t smem, int* ctas) {
  const void* f = select(p.k, pot, guard, p.j_lanes);
  if (!f) return cudaErrorInvalidValue;
  cudaError_t e = prepare_kernel(f, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, f, p.threads, smem);
}

cudaError_t launch_jerk(const PairArgs& a, const Plan& p, bool pot, bool guard, int grid, cudaStream_t s) {
  const void* f = select(p.k, pot, guard, p.j_lanes);
  if (!f) return cudaErrorInvalidValue;
  const size_t smem = adjoint_smem_bytes(p);  // two 16-byte records per j
  cudaError_t e = prepare_kernel(f, smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<PairArgs*>(&a)};
  return launch_pdl(f, dim3(grid), dim3(p.threads), args, smem, s);
}

}  // namespace cn
