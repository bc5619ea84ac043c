// Compensated pair-kernel instantiations, single system: K = 1 (the
// guarded kernel) in scalar form, K = 2 and 4 packed (f32x2), with
// bitwise the same results.
#include "cn_pair.cuh"

namespace cn {
namespace {

template <int K, bool POT, bool GUARD>
const void* fn() {
  if constexpr (K >= 2)
    return reinterpret_cast<const void*>(&pair_kernel<DDx2Policy<K, POT, GUARD>, K, false>);
  else
    return reinterpret_cast<const void*>(&pair_kernel<DDPolicy<K, POT, GUARD>, K, false>);
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

const void* select(int k, bool pot, bool guard) {
  if (pot) return guard ? by_k<true, true>(k) : by_k<true, false>(k);
  return guard ? by_k<false, true>(k) : by_k<false, false>(k);
}

}  // namespace

cudaError_t occupancy_dd(const Plan& p, bool pot, bool guard, size_t smem, int* ctas) {
  const void* f = select(p.k, pot, guard);
  if (!f) return cudaErrorInvalidValue;
  cudaError_t e = prepare_kernel(f, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, f, p.threads, smem);
}

cudaError_t launch_dd(const PairArgs& a, const Plan& p, bool pot, bool guard, int grid, cudaStream_t s) {
  const void* f = select(p.k, pot, guard);
  if (!f) return cudaErrorInvalidValue;
  const size_t smem = ring_smem_bytes(p);
  cudaError_t e = prepare_kernel(f, smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<PairArgs*>(&a)};
  return launch_pdl(f, dim3(grid), dim3(p.threads), args, smem, s);
}

}  // namespace cn
