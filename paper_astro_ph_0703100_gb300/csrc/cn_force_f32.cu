// FP32 pair-kernel instantiations (single system and batched ensemble).
#include "cn_pair.cuh"

namespace cn {

// split-j kernels with K = 4 or 8 (and the batched K = 2 form): cn_force_f32_splitj.cu
const void* select_f32_splitj_wide(int k, bool pot, bool batched);

namespace {

// K >= 2 runs the packed (f32x2) policy: the same results, fewer issued
// instructions per pair.
template <int K, bool POT, bool GUARD, bool BATCHED, bool SPLITJ = false, bool EPSI = false>
const void* fn() {
  if constexpr (K >= 2)
    return reinterpret_cast<const void*>(&pair_kernel<F32x2Policy<K, POT, GUARD, SPLITJ, EPSI>, K, BATCHED>);
  else
    return reinterpret_cast<const void*>(&pair_kernel<F32Policy<K, POT, GUARD, SPLITJ, EPSI>, K, BATCHED>);
}

// Softening per i-particle (the i record's 4th slot): always guarded, since
// any particle's eps2 may be 0; single systems, split-j up to two particles.
template <bool POT>
const void* epsi(int k, int j_lanes) {
  if (j_lanes > 1) {
    if (k == 1) return fn<1, POT, true, false, true, true>();
    if (k == 2) return fn<2, POT, true, false, true, true>();
    return nullptr;
  }
  switch (k) {
    case 1: return fn<1, POT, true, false, false, true>();
    case 2: return fn<2, POT, true, false, false, true>();
    case 4: return fn<4, POT, true, false, false, true>();
    case 8: return fn<8, POT, true, false, false, true>();
    default: return nullptr;
  }
}

template <bool POT, bool GUARD, bool BATCHED>
const void* by_k(int k) {
  if constexpr (GUARD) {
    return k == 1 ? fn<1, POT, true, BATCHED>() : nullptr;
  } else {
    switch (k) {
      case 1: return fn<1, POT, false, BATCHED>();
      case 2: return fn<2, POT, false, BATCHED>();
      case 4: return fn<4, POT, false, BATCHED>();
      case 8: return fn<8, POT, false, BATCHED>();
      default: return nullptr;
    }
  }
}

const void* select(int k, bool pot, bool guard, bool batched, int j_lanes, bool eps_i) {
  if (eps_i) return batched ? nullptr : (pot ? epsi<true>(k, j_lanes) : epsi<false>(k, j_lanes));
  if (j_lanes > 1) {  // split-j kernels: 1, 2, 4 or 8 i-particles per j-lane group
    if (k > 1 && guard) return nullptr;
    if (batched || k > 2) return k == 1 ? nullptr : select_f32_splitj_wide(k, pot, batched);
    if (k == 2) return pot ? fn<2, true, false, false, true>() : fn<2, false, false, false, true>();
    if (pot) return guard ? fn<1, true, true, false, true>() : fn<1, true, false, false, true>();
    return guard ? fn<1, false, true, false, true>() : fn<1, false, false, false, true>();
  }
  if (batched) {
    if (pot) return guard ? by_k<true, true, true>(k) : by_k<true, false, true>(k);
    return guard ? by_k<false, true, true>(k) : by_k<false, false, true>(k);
  }
  if (pot) return guard ? by_k<true, true, false>(k) : by_k<true, false, false>(k);
  return guard ? by_k<false, true, false>(k) : by_k<false, false, false>(k);
}

}  // namespace

cudaError_t occupancy_f32(const Plan& p, bool pot, bool guard, bool batched, size_t smem, int* ctas, bool eps_i) {
  const void* f = select(p.k, pot, guard, batched, p.j_lanes, eps_i);
  if (!f) return cudaErrorInvalidValue;
  cudaError_t e = prepare_kernel(f, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, f, p.threads, smem);
}

cudaError_t launch_f32(const PairArgs& a, const Plan& p, bool pot, bool guard, bool batched, int grid,
                       cudaStream_t s, bool eps_i) {
  const void* f = select(p.k, pot, guard, batched, p.j_lanes, eps_i);
  if (!f) return cudaErrorInvalidValue;
  const size_t smem = ring_smem_bytes(p);
  cudaError_t e = prepare_kernel(f, smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<PairArgs*>(&a)};
  return launch_pdl(f, dim3(grid), dim3(p.threads), args, smem, s);
}

}  // namespace cn
