// Gathering interaction-list kernels without the potential, plus the
// selection, occupancy and launch entry points of both halves.
#include "cn_force_lists_gather.cuh"

namespace cn {

const void* select_gather_pot(int k, bool guard, int j_lanes);  // cn_force_lists_gather_pot.cu

namespace {
const void* select_any(int k, bool pot, bool guard, int j_lanes) {
  return pot ? select_gather_pot(k, guard, j_lanes) : gather::select<false>(k, guard, j_lanes);
}
}  // namespace

cudaError_t occupancy_f32_gather(const Plan& p, bool pot, bool guard, size_t smem, int* ctas) {
  const void* f = select_any(p.k, pot, guard, p.j_lanes);
  if (!f) return cudaErrorInvalidValue;
  cudaError_t e = prepare_kernel(f, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, f, p.threads, smem);
}

cudaError_t launch_f32_gather(const PairArgs& a, const Plan& p, bool pot, bool guard, int grid, cudaStream_t s) {
  const void* f = select_any(p.k, pot, guard, p.j_lanes);
  if (!f) return cudaErrorInvalidValue;
  const size_t smem = gather_smem_bytes(p);
  cudaError_t e = prepare_kernel(f, smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<PairArgs*>(&a)};
  return launch_pdl(f, dim3(grid), dim3(p.threads), args, smem, s);
}

}  // namespace cn
