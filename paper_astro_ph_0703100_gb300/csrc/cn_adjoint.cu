// Adjoint pair-kernel instantiations and the weight-packing pre-pass.
#include "cn_pair.cuh"

namespace cn {
namespace {

// K >= 2 runs the packed (f32x2) policy: the same results, fewer issued
// instructions per pair.
template <int K, bool GUARD, bool SPLITJ = false>
const void* fn() {
  if constexpr (K >= 2)
    return reinterpret_cast<const void*>(&pair_kernel<AdjointX2Policy<K, GUARD, SPLITJ>, K, false>);
  else
    return reinterpret_cast<const void*>(&pair_kernel<AdjointPolicy<K, GUARD>, K, false>);
}

// j_lanes > 1 (small systems): the packed form with two i-particles per lane group
const void* select(int k, bool guard, int j_lanes) {
  if (j_lanes > 1) return (k == 2 && !guard) ? fn<2, false, true>() : nullptr;
  if (guard) return k == 1 ? fn<1, true>() : nullptr;
  switch (k) {
    case 1: return fn<1, false>();
    case 2: return fn<2, false>();
    case 4: return fn<4, false>();
    default: return nullptr;
  }
}

// w is float[n][3] with 4-byte alignment; pack it into 16-byte records so the
// j-tiles of the weights can be staged by bulk copies like the positions.
__global__ void pack_w_kernel(const float* __restrict__ w, float4* __restrict__ wrec, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    wrec[i] = make_float4(w[3 * i + 0], w[3 * i + 1], w[3 * i + 2], 0.f);
  }
}

}  // namespace

cudaError_t occupancy_adjoint(const Plan& p, bool guard, size_t smem, int* ctas) {
  const void* f = select(p.k, guard, p.j_lanes);
  if (!f) return cudaErrorInvalidValue;
  cudaError_t e = prepare_kernel(f, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, f, p.threads, smem);
}

cudaError_t launch_adjoint(const PairArgs& a, const Plan& p, bool guard, int grid, cudaStream_t s) {
  const void* f = select(p.k, guard, p.j_lanes);
  if (!f) return cudaErrorInvalidValue;
  const size_t smem = adjoint_smem_bytes(p);
  cudaError_t e = prepare_kernel(f, smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<PairArgs*>(&a)};
  return launch_pdl(f, dim3(grid), dim3(p.threads), args, smem, s);
}

cudaError_t launch_pack_w(const float* w, float4* wrec, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  pack_w_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(w, wrec, n);
  return cudaGetLastError();
}

}  // namespace cn
