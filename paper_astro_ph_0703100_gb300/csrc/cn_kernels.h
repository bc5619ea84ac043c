// Launch-side structures shared by the host dispatcher and the kernels.
// Not part of the public C ABI (that is include/cunbody.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cstdlib>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

namespace cn {

// One (system, i-tile) of the work: the batched schedule keeps a table of
// these in device memory; the single-system schedule derives them from the
// tile index.
struct TileDesc {
  int64_t i0;     // first i index of the tile (into pos_i and the outputs)
  int64_t j0;     // first j index of the tile's system (into pos_j; gathering plans: into j_index)
  int64_t nj;     // number of j-particles of the system
  int64_t unit0;  // first unit of the tile in the global unit sequence
  int32_t ni;     // valid i-particles in the tile (<= i_tile)
  int32_t njt;    // j-tiles of the system: ceil(nj / j_tile)
  float eps2;     // softening of the system
  int32_t pad;
};

// Everything one launch of the pair kernel needs. A "unit" is one i-tile
// (threads x i-per-thread particles) against one j-tile (j_tile records).
// Units are numbered tile-major; a "chunk" is a contiguous unit range
// processed by one CTA (static: chunk q = CTA q, dynamic: popped from a
// queue). Tiles split over several chunks are merged by the last chunk
// to finish, in chunk order, in FP64.
struct PairArgs {
  const float4* pos_i;
  const float4* pos_j;
  const float4* pos_i2;   // second i record (adjoint: loss weights), else unused
  const float4* pos_j2;   // second j record (adjoint: loss weights), else unused
  void* acc_out;          // float[n_i][3] (FP32 forms), double[n_i][3] (compensated), dL/dx (adjoint)
  void* pot_out;          // float[n_i] / double[n_i] / dL/dm (adjoint) or nullptr
  void* jerk_out;         // float[n_i][3] (force-jerk-potential form) or nullptr
  float4* partials;       // [n_chunks][2][i_tile] float4 (x2 for hi/lo in the compensated form)
  unsigned int* counters;  // [n_tiles] arrival counters (zero at launch; the merging CTA re-zeroes its own)
  int* queue;             // [0] next chunk, [1] finished CTAs (dynamic schedule; zero between launches)
  int* status;            // device status word
  const TileDesc* tiles;  // batched schedule only
  const int32_t* j_index;  // gathering list plans: list entries, each the index of a pos_j record
  int64_t n_index;         // gathering list plans: entries in j_index
  int64_t n_i;            // single system: i count
  int64_t n_j;            // single system: j count
  int64_t total_units;
  int64_t chunk_units;    // 0: static schedule (gridDim.x chunks); > 0: dynamic chunks of this size
  int64_t n_chunks;
  int32_t n_tiles;
  int32_t njt;            // single system: ceil(n_j / j_tile)
  int32_t j_tile;
  int32_t stages;
  float eps2;             // single system
  int32_t j_lanes;        // lanes sharing one i-particle (split-j FP32 kernels; 1 otherwise)
  uint64_t wait_ns;       // bound on every barrier wait
};

// Tuning knobs of one launch (mirrors cn_tune of the public header).
struct Plan {
  int k = 4;              // i-particles per thread
  int threads = 128;      // threads per CTA (64, 128 or 256)
  int j_tile = 512;       // j records per shared-memory stage (multiple of 16)
  int stages = 4;         // ring depth
  int ctas_per_sm = 0;    // 0: occupancy maximum
  int64_t chunk_units = 0;  // 0: static schedule
  int j_lanes = 1;          // lanes sharing one i-particle (split-j kernels, k = 1)
  int i_tile() const { return k * threads / j_lanes; }
};

enum Variant : int {
  kF32 = 0,
  kF32Pot = 1,
  kDD = 2,
  kDDPot = 3,
  kAdjoint = 4,
  kBatched = 5,
  kBatchedPot = 6,
  kJerk = 7,
  kJerkPot = 8,
  kSym = 9,  // symmetric form (cn_sym.h)
  kF32EpsI = 10,     // softening per i-particle (the i record's 4th slot)
  kF32EpsIPot = 11,
};

// Kernel selection, occupancy and launch (defined in the per-variant
// translation units).
cudaError_t launch_f32(const PairArgs& a, const Plan& p, bool pot, bool guard, bool batched, int grid,
                       cudaStream_t s, bool eps_i = false);
cudaError_t occupancy_f32(const Plan& p, bool pot, bool guard, bool batched, size_t smem, int* ctas,
                          bool eps_i = false);
// list plans whose j records are gathered through an index array
cudaError_t launch_f32_gather(const PairArgs& a, const Plan& p, bool pot, bool guard, int grid, cudaStream_t s);
cudaError_t occupancy_f32_gather(const Plan& p, bool pot, bool guard, size_t smem, int* ctas);
cudaError_t launch_dd(const PairArgs& a, const Plan& p, bool pot, bool guard, int grid, cudaStream_t s);
cudaError_t occupancy_dd(const Plan& p, bool pot, bool guard, size_t smem, int* ctas);
cudaError_t launch_adjoint(const PairArgs& a, const Plan& p, bool guard, int grid, cudaStream_t s);
cudaError_t occupancy_adjoint(const Plan& p, bool guard, size_t smem, int* ctas);
cudaError_t launch_pack_w(const float* w, float4* wrec, int64_t n, cudaStream_t s);
cudaError_t launch_jerk(const PairArgs& a, const Plan& p, bool pot, bool guard, int grid, cudaStream_t s);
cudaError_t occupancy_jerk(const Plan& p, bool pot, bool guard, size_t smem, int* ctas);
cudaError_t launch_energy(int64_t n, const float4* pos_mass, const float* pot_f, const double* pot_d,
                          double* partials, int* counter, double* w_out, cudaStream_t s);

// Launches a kernel with programmatic stream serialization allowed
// (programmatic dependent launch): the GPU may schedule it while the
// previous kernel of the stream is still running, which removes most of the
// gap between back-to-back launches. Every kernel launched this way calls
// grid_dependency_wait() before its first global memory access, so stream
// order still holds for the data. CN_PDL=0 in the environment (read once)
// launches in plain stream order instead.
inline bool pdl_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("CN_PDL");
    return !(v && v[0] == '0');
  }();
  return on;
}

inline cudaError_t launch_pdl(const void* fn, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t s) {
  if (!pdl_enabled()) return cudaLaunchKernel(fn, grid, block, args, smem, s);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

// Raises a kernel's dynamic shared-memory limit once per (device, kernel).
inline cudaError_t prepare_kernel(const void* fn, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> raised;
  // this thread's last (device, kernel, limit): repeated launches skip the lock
  thread_local int last_dev = -1;
  thread_local const void* last_fn = nullptr;
  thread_local size_t last_smem = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev == last_dev && fn == last_fn && smem <= last_smem) return cudaSuccess;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = raised[{dev, fn}];
  if (smem > cur) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    cur = smem;
  }
  last_dev = dev;
  last_fn = fn;
  last_smem = cur;
  return cudaSuccess;
}

inline size_t ring_smem_bytes(const Plan& p) {
  return 256 + static_cast<size_t>(p.stages) * p.j_tile * 16;
}
// the gathering list kernel adds two buffers of j_tile list indices
inline size_t gather_smem_bytes(const Plan& p) { return ring_smem_bytes(p) + static_cast<size_t>(p.j_tile) * 8; }
inline size_t adjoint_smem_bytes(const Plan& p) {
  return 256 + static_cast<size_t>(p.stages) * p.j_tile * 32;
}

}  // namespace cn
