// cn_force_noalloc: the plain FP32 force for callers that cannot allocate
// device memory. Some callers are not allowed to call cudaMalloc at all -
// for instance a host application whose own memory manager owns every
// device allocation, or a latency-bound loop that cannot afford the
// device-wide synchronisation cudaMalloc and cudaFree may imply. This entry
// point takes its scratch space (the partial sums of i-tiles split across
// CTAs, their arrival counters and the queue words) from a fixed-size
// array that is part of the library's device image, so it allocates
// nothing. The paper has no counterpart.
#include "cunbody.h"
#include "cn_guard.h"
#include "cn_kernels.h"

#include <nvtx3/nvToolsExt.h>

#include <map>
#include <mutex>
#include <string>

namespace cn {
cn_status force_f32_on_workspace(int64_t n_i, const float* pos_i, int64_t n_j, const float* pos_mass_j, float eps2,
                                 float* acc_out, float* pot_out, void* ws, size_t ws_bytes, cudaStream_t s);
cn_status set_error(cn_status st, const std::string& msg);
}  // namespace cn

namespace {

// The scratch: 32 MiB of device memory in the library image. Every GPU on
// which the library has been used holds it until the process exits,
// whether or not this entry point is ever called there.
constexpr size_t kStaticScratchBytes = static_cast<size_t>(32) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
std::map<int, void*> g_scratch_addr;  // device ordinal -> device address of g_static_scratch

// The address recorded for the current device by the device set-up below.
cn_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cn::set_error(CN_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_scratch_addr.find(dev);
  if (it == g_scratch_addr.end())
    return cn::set_error(CN_ERR_CUDA, "cn_force_noalloc: the static scratch of this device was not set up");
  *out = it->second;
  return CN_OK;
}

}  // namespace

namespace cn {
// Device set-up, run once per device by the library's first call there
// (any entry point), with that device current. Host code cannot use
// g_static_scratch directly: on the host that name is a stand-in, not a
// device address, so the address is looked up here. With CUDA's lazy
// module loading the lookup also loads this file's device module, which
// is when the 32 MiB array is allocated on the device - inside the
// library's first call on that device, never inside a cn_force_noalloc
// call made after it.
cudaError_t static_scratch_setup() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  if (p == nullptr) return cudaErrorInvalidSymbol;
  std::lock_guard<std::mutex> lock(g_mu);
  g_scratch_addr[dev] = p;
  return cudaSuccess;
}
}  // namespace cn

namespace {
cn_status noalloc_call(int64_t n_i, const float* pos_i, int64_t n_j, const float* pos_mass_j, float eps2,
                       float* acc_out, float* pot_out, cn_stream stream);
}  // namespace

extern "C" cn_status cn_force_noalloc(int64_t n_i, const float* pos_i, int64_t n_j, const float* pos_mass_j,
                                      float eps2, float* acc_out, float* pot_out, cn_stream stream) {
  nvtxRangePushA("cn_force_noalloc");
  const cn_status st =
      cn::guard([&]() -> cn_status { return noalloc_call(n_i, pos_i, n_j, pos_mass_j, eps2, acc_out, pot_out, stream); });
  nvtxRangePop();
  return st;
}

namespace {
cn_status noalloc_call(int64_t n_i, const float* pos_i, int64_t n_j, const float* pos_mass_j, float eps2,
                       float* acc_out, float* pot_out, cn_stream stream) {
  auto s = reinterpret_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  if (n_i > 0 && n_j > 0) {
    // Scratch this problem needs under its launch shape (this also sets the
    // device up on a first call); 0 means the arguments or the device are
    // invalid, which the call below reports.
    const size_t need = cn_workspace_bytes(pot_out ? CN_VARIANT_F32_POT : CN_VARIANT_F32, n_i, n_j);
    if (need > kStaticScratchBytes)
      return cn::set_error(CN_ERR_WORKSPACE,
                           "cn_force_noalloc: this problem needs " + std::to_string(need) +
                               " bytes of scratch but the static scratch holds " +
                               std::to_string(kStaticScratchBytes) +
                               " bytes (use cn_force or cn_force_ws, or a launch shape with fewer i-tiles)");
    if (need > 0) {
      // the force call below clears the scratch's control head (queue words
      // and arrival counters) on the stream before it launches
      cn_status st = scratch_address(&scratch);
      if (st != CN_OK) return st;
    }
  }
  return cn::force_f32_on_workspace(n_i, pos_i, n_j, pos_mass_j, eps2, acc_out, pot_out, scratch,
                                    scratch ? kStaticScratchBytes : 0, s);
}
}  // namespace
