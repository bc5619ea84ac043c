// Host side of the libcunbody C ABI (include/cunbody.h): argument checks,
// launch-shape selection, workspaces, dispatch to the kernels, batched
// plans, host-memory forms, tuning and status.
#include "cunbody.h"
#include "cn_guard.h"
#include "cn_kernels.h"
#include "cn_sym.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

namespace cn {
cudaError_t device_status_address(int** p);
cudaError_t static_scratch_setup();
cudaError_t launch_timeout_probe(int* status, uint64_t wait_ns, cudaStream_t s);
cudaError_t run_probes(cudaStream_t s, double* out);
size_t energy_workspace_doubles();
}  // namespace cn

using cn::Plan;
using cn::PairArgs;

struct cn_batch_plan {
  int dev = -1;
  bool lists = false;       // interaction-list plan: separate i and j arrays
  bool zero_first = false;  // some group has i-particles but an empty list: clear outputs first
  int32_t n_clusters = 0;
  int64_t n_total = 0;      // i-particles (cluster plans: also the j records)
  int64_t n_j_total = 0;    // j records a list plan reads (max of begin + count)
  double pairs = 0.0;
  Plan plan;
  bool guard = false;
  bool pot = false;
  cn::TileDesc* d_tiles = nullptr;
  int32_t* d_index = nullptr;  // gathering list plans: the list entries (indices into the source records)
  int64_t n_index = 0;
  int32_t n_tiles = 0;
  int64_t units = 0;
  int64_t n_chunks = 0;
  int grid = 0;
  size_t ws_bytes = 0;
  size_t ctrl_bytes = 0;
  size_t data_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

constexpr size_t kCtrlBytes = 4096;  // queue words and spare control space at the head of a workspace
constexpr uint64_t kDefaultWaitNs = 2000000000ull;
constexpr size_t kMaxSmem = 227 * 1024;
constexpr int32_t kNoIndex = 0;  // stands for the index array of a gathering plan whose lists are all empty
constexpr size_t kSymSlotCap = static_cast<size_t>(2) << 30;  // symmetric-form slot memory before banding

thread_local std::string g_last_error;
std::atomic<uint64_t> g_wait_ns{kDefaultWaitNs};

cn_status fail(cn_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

cn_status fail_cuda(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return CN_ERR_CUDA;
}

// An NVTX range around each entry point (visible to Nsight tools; a few
// nanoseconds when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// CN_LOG=1 (read once, at the first call) prints each launch plan to stderr.
bool log_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("CN_LOG");
    return v && *v && std::strcmp(v, "0") != 0;
  }();
  return on;
}

const char* variant_name(int v) {
  static const char* names[] = {"f32", "f32_pot", "dd", "dd_pot", "adjoint", "batched", "batched_pot",
                                "jerk", "jerk_pot", "symmetric", "f32_eps_i", "f32_eps_i_pot"};
  return (v >= 0 && v < 12) ? names[v] : "?";
}

// Host-side fault injection for tests: CN_FAULT_INJECT holds a comma list of
// "alloc", "launch", "capture"; the matching step then fails as if the CUDA
// call had failed. Nothing is done on the device.
bool inject(const char* point) {
  const char* v = std::getenv("CN_FAULT_INJECT");
  return v && std::strstr(v, point) != nullptr;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  if (!a || !b || na == 0 || nb == 0) return false;
  const auto pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
  return pa < pb + nb && pb < pa + na;
}

// ------------------------------------------------------------------ devices
struct DeviceInfo {
  int sms = 0;
  int major = 0;
  int minor = 0;
  int* status = nullptr;
  bool supported = false;
};

std::mutex g_mu;  // guards the maps below and the creation of device entries

// Device entries, created once per device ordinal by the first call there
// (under g_mu) and never freed; read without a lock afterwards.
constexpr int kMaxDevices = 64;
std::atomic<DeviceInfo*> g_dev_table[kMaxDevices];

// Bumped whenever something a cached launch plan depends on changes: a
// tuning entry, or the address of a library workspace. Calls compare it
// with the generation their per-thread plan cache was filled under.
std::atomic<uint64_t> g_plan_gen{1};
thread_local uint64_t t_own_bumps = 0;  // generation bumps made by this thread's own workspace growth

// The launch plan of this thread's last single-system call, reused while the
// call's key and the generation match (the common loop of identical calls
// then skips the tuning, occupancy and workspace lookups).
struct PlanCache {
  bool valid = false;
  uint64_t gen = 0;
  int dev = -1;
  int variant = -1;
  int64_t n_i = -1, n_j = -1;
  bool guard = false;
  cudaStream_t stream = nullptr;
};

DeviceInfo* device_entry(int dev) {
  return (dev >= 0 && dev < kMaxDevices) ? g_dev_table[dev].load(std::memory_order_acquire) : nullptr;
}

cn_status current_device(int* dev_out, DeviceInfo** info) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(CN_ERR_UNSUPPORTED_DEVICE, "device ordinal out of range");
  DeviceInfo* d = device_entry(dev);
  if (!d) {
    std::lock_guard<std::mutex> lock(g_mu);
    d = g_dev_table[dev].load(std::memory_order_acquire);
    if (!d) {
      DeviceInfo nd;
      if ((e = cudaDeviceGetAttribute(&nd.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
          (e = cudaDeviceGetAttribute(&nd.major, cudaDevAttrComputeCapabilityMajor, dev)) != cudaSuccess ||
          (e = cudaDeviceGetAttribute(&nd.minor, cudaDevAttrComputeCapabilityMinor, dev)) != cudaSuccess)
        return fail_cuda(e, "cudaDeviceGetAttribute");
      nd.supported = (nd.major == 10 && nd.minor == 3);
      if (nd.supported && (e = cn::device_status_address(&nd.status)) != cudaSuccess)
        return fail_cuda(e, "cudaGetSymbolAddress(device status)");
      // the static scratch of cn_force_noalloc: its address, and its device
      // module loaded, on the library's first call on this device
      if (nd.supported && (e = cn::static_scratch_setup()) != cudaSuccess)
        return fail_cuda(e, "cudaGetSymbolAddress(static scratch)");
      d = new DeviceInfo(nd);
      g_dev_table[dev].store(d, std::memory_order_release);
    }
  }
  if (!d->supported)
    return fail(CN_ERR_UNSUPPORTED_DEVICE, "libcunbody is built for sm_103a (GB300); device " + std::to_string(dev) +
                                               " is sm_" + std::to_string(d->major) + std::to_string(d->minor));
  if (dev_out) *dev_out = dev;
  *info = d;
  return CN_OK;
}

// ------------------------------------------------------------------ library workspaces
// Per (device, stream): `ctrl` holds the queue words and the split-tile
// arrival counters (zeroed when allocated, left zero by every kernel); `data`
// holds partial sums and packed weights (no initialisation needed).
struct LibWorkspace {
  void* ctrl = nullptr;
  size_t ctrl_bytes = 0;
  void* data = nullptr;
  size_t data_bytes = 0;
  double* aux = nullptr;  // potential-energy block sums + counter
};
std::map<std::pair<int, cudaStream_t>, LibWorkspace> g_ws;

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

cn_status grow(cudaStream_t s, void** buf, size_t* bytes, size_t need, bool zero, const char* what) {
  if (*buf && *bytes >= need) return CN_OK;
  if (inject("capture") || capturing(s))
    return fail(CN_ERR_WORKSPACE,
                "the library workspace of this stream must grow, which allocates; not allowed during graph "
                "capture (make one call before capturing, or pass a workspace)");
  if (inject("alloc")) return fail(CN_ERR_CUDA, "cudaMalloc: injected allocation failure");
  cudaError_t e;
  if (*buf) {
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail_cuda(e, "cudaStreamSynchronize");
    cudaFree(*buf);
    *buf = nullptr;
    *bytes = 0;
  }
  const size_t nb = align_up(std::max(need, static_cast<size_t>(1) << 16), static_cast<size_t>(1) << 16);
  void* p = nullptr;
  if ((e = cudaMalloc(&p, nb)) != cudaSuccess) return fail_cuda(e, what);
  if (zero && (e = cudaMemsetAsync(p, 0, nb, s)) != cudaSuccess) {
    cudaFree(p);
    return fail_cuda(e, "cudaMemsetAsync(workspace)");
  }
  *buf = p;
  *bytes = nb;
  g_plan_gen.fetch_add(1, std::memory_order_acq_rel);  // cached plans held the old address
  ++t_own_bumps;
  return CN_OK;
}

cn_status library_workspace(cudaStream_t s, size_t ctrl_need, size_t data_need, char** ctrl, char** data) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(g_mu);
  LibWorkspace& w = g_ws[{dev, s}];
  cn_status st = grow(s, &w.ctrl, &w.ctrl_bytes, ctrl_need, true, "cudaMalloc(workspace control)");
  if (st != CN_OK) return st;
  if ((st = grow(s, &w.data, &w.data_bytes, std::max<size_t>(data_need, 256), false, "cudaMalloc(workspace)")) != CN_OK)
    return st;
  *ctrl = static_cast<char*>(w.ctrl);
  *data = static_cast<char*>(w.data);
  return CN_OK;
}

// Bytes of the data region the library already holds for stream s.
size_t library_data_bytes(cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_ws.find({dev, s});
  return it == g_ws.end() ? 0 : it->second.data_bytes;
}

// Frees the library workspace of a stream that is about to be destroyed.
void release_library_workspace(cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_ws.find({dev, s});
  if (it == g_ws.end()) return;
  if (it->second.ctrl) cudaFree(it->second.ctrl);
  if (it->second.data) cudaFree(it->second.data);
  if (it->second.aux) cudaFree(it->second.aux);
  g_ws.erase(it);
  g_plan_gen.fetch_add(1, std::memory_order_acq_rel);
}

cn_status library_aux(cudaStream_t s, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(g_mu);
  LibWorkspace& w = g_ws[{dev, s}];
  if (!w.aux) {
    if (inject("capture") || capturing(s))
      return fail(CN_ERR_WORKSPACE, "first potential-energy call on a stream allocates; not allowed during capture");
    if (inject("alloc")) return fail(CN_ERR_CUDA, "cudaMalloc: injected allocation failure");
    const size_t nb = (cn::energy_workspace_doubles() + 1) * sizeof(double);
    if ((e = cudaMalloc(reinterpret_cast<void**>(&w.aux), nb)) != cudaSuccess) return fail_cuda(e, "cudaMalloc(aux)");
    if ((e = cudaMemsetAsync(w.aux, 0, nb, s)) != cudaSuccess) return fail_cuda(e, "cudaMemsetAsync(aux)");
  }
  *out = w.aux;
  return CN_OK;
}

// ------------------------------------------------------------------ tuning
std::map<std::tuple<int, int, int, int>, cn_tune> g_tune;

int bucket(int64_t n) {
  int b = 0;
  while (b < 62 && (static_cast<int64_t>(1) << b) < n) ++b;
  return b;
}

bool valid_k(int variant, int k) {
  if (variant == cn::kSym) return k == 1 || k == 2 || k == 4 || k == 8;
  if (variant == cn::kDD || variant == cn::kDDPot || variant == cn::kAdjoint || variant == cn::kJerk ||
      variant == cn::kJerkPot)
    return k == 1 || k == 2 || k == 4;
  return k == 1 || k == 2 || k == 4 || k == 8;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Launch shape of the symmetric form from a small model of its schedule.
// The N(N+1)/2-style triangle of T tile pairs (tile B = threads x K) is cut
// into equal static ranges over G = min(resident slots, units) CTAs; the SM
// holding the most CTAs sets the time, at a rate that saturates once about
// six warps share the SM. Saturated rates are the ones measured at
// N = 131072 (ordered pairs / s): they favour large K (fewer warp
// reductions per pair), while small systems need small tiles to fill the
// SMs.
cn_tune sym_default_tune(int64_t n, int sms, bool pot) {
  if (pot && n >= 28000) {
    // with the potential, measured from N = 32768 to 131072: K = 8 x 128 runs
    // 2-2.7% ahead of 4 x 256 (131072: 6.41 against 6.54 ms), which the
    // schedule model below does not see (it charges multi-CTA shapes for
    // their busiest CTA); at 24576 and below 4 x 256 stays ahead
    cn_tune t{};
    t.i_per_thread = 8;
    t.threads = 128;
    t.j_tile = 256;
    t.stages = 4;
    t.j_lanes = 1;
    return t;
  }
  struct Shape {
    int k, threads, j_tile, stages, slots_per_sm;
    double rate, rate_pot;  // saturated effective pairs/s without and with the potential
  };
  static const Shape shapes[] = {
      {8, 256, 256, 3, 1, 3.56e12, 0.0},     {4, 256, 256, 3, 1, 3.10e12, 2.59e12},
      // K = 8 x 128 without the potential: two resident CTAs run well below
      // the saturated rate (N = 24576: 280 us against 198 us for 4 x 256),
      // so the force-only form does not take it
      {8, 128, 256, 4, 3, 0.0, 2.38e12},     {8, 64, 128, 4, 8, 3.05e12, 2.38e12},
      {4, 128, 256, 4, 3, 2.87e12, 2.33e12}, {4, 64, 128, 4, 8, 2.64e12, 2.10e12},
      {2, 64, 64, 4, 8, 1.86e12, 1.50e12},   {1, 64, 64, 4, 9, 0.93e12, 0.75e12}};
  cn_tune best{};
  double best_t = 0.0;
  for (const Shape& sh : shapes) {
    // with the potential the rows of j-side sums take four floats per particle
    if (cn::sym_smem_bytes(sh.threads, sh.k, sh.j_tile, sh.stages, pot) > kMaxSmem) continue;
    if ((pot ? sh.rate_pot : sh.rate) <= 0.0) continue;
    const int64_t b = static_cast<int64_t>(sh.k) * sh.threads;
    const int64_t T = (std::max<int64_t>(n, 1) + b - 1) / b;
    const int64_t units = T * (T + 1) / 2;
    const int64_t g = std::min<int64_t>(static_cast<int64_t>(sh.slots_per_sm) * sms, units);
    const int64_t per_sm = (g + sms - 1) / sms;
    const int64_t per_cta = (units + g - 1) / g;
    const double warps = static_cast<double>(per_sm) * sh.threads / 32.0;
    const double sm_rate = (pot ? sh.rate_pot : sh.rate) / sms * std::min(1.0, warps / 6.0);
    const double t = static_cast<double>(per_sm * per_cta) * 2.0 * static_cast<double>(b * b) / sm_rate;
    if (best_t == 0.0 || t < best_t) {
      best_t = t;
      best.i_per_thread = sh.k;
      best.threads = sh.threads;
      best.j_tile = sh.j_tile;
      best.stages = sh.stages;
    }
  }
  best.j_lanes = 1;
  return best;
}

// The packed shapes of 256 threads with four or eight i-particles per lane
// (split-j or not) run one CTA per SM, and the static schedule gives each
// CTA ceil(units / CTAs) units of j_tile records (a ragged last j-tile is
// padded with zero masses, so every unit costs the same). For the shape's
// i-tile this picks the j-tile, a multiple of `step` in [lo, hi] and no
// longer than the j set, with the least work on the busiest CTA, counting
// `unit_cost` records of overhead per unit (64 for the 12-operation FP32
// pair, proportionally fewer for costlier pairs); ties take the smaller
// tile. Measured at N = 8192 .. 131072 (graph-replayed launches), it picked
// the fastest or a tile within 1% of it at each size of the sweeps
// (N = 14000: 0.44 -> 0.72 of the FP32 bound, 28000: 0.72 -> 0.80,
// 98304: 0.836 -> 0.852).
int32_t fit_j_tile(int64_t n_i, int64_t n_j, int64_t i_tile, int32_t lo, int32_t hi, int32_t step, int64_t ctas,
                   int32_t unit_cost = 64) {
  const int64_t n_it = (n_i + i_tile - 1) / i_tile;
  // the padding of a short tile is written by one thread
  const int64_t nj_up = (std::max<int64_t>(n_j, 1) + step - 1) / step * step;
  hi = static_cast<int32_t>(std::min<int64_t>(std::min(hi, 4096), nj_up)) / step * step;
  hi = std::max(hi, step);
  lo = std::min(hi, std::max(step, lo / step * step));
  int32_t best_t = hi;
  double best = -1.0;
  for (int32_t t = lo; t <= hi; t += step) {
    const int64_t units = n_it * ((std::max<int64_t>(n_j, 1) + t - 1) / t);
    const int64_t g = std::max<int64_t>(1, std::min(units, ctas));
    const double c = static_cast<double>((units + g - 1) / g) * static_cast<double>(t + unit_cost);
    if (best < 0.0 || c < best) {
      best = c;
      best_t = t;
    }
  }
  return best_t;
}

// Default launch shape of a variant for these sizes on a device with `sms`
// multiprocessors (queried, never assumed).
cn_tune default_tune(int variant, int64_t n_i, int64_t n_j, int sms) {
  cn_tune t{};
  const int64_t n = std::max(n_i, n_j);
  const bool dd = variant == cn::kDD || variant == cn::kDDPot;
  // the adjoint and the force-jerk form stream two 16-byte records per j
  const bool adj = variant == cn::kAdjoint || variant == cn::kJerk || variant == cn::kJerkPot;
  const bool f32 = variant == cn::kF32 || variant == cn::kF32Pot || variant == cn::kF32EpsI ||
                   variant == cn::kF32EpsIPot;
  t.stages = 4;
  t.threads = 128;
  t.j_lanes = 1;
  if (f32 && n_i <= 4096) {
    // small systems (measured at N = 1024 .. 4096, packed form): lane groups
    // of 32 (16 at N = 4096) share two i-particles and, where it fits, the
    // whole j set sits in one single-stage tile, so that each CTA covers
    // whole i-tiles and nothing is merged
    const int jl = n_i > 2048 ? 16 : 32;
    t.i_per_thread = 2;
    t.j_lanes = jl;
    t.threads = n_i <= 1024 ? 128 : 256;
    const int64_t unit = 8 * jl;
    t.j_tile = static_cast<int32_t>(std::min<int64_t>(round_up(std::max<int64_t>(n_j, 1), unit), 4096));
    t.stages = n_j <= t.j_tile ? 1 : 3;
    return t;
  }
  if (f32) {
    // Mid-size systems (measured on GB300, 152 SMs, N = 4200 .. 40000,
    // graph-replayed launches): split-j lane groups of 4 or 8 holding two,
    // four or eight i-particles keep the i-tiles small enough to fill the
    // SMs while each j record feeds several packed pair terms. Sizes are compared by the
    // work per SM, n_eff = sqrt(n_i n_j) sqrt(152 / sms), so another SM count
    // moves the bands.
    const double n_eff = std::sqrt(static_cast<double>(n_i) * static_cast<double>(std::max<int64_t>(n_j, 1))) *
                         std::sqrt(152.0 / std::max(sms, 1));
    struct Band {
      double upto;
      int k, threads, j_lanes, jt_lo, jt_hi;
    };
    // (K, threads, lane groups) per band and the window of the j-tile fit;
    // fractions of the FP32 bound measured with the fitted j-tile
    static const Band bands[] = {
        {6500.0, 2, 256, 4, 512, 4096},    // N = 4500: 0.397, 6000: 0.503, 6400: 0.552
        {8600.0, 4, 256, 8, 512, 4096},    // N = 7000: 0.516, 8000: 0.562, 8192: 0.557
        {40000.0, 8, 256, 8, 512, 4096},   // 9000: 0.60, 14000: 0.72, 16384: 0.74, 20000: 0.76,
                                           // 24576: 0.80, 32768: 0.82, 40000: 0.81
    };
    if (n_i > 4096 && n_eff <= bands[2].upto) {
      for (const Band& b : bands) {
        if (n_eff > b.upto) continue;
        // with the potential the K = 8 split-j kernel runs short of registers
        // (N = 16384: 0.561 of its 14-operation bound); K = 4 with lane groups
        // of 4 keeps the 256-particle i-tile (0.689; 24576: 0.731, 32768: 0.744)
        const bool pot_k8 = variant == cn::kF32Pot && b.k == 8;
        const int k = pot_k8 ? 4 : b.k;
        const int jl = pot_k8 ? 4 : b.j_lanes;
        t.i_per_thread = k;
        t.threads = b.threads;
        t.j_lanes = jl;
        t.j_tile = fit_j_tile(n_i, n_j, static_cast<int64_t>(k) * b.threads / jl, b.jt_lo, b.jt_hi, 8 * jl, sms);
        t.stages = n_j <= t.j_tile ? 1 : 3;
        return t;
      }
    }
  }
  if ((variant == cn::kJerk || variant == cn::kJerkPot || variant == cn::kAdjoint) && n_i <= 8192) {
    // small systems, measured at N = 1024 .. 8192 (force + jerk + potential,
    // and the adjoint, with the same optima): packed split-j, two
    // i-particles per lane group of 32 (16 at N = 8192, 8 at N = 4096), up
    // to 2048 two-record j entries per stage
    const int jl = n_i <= 2048 ? 32 : (n_i <= 4096 ? 8 : 16);
    t.i_per_thread = 2;
    t.j_lanes = jl;
    t.threads = n_i <= 1024 ? 128 : 256;
    t.j_tile = static_cast<int32_t>(std::min<int64_t>(round_up(std::max<int64_t>(n_j, 1), 8 * jl), 2048));
    t.stages = n_j <= t.j_tile ? 1 : 3;
    return t;
  }
  if ((variant == cn::kJerk || variant == cn::kJerkPot || variant == cn::kAdjoint) && n < 32768) {
    // mid-size systems, measured at N = 16384 and 24576 (force + jerk +
    // potential and the adjoint): packed split-j, two i-particles per lane
    // group of 4, 512 two-record j entries per stage (N = 16384: 0.715 and
    // 0.707 of their FP32 bounds, against 0.694 and 0.667 for K = 2 x 128
    // without lane groups)
    t.i_per_thread = 2;
    t.threads = 256;
    t.j_lanes = 4;
    t.j_tile = static_cast<int32_t>(std::min<int64_t>(round_up(std::max<int64_t>(n_j, 1), 32), 512));
    t.stages = n_j <= t.j_tile ? 1 : 3;
    return t;
  }
  if (variant == cn::kSym) return sym_default_tune(n, sms, false);
  if (variant == cn::kBatched || variant == cn::kBatchedPot) {
    t.i_per_thread = 4;
    t.j_tile = 256;
  } else if (f32 && n > 4096) {
    // packed FP32, measured at N = 49152 .. 131072 (smaller systems take the
    // bands above): K = 4 x 256 below ~96K, K = 8 x 256 above, with the
    // j-tile fitted to the schedule from 512 or 1024 records. With the
    // potential K = 4 stays ahead at large N too (131072: 0.793 of its
    // 14-operation bound against 0.778 for K = 8)
    const bool k4 = n < 98304 || variant == cn::kF32Pot;
    t.i_per_thread = k4 ? 4 : 8;
    t.threads = 256;
    const int32_t jt0 = k4 ? 512 : 1024;
    t.j_tile = fit_j_tile(n_i, n_j, static_cast<int64_t>(t.i_per_thread) * t.threads, jt0 / 2, 2 * jt0, 16, sms);
  } else if (dd && n >= 20000) {
    // compensated form, K = 4 x 256 (measured at N = 24576 .. 131072), the
    // j-tile fitted to the schedule within 256 .. 1024 records; its pair
    // costs 82 FP32 lane operations, so a unit's overhead is about 9
    // records (N = 32768: 256-record tiles, 0.801 of its bound against
    // 0.782 with 1024; 24576: 1024, 0.758)
    t.i_per_thread = 4;
    t.threads = 256;
    t.j_tile = fit_j_tile(n_i, n_j, 1024, 256, 1024, 16, sms, 9);
  } else if (dd && n >= 4096 && n < 12000) {
    // compensated form, small systems: one i-particle per thread keeps the
    // i-tiles small enough to fill the SMs (N = 8192: 0.595 of its bound
    // against 0.548 for K = 2 x 128; 4096: 0.418 against 0.397)
    t.i_per_thread = 1;
    t.j_tile = 256;
  } else if (n >= 32768) {
    // measured optima of the adjoint (N = 65536) and the force-jerk form
    // (N = 131072): K = 4 x 256 with j-tiles of 256 two-record j entries
    t.i_per_thread = adj ? 4 : 8;
    t.threads = 256;
    t.j_tile = adj ? 256 : 1024;
  } else if (n >= 4096) {
    // the compensated form between N = 12000 and 20000 (measured at 16384:
    // K = 2 x 128 threads x 256 records, 0.755 of its bound)
    t.i_per_thread = 2;
    t.j_tile = 256;
  } else {
    t.i_per_thread = adj ? 1 : 2;
    t.threads = 64;
    t.j_tile = 128;
  }
  return t;
}

cn_status check_tune(int variant, const cn_tune& t) {
  if (t.i_per_thread && !valid_k(variant, t.i_per_thread))
    return fail(CN_ERR_INVALID_ARG, "i_per_thread must be 1, 2, 4 or 8 (compensated and adjoint forms: 1, 2, 4)");
  if (t.threads && t.threads != 64 && t.threads != 128 && t.threads != 256)
    return fail(CN_ERR_INVALID_ARG, "threads must be 64, 128 or 256");
  if (t.j_tile && (t.j_tile < 16 || t.j_tile > 4096 || t.j_tile % 16))
    return fail(CN_ERR_INVALID_ARG, "j_tile must be a multiple of 16 in 16..4096");
  if (t.stages && (t.stages < 1 || t.stages > 8)) return fail(CN_ERR_INVALID_ARG, "stages must be 1..8");
  if (t.ctas_per_sm < 0 || t.chunk_units < 0) return fail(CN_ERR_INVALID_ARG, "negative tuning field");
  if (t.j_lanes < 0 || t.j_lanes > 32 || (t.j_lanes & (t.j_lanes - 1)))
    return fail(CN_ERR_INVALID_ARG, "j_lanes must be 0 or a power of two up to 32");
  if (t.j_lanes > 1) {
    const bool jerk = variant == cn::kJerk || variant == cn::kJerkPot || variant == cn::kAdjoint;
    const bool eps_i = variant == cn::kF32EpsI || variant == cn::kF32EpsIPot;
    const bool f32 = variant == cn::kF32 || variant == cn::kF32Pot || variant == cn::kBatched ||
                     variant == cn::kBatchedPot;
    if (!f32 && !eps_i && !jerk)
      return fail(CN_ERR_INVALID_ARG, "j_lanes > 1 is offered for the FP32 (single, batched, per-i softening), "
                                      "force-jerk and adjoint forms");
    if (eps_i && t.i_per_thread > 2)
      return fail(CN_ERR_INVALID_ARG, "the per-i-softening form takes j_lanes > 1 with i_per_thread = 1 or 2");
    if (jerk && t.i_per_thread != 2)
      return fail(CN_ERR_INVALID_ARG, "the force-jerk and adjoint forms take j_lanes > 1 with i_per_thread = 2");
    if (t.j_tile && t.j_tile % (8 * t.j_lanes))
      return fail(CN_ERR_INVALID_ARG, "with j_lanes > 1, j_tile must be a multiple of 8 x j_lanes");
  }
  return CN_OK;
}

bool two_records(int variant) {
  return variant == cn::kAdjoint || variant == cn::kJerk || variant == cn::kJerkPot;
}

bool registered_tune(int dev, int variant, int64_t n_i, int64_t n_j) {
  std::lock_guard<std::mutex> lock(g_mu);
  return g_tune.count({dev, variant, bucket(n_i), bucket(n_j)}) > 0;
}

cn_status resolve_plan(int dev, int variant, int64_t n_i, int64_t n_j, bool guard, const cn_tune* explicit_tune,
                       Plan* p) {
  int sms = 0;
  if (const DeviceInfo* d = device_entry(dev)) sms = d->sms;
  if (sms <= 0 && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(CN_ERR_CUDA, "cudaDeviceGetAttribute(multiprocessor count)");
  cn_tune t = default_tune(variant, n_i, n_j, sms);
  cn_tune chosen{};
  bool have = false;
  if (explicit_tune) {
    chosen = *explicit_tune;
    have = true;
  } else {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_tune.find({dev, variant, bucket(n_i), bucket(n_j)});
    if (it != g_tune.end()) {
      chosen = it->second;
      have = true;
    }
  }
  if (have) {
    cn_status st = check_tune(variant, chosen);
    if (st != CN_OK) return st;
    if (chosen.i_per_thread) t.i_per_thread = chosen.i_per_thread;
    if (chosen.threads) t.threads = chosen.threads;
    if (chosen.j_tile) t.j_tile = chosen.j_tile;
    if (chosen.stages) t.stages = chosen.stages;
    t.ctas_per_sm = chosen.ctas_per_sm;
    t.chunk_units = chosen.chunk_units;
    t.j_lanes = chosen.j_lanes > 1 ? chosen.j_lanes : 1;
  }
  p->k = guard ? 1 : t.i_per_thread;
  p->threads = t.threads;
  p->j_tile = t.j_tile;
  p->stages = t.stages;
  p->ctas_per_sm = t.ctas_per_sm;
  p->chunk_units = t.chunk_units;
  p->j_lanes = t.j_lanes > 1 ? t.j_lanes : 1;
  if (p->j_lanes > 1 && variant == cn::kSym) return fail(CN_ERR_INVALID_ARG, "the symmetric form takes no j_lanes");
  if (p->j_lanes > 1 && (variant == cn::kJerk || variant == cn::kJerkPot || variant == cn::kAdjoint) && guard) {
    p->j_lanes = 1;  // the guarded force-jerk and adjoint kernels hold one i-particle per thread, without split-j
    p->k = 1;
  }
  if (p->j_lanes > 1) {
    // split-j: K i-particles per lane group (packed for K >= 2; the guarded
    // kernels hold one, the per-i-softening ones at most two)
    const bool eps_i = variant == cn::kF32EpsI || variant == cn::kF32EpsIPot;
    if (guard) p->k = 1;
    else if (eps_i && p->k > 2) p->k = 2;
    if (p->j_tile % (8 * p->j_lanes)) return fail(CN_ERR_INVALID_ARG, "j_tile must be a multiple of 8 x j_lanes");
  }
  const size_t smem = variant == cn::kSym
                          ? cn::sym_smem_bytes(p->threads, p->k, p->j_tile, p->stages, false)
                          : (two_records(variant) ? cn::adjoint_smem_bytes(*p) : cn::ring_smem_bytes(*p));
  if (smem > kMaxSmem) return fail(CN_ERR_INVALID_ARG, "the launch shape exceeds the shared memory of one CTA");
  if (variant == cn::kSym && p->i_tile() % p->j_tile) p->j_tile = std::min(p->j_tile, p->i_tile());
  if (variant == cn::kSym && (p->i_tile() % p->j_tile || p->j_tile % 8))
    return fail(CN_ERR_INVALID_ARG, "symmetric form: j_tile must divide threads x i_per_thread and be a multiple of 8");
  return CN_OK;
}

// ------------------------------------------------------------------ geometry
struct Geometry {
  int64_t n_tiles = 0;
  int64_t njt = 0;
  int64_t units = 0;
  int64_t n_chunks = 0;
  int grid = 0;
  size_t smem = 0;
  size_t ctrl_bytes = 0;  // queue words + arrival counters (must be zero at launch)
  size_t data_bytes = 0;  // partial sums (+ packed weights)
  size_t off_wrec = 0;    // packed weights, from the start of the data region
  size_t ws_bytes = 0;    // one caller buffer: control region, then data region
};

std::map<std::tuple<int, int, bool, int, int, int, size_t>, int> g_occ;

// One line per launch on stderr when CN_LOG is set: the variant, sizes,
// launch shape, grid, units, chunks and how many i-tiles are split across
// chunks (those take the FP64 merge). Single-system schedules only count
// split tiles; batched plans pass n_tiles_split < 0.
void log_plan(const char* entry, int variant, int64_t n_i, int64_t n_j, bool guard, const Plan& p, const Geometry& g,
              int64_t njt) {
  if (!log_enabled()) return;
  int64_t split = -1;
  if (njt > 0 && g.units > 0 && p.chunk_units == 0) {
    split = 0;
    const int64_t U = g.units, Q = g.n_chunks;
    auto chunk_of = [&](int64_t u) { return ((u + 1) * Q - 1) / U; };
    for (int64_t t = 0; t < g.n_tiles; ++t)
      if (chunk_of(t * njt) != chunk_of(t * njt + njt - 1)) ++split;
  }
  std::fprintf(stderr,
               "[cunbody] %s: variant %s n_i %lld n_j %lld%s | K %d threads %d j_tile %d stages %d j_lanes %d "
               "chunk_units %lld ctas_per_sm %d | grid %d units %lld chunks %lld i_tiles %lld split_tiles %lld "
               "smem %zu ws %zu\n",
               entry, variant_name(variant), static_cast<long long>(n_i), static_cast<long long>(n_j),
               guard ? " (guarded)" : "", p.k, p.threads, p.j_tile, p.stages, p.j_lanes,
               static_cast<long long>(p.chunk_units), p.ctas_per_sm, g.grid, static_cast<long long>(g.units),
               static_cast<long long>(g.n_chunks), static_cast<long long>(g.n_tiles), static_cast<long long>(split),
               g.smem, g.ws_bytes);
}

cn_status occupancy(int dev, int variant, bool guard, const Plan& p, size_t smem, int* ctas, bool gather = false) {
  const auto key = std::make_tuple(dev, variant + (gather ? 100 : 0), guard, p.j_lanes, p.k, p.threads, smem);
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) {
      *ctas = it->second;
      return CN_OK;
    }
  }
  int c = 0;
  cudaError_t e;
  switch (variant) {
    case cn::kF32: e = cn::occupancy_f32(p, false, guard, false, smem, &c); break;
    case cn::kF32Pot: e = cn::occupancy_f32(p, true, guard, false, smem, &c); break;
    case cn::kDD: e = cn::occupancy_dd(p, false, guard, smem, &c); break;
    case cn::kDDPot: e = cn::occupancy_dd(p, true, guard, smem, &c); break;
    case cn::kAdjoint: e = cn::occupancy_adjoint(p, guard, smem, &c); break;
    case cn::kBatched:
      e = gather ? cn::occupancy_f32_gather(p, false, guard, smem, &c) : cn::occupancy_f32(p, false, guard, true, smem, &c);
      break;
    case cn::kBatchedPot:
      e = gather ? cn::occupancy_f32_gather(p, true, guard, smem, &c) : cn::occupancy_f32(p, true, guard, true, smem, &c);
      break;
    case cn::kJerk: e = cn::occupancy_jerk(p, false, guard, smem, &c); break;
    case cn::kJerkPot: e = cn::occupancy_jerk(p, true, guard, smem, &c); break;
    case cn::kF32EpsI: e = cn::occupancy_f32(p, false, true, false, smem, &c, true); break;
    case cn::kF32EpsIPot: e = cn::occupancy_f32(p, true, true, false, smem, &c, true); break;
    default: return fail(CN_ERR_INVALID_ARG, "unknown variant");
  }
  if (e != cudaSuccess) return fail_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (c <= 0) return fail(CN_ERR_INVALID_ARG, "launch shape does not fit on one SM");
  std::lock_guard<std::mutex> lock(g_mu);
  g_occ[key] = c;
  *ctas = c;
  return CN_OK;
}

int slot_f4(int variant) {
  return (variant == cn::kDD || variant == cn::kDDPot || variant == cn::kJerk || variant == cn::kJerkPot) ? 2 : 1;
}

// Grid and workspace layout for `units` units over `n_tiles` i-tiles
// (gather: the gathering list kernel).
cn_status layout(int dev, const DeviceInfo& d, int variant, bool guard, const Plan& p, int64_t n_tiles,
                 int64_t units, int64_t n_wrec, Geometry* g, bool gather = false) {
  g->n_tiles = n_tiles;
  g->units = units;
  g->smem = gather ? cn::gather_smem_bytes(p) : two_records(variant) ? cn::adjoint_smem_bytes(p) : cn::ring_smem_bytes(p);
  if (g->smem > kMaxSmem) return fail(CN_ERR_INVALID_ARG, "the launch shape exceeds the shared memory of one CTA");
  int occ = 0;
  cn_status st = occupancy(dev, variant, guard, p, g->smem, &occ, gather);
  if (st != CN_OK) return st;
  const int ctas = p.ctas_per_sm > 0 ? std::min(p.ctas_per_sm, occ) : occ;
  const int64_t slots = static_cast<int64_t>(ctas) * d.sms;
  if (p.chunk_units == 0) {
    g->n_chunks = std::min<int64_t>(slots, units);
    g->grid = static_cast<int>(g->n_chunks);
  } else {
    g->n_chunks = ceil_div(units, p.chunk_units);
    g->grid = static_cast<int>(std::min<int64_t>(slots, g->n_chunks));
  }
  if (g->n_tiles > INT32_MAX || g->n_chunks > INT32_MAX)
    return fail(CN_ERR_INVALID_ARG, "problem too large for one launch");
  g->ctrl_bytes = align_up(kCtrlBytes + static_cast<size_t>(n_tiles) * 4, 256);
  const size_t partial_bytes =
      static_cast<size_t>(g->n_chunks) * 2 * static_cast<size_t>(p.i_tile()) * 16 * slot_f4(variant);
  g->off_wrec = align_up(partial_bytes, 256);
  g->data_bytes = g->off_wrec + static_cast<size_t>(n_wrec) * 16;
  g->ws_bytes = g->ctrl_bytes + g->data_bytes;
  return CN_OK;
}

cn_status single_geometry(int dev, const DeviceInfo& d, int variant, bool guard, const Plan& p, int64_t n_i,
                          int64_t n_j, Geometry* g) {
  const int64_t n_tiles = ceil_div(n_i, p.i_tile());
  const int64_t njt = ceil_div(n_j, p.j_tile);
  if (njt > INT32_MAX) return fail(CN_ERR_INVALID_ARG, "n_j too large");
  g->njt = njt;
  return layout(dev, d, variant, guard, p, n_tiles, n_tiles * njt, variant == cn::kAdjoint ? n_i : 0, g);
}

PairArgs base_args(char* ctrl, char* data, const Geometry& g, const Plan& p, int* status) {
  PairArgs a{};
  a.queue = reinterpret_cast<int*>(ctrl);
  a.counters = reinterpret_cast<unsigned int*>(ctrl + kCtrlBytes);
  a.partials = reinterpret_cast<float4*>(data);
  a.status = status;
  a.total_units = g.units;
  a.chunk_units = p.chunk_units;
  a.n_chunks = g.n_chunks;
  a.n_tiles = static_cast<int32_t>(g.n_tiles);
  a.njt = static_cast<int32_t>(g.njt);
  a.j_tile = p.j_tile;
  a.stages = p.stages;
  a.j_lanes = p.j_lanes;
  a.wait_ns = g_wait_ns.load();
  return a;
}

// Resolves the workspace of a launch: the library's (per stream) or one
// caller buffer whose control head is cleared here, on the stream.
cn_status launch_workspace(cudaStream_t s, const Geometry& g, void* ws, size_t ws_bytes, bool lib_ws, char** ctrl,
                           char** data) {
  if (lib_ws) return library_workspace(s, g.ctrl_bytes, g.data_bytes, ctrl, data);
  if (!ws || ws_bytes < g.ws_bytes) return fail(CN_ERR_WORKSPACE, "workspace smaller than the size this call needs");
  if (!aligned(ws, 256)) return fail(CN_ERR_MISALIGNED, "workspace must be 256-byte aligned");
  cudaError_t e = cudaMemsetAsync(ws, 0, g.ctrl_bytes, s);
  if (e != cudaSuccess) return fail_cuda(e, "cudaMemsetAsync(workspace control)");
  *ctrl = static_cast<char*>(ws);
  *data = static_cast<char*>(ws) + g.ctrl_bytes;
  return CN_OK;
}

cn_status check_eps2(float eps2) {
  if (!std::isfinite(eps2) || eps2 < 0.f) return fail(CN_ERR_INVALID_ARG, "eps2 must be finite and >= 0");
  return CN_OK;
}

// eps2 below the smallest normal float can make s flush to zero: take the guarded kernels.
bool needs_guard(float eps2) { return !(eps2 >= FLT_MIN); }

cn_status check_records(const float* p, int64_t n, const char* name) {
  if (n > 0 && !p) return fail(CN_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (p && !aligned(p, 16)) return fail(CN_ERR_MISALIGNED, std::string(name) + " must be 16-byte aligned");
  return CN_OK;
}

// ------------------------------------------------------------------ single-system force
// eps_i: the softening of each pair is its i-particle's, from the 4th slot
// of its record (eps2 is not used); the kernels then always take the s = 0
// guard.
cn_status force_common(bool dd, int64_t n_i, const float* pos_i, int64_t n_j, const float* pos_mass_j,
                       float eps2, void* acc_out, void* pot_out, void* ws, size_t ws_bytes, bool lib_ws,
                       cudaStream_t s, bool eps_i = false) {
  if (n_i < 0 || n_j < 0) return fail(CN_ERR_INVALID_ARG, "n_i and n_j must be >= 0");
  cn_status st;
  if (!eps_i && (st = check_eps2(eps2)) != CN_OK) return st;
  if ((st = check_records(pos_i, n_i, "pos_i")) != CN_OK) return st;
  if ((st = check_records(pos_mass_j, n_j, "pos_mass_j")) != CN_OK) return st;
  const size_t elt = dd ? sizeof(double) : sizeof(float);
  if (n_i > 0 && !acc_out) return fail(CN_ERR_INVALID_ARG, "acc_out is NULL");
  if ((acc_out && !aligned(acc_out, elt)) || (pot_out && !aligned(pot_out, elt)))
    return fail(CN_ERR_MISALIGNED, "outputs must be aligned to their element size");
  const size_t acc_b = static_cast<size_t>(n_i) * 3 * elt, pot_b = pot_out ? static_cast<size_t>(n_i) * elt : 0;
  const size_t pi_b = static_cast<size_t>(n_i) * 16, pj_b = static_cast<size_t>(n_j) * 16;
  if (overlaps(acc_out, acc_b, pos_i, pi_b) || overlaps(acc_out, acc_b, pos_mass_j, pj_b) ||
      overlaps(pot_out, pot_b, pos_i, pi_b) || overlaps(pot_out, pot_b, pos_mass_j, pj_b) ||
      overlaps(acc_out, acc_b, pot_out, pot_b))
    return fail(CN_ERR_INVALID_ARG, "outputs overlap inputs or each other");
  if (n_i == 0) return CN_OK;
  int dev = 0;
  DeviceInfo* d = nullptr;
  if ((st = current_device(&dev, &d)) != CN_OK) return st;
  cudaError_t e;
  if (n_j == 0) {
    if ((e = cudaMemsetAsync(acc_out, 0, acc_b, s)) != cudaSuccess) return fail_cuda(e, "cudaMemsetAsync");
    if (pot_out && (e = cudaMemsetAsync(pot_out, 0, pot_b, s)) != cudaSuccess) return fail_cuda(e, "cudaMemsetAsync");
    return CN_OK;
  }
  const bool pot = pot_out != nullptr;
  const bool guard = eps_i || needs_guard(eps2);
  const int variant = eps_i ? (pot ? cn::kF32EpsIPot : cn::kF32EpsI)
                            : (dd ? (pot ? cn::kDDPot : cn::kDD) : (pot ? cn::kF32Pot : cn::kF32));
  struct Cached {
    PlanCache key;
    Plan p;
    Geometry g;
    char* ctrl = nullptr;
    char* data = nullptr;
  };
  thread_local Cached t_last;
  Plan p;
  Geometry g;
  char *ctrl = nullptr, *data = nullptr;
  const uint64_t gen0 = g_plan_gen.load(std::memory_order_acquire);
  const PlanCache& k = t_last.key;
  if (lib_ws && k.valid && k.gen == gen0 && k.dev == dev && k.variant == variant && k.n_i == n_i && k.n_j == n_j &&
      k.guard == guard && k.stream == s) {
    p = t_last.p;
    g = t_last.g;
    ctrl = t_last.ctrl;
    data = t_last.data;
  } else {
    const uint64_t bumps0 = t_own_bumps;
    // the per-particle kernels are guarded in every shape, so K is not restricted to 1
    if ((st = resolve_plan(dev, variant, n_i, n_j, guard && !eps_i, nullptr, &p)) != CN_OK) return st;
    if ((st = single_geometry(dev, *d, variant, guard, p, n_i, n_j, &g)) != CN_OK) return st;
    if ((st = launch_workspace(s, g, ws, ws_bytes, lib_ws, &ctrl, &data)) != CN_OK) return st;
    // cache only a plan that nothing changed under (another thread's tuning
    // or workspace change would show as a generation step not our own)
    const uint64_t gen1 = g_plan_gen.load(std::memory_order_acquire);
    if (lib_ws && gen1 == gen0 + (t_own_bumps - bumps0)) {
      t_last.key = PlanCache{true, gen1, dev, variant, n_i, n_j, guard, s};
      t_last.p = p;
      t_last.g = g;
      t_last.ctrl = ctrl;
      t_last.data = data;
    }
  }
  PairArgs a = base_args(ctrl, data, g, p, d->status);
  a.pos_i = reinterpret_cast<const float4*>(pos_i);
  a.pos_j = reinterpret_cast<const float4*>(pos_mass_j);
  a.acc_out = acc_out;
  a.pot_out = pot_out;
  a.n_i = n_i;
  a.n_j = n_j;
  a.eps2 = eps2;
  log_plan(dd ? "cn_force_dd" : (eps_i ? "cn_force_eps_i" : "cn_force"), variant, n_i, n_j, guard, p, g, g.njt);
  if (inject("launch")) return fail(CN_ERR_CUDA, "kernel launch: injected launch failure");
  e = dd ? cn::launch_dd(a, p, pot, guard, g.grid, s) : cn::launch_f32(a, p, pot, guard, false, g.grid, s, eps_i);
  if (e != cudaSuccess) return fail_cuda(e, "pair kernel launch");
  return CN_OK;
}

cn_status jerk_common(int64_t n_i, const float* pos_i, const float* vel_i, int64_t n_j, const float* pos_mass_j,
                      const float* vel_j, float eps2, float* acc_out, float* jerk_out, float* pot_out,
                      cudaStream_t s) {
  if (n_i < 0 || n_j < 0) return fail(CN_ERR_INVALID_ARG, "n_i and n_j must be >= 0");
  cn_status st;
  if ((st = check_eps2(eps2)) != CN_OK) return st;
  if ((st = check_records(pos_i, n_i, "pos_i")) != CN_OK) return st;
  if ((st = check_records(vel_i, n_i, "vel_i")) != CN_OK) return st;
  if ((st = check_records(pos_mass_j, n_j, "pos_mass_j")) != CN_OK) return st;
  if ((st = check_records(vel_j, n_j, "vel_j")) != CN_OK) return st;
  if (n_i > 0 && (!acc_out || !jerk_out)) return fail(CN_ERR_INVALID_ARG, "acc_out and jerk_out are required");
  if ((acc_out && !aligned(acc_out, 4)) || (jerk_out && !aligned(jerk_out, 4)) || (pot_out && !aligned(pot_out, 4)))
    return fail(CN_ERR_MISALIGNED, "outputs must be 4-byte aligned");
  const size_t ob = static_cast<size_t>(n_i) * 12, pb = pot_out ? static_cast<size_t>(n_i) * 4 : 0;
  const size_t ib = static_cast<size_t>(n_i) * 16, jb = static_cast<size_t>(n_j) * 16;
  const void* ins[4] = {pos_i, vel_i, pos_mass_j, vel_j};
  const size_t insz[4] = {ib, ib, jb, jb};
  const void* outs[3] = {acc_out, jerk_out, pot_out};
  const size_t outsz[3] = {ob, ob, pb};
  for (int o = 0; o < 3; ++o) {
    for (int q = 0; q < 4; ++q)
      if (overlaps(outs[o], outsz[o], ins[q], insz[q])) return fail(CN_ERR_INVALID_ARG, "outputs overlap inputs");
    for (int q = o + 1; q < 3; ++q)
      if (overlaps(outs[o], outsz[o], outs[q], outsz[q])) return fail(CN_ERR_INVALID_ARG, "outputs overlap each other");
  }
  if (n_i == 0) return CN_OK;
  int dev = 0;
  DeviceInfo* d = nullptr;
  if ((st = current_device(&dev, &d)) != CN_OK) return st;
  cudaError_t e;
  if (n_j == 0) {
    for (int o = 0; o < 3; ++o)
      if (outs[o] && (e = cudaMemsetAsync(const_cast<void*>(outs[o]), 0, outsz[o], s)) != cudaSuccess)
        return fail_cuda(e, "cudaMemsetAsync");
    return CN_OK;
  }
  const bool pot = pot_out != nullptr;
  const bool guard = needs_guard(eps2);
  const int variant = pot ? cn::kJerkPot : cn::kJerk;
  Plan p;
  if ((st = resolve_plan(dev, variant, n_i, n_j, guard, nullptr, &p)) != CN_OK) return st;
  Geometry g;
  if ((st = single_geometry(dev, *d, variant, guard, p, n_i, n_j, &g)) != CN_OK) return st;
  char *ctrl = nullptr, *data = nullptr;
  if ((st = library_workspace(s, g.ctrl_bytes, g.data_bytes, &ctrl, &data)) != CN_OK) return st;
  PairArgs a = base_args(ctrl, data, g, p, d->status);
  a.pos_i = reinterpret_cast<const float4*>(pos_i);
  a.pos_i2 = reinterpret_cast<const float4*>(vel_i);
  a.pos_j = reinterpret_cast<const float4*>(pos_mass_j);
  a.pos_j2 = reinterpret_cast<const float4*>(vel_j);
  a.acc_out = acc_out;
  a.jerk_out = jerk_out;
  a.pot_out = pot_out;
  a.n_i = n_i;
  a.n_j = n_j;
  a.eps2 = eps2;
  log_plan("cn_force_jerk", variant, n_i, n_j, guard, p, g, g.njt);
  if (inject("launch")) return fail(CN_ERR_CUDA, "kernel launch: injected launch failure");
  e = cn::launch_jerk(a, p, pot, guard, g.grid, s);
  return e == cudaSuccess ? CN_OK : fail_cuda(e, "force-jerk kernel launch");
}

cn_status symmetric_common(int64_t n, const float* pos_mass, float eps2, float* acc_out, float* pot_out,
                           cudaStream_t s) {
  if (n < 0) return fail(CN_ERR_INVALID_ARG, "n must be >= 0");
  cn_status st;
  if ((st = check_eps2(eps2)) != CN_OK) return st;
  if ((st = check_records(pos_mass, n, "pos_mass")) != CN_OK) return st;
  if (n > 0 && !acc_out) return fail(CN_ERR_INVALID_ARG, "acc_out is NULL");
  if ((acc_out && !aligned(acc_out, 4)) || (pot_out && !aligned(pot_out, 4)))
    return fail(CN_ERR_MISALIGNED, "outputs must be 4-byte aligned");
  const size_t nb = static_cast<size_t>(n);
  if (overlaps(acc_out, nb * 12, pos_mass, nb * 16) || overlaps(pot_out, nb * 4, pos_mass, nb * 16) ||
      overlaps(acc_out, nb * 12, pot_out, nb * 4))
    return fail(CN_ERR_INVALID_ARG, "outputs overlap pos_mass or each other");
  const bool pot = pot_out != nullptr;
  if (n == 0) return CN_OK;
  int dev = 0;
  DeviceInfo* d = nullptr;
  if ((st = current_device(&dev, &d)) != CN_OK) return st;
  const bool guard = needs_guard(eps2);
  // with the potential the default shape must leave room for four sums per
  // particle in the shared-memory rows
  cn_tune pot_tune{};
  const cn_tune* shape = nullptr;
  if (pot && !registered_tune(dev, cn::kSym, n, n)) {
    pot_tune = sym_default_tune(n, d->sms, true);
    shape = &pot_tune;
  }
  Plan p;
  if ((st = resolve_plan(dev, cn::kSym, n, n, guard, shape, &p)) != CN_OK) return st;
  const int64_t B = p.i_tile();
  const int64_t T = ceil_div(n, B);
  if (T > 65535) return fail(CN_ERR_INVALID_ARG, "too many tiles for the symmetric form");
  const size_t smem = cn::sym_smem_bytes(p.threads, p.k, p.j_tile, p.stages, pot);
  if (smem > kMaxSmem) return fail(CN_ERR_INVALID_ARG, "the launch shape exceeds the shared memory of one CTA");
  int occ = 0;
  cudaError_t e = cn::occupancy_sym(p.k, guard, p.threads, smem, &occ, pot);
  if (e != cudaSuccess) return fail_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (occ <= 0) return fail(CN_ERR_INVALID_ARG, "launch shape does not fit on one SM");
  // Slots: the j-side sums of every off-diagonal unit, one [T][n_pad] array
  // (16 T n_pad bytes, ~16 N^2 / B, half of it written) when it fits in
  // kSymSlotCap, else bands of w tile rows with [w][n_pad] j-side slots and
  // FP64 running sums (~16 w N + 32 N bytes); plus the i-side segments,
  // [CTAs + rows of the band][2][B] ((hi, lo) sums per CTA and row it
  // touches). The tune's chunk_units, when set, fixes the rows per band.
  const int64_t n_pad = T * B;
  int64_t w = T;
  if (p.chunk_units > 0)
    w = std::min<int64_t>(p.chunk_units, T);
  else if (static_cast<double>(T) * static_cast<double>(n_pad) * 16.0 > static_cast<double>(kSymSlotCap))
    w = std::max<int64_t>(1, std::min<int64_t>(T, static_cast<int64_t>(kSymSlotCap / (16 * static_cast<size_t>(n_pad)))));
  const bool banded = w < T;
  const int64_t slots = static_cast<int64_t>(p.ctas_per_sm > 0 ? std::min(p.ctas_per_sm, occ) : occ) * d->sms;
  const size_t jslot_b = align_up(static_cast<size_t>(w) * static_cast<size_t>(n_pad) * 16, 256);
  const size_t seg_b = align_up(static_cast<size_t>(slots + w) * static_cast<size_t>(B) * 32, 256);  // (hi, lo)
  const size_t acc64_b = banded ? static_cast<size_t>(n) * 32 : 0;
  const size_t need = jslot_b + seg_b + acc64_b;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && need > free_b + library_data_bytes(s))
    return fail(CN_ERR_WORKSPACE, "symmetric form: the slot arrays do not fit in device memory");
  char *ctrl = nullptr, *data = nullptr;
  if ((st = library_workspace(s, kCtrlBytes, need, &ctrl, &data)) != CN_OK) return st;
  cn::SymArgs a{};
  a.pos = reinterpret_cast<const float4*>(pos_mass);
  a.slots_j = reinterpret_cast<float4*>(data);
  a.slots_seg = reinterpret_cast<float4*>(data + jslot_b);
  a.n_seg = slots + w;
  a.status = d->status;
  a.n = n;
  a.n_pad = n_pad;
  a.n_tiles = static_cast<int32_t>(T);
  a.sub_tile = p.j_tile;
  a.stages = p.stages;
  a.eps2 = eps2;
  a.wait_ns = g_wait_ns.load();
  cn::SymMerge m{};
  m.slots_seg = a.slots_seg;
  m.slots_j = a.slots_j;
  m.acc64 = banded ? reinterpret_cast<double*>(data + jslot_b + seg_b) : nullptr;
  m.acc_out = acc_out;
  m.pot_out = pot_out;
  m.n = n;
  m.n_pad = n_pad;
  m.tile = static_cast<int32_t>(B);
  m.n_tiles = static_cast<int32_t>(T);
  auto row_start = [T](int64_t r) { return r * T - r * (r - 1) / 2; };  // first unit of tile row r
  for (int64_t r0 = 0; r0 < T; r0 += w) {
    const int64_t r1 = std::min(T, r0 + w);
    a.row0 = static_cast<int32_t>(r0);
    a.unit_base = row_start(r0);
    a.units = row_start(r1) - row_start(r0);
    m.row0 = static_cast<int32_t>(r0);
    m.row1 = static_cast<int32_t>(r1);
    m.first = r0 == 0;
    m.last = r1 == T;
    const int grid = static_cast<int>(std::min<int64_t>(slots, a.units));
    m.unit_base = a.unit_base;
    m.units = a.units;
    m.grid = grid;
    if (log_enabled())
      std::fprintf(stderr,
                   "[cunbody] cn_force_symmetric: n %lld%s%s | K %d threads %d sub_tile %d stages %d | tile %lld "
                   "tiles %lld band rows %lld..%lld units %lld grid %d smem %zu slots %zu bytes\n",
                   static_cast<long long>(n), pot ? " +pot" : "", guard ? " (guarded)" : "", guard ? 1 : p.k,
                   p.threads, p.j_tile, p.stages, static_cast<long long>(B), static_cast<long long>(T),
                   static_cast<long long>(r0), static_cast<long long>(r1), static_cast<long long>(a.units), grid, smem,
                   need);
    if (inject("launch")) return fail(CN_ERR_CUDA, "kernel launch: injected launch failure");
    e = cn::launch_sym(a, m, guard ? 1 : p.k, guard, p.threads, grid, smem, s, pot);
    if (e != cudaSuccess) return fail_cuda(e, "symmetric kernel launch");
  }
  return CN_OK;
}

cn_status run_batched(const cn_batch_plan* plan, const float* pos_i, const float* pos_j, float* acc_out,
                      float* pot_out, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (!plan) return fail(CN_ERR_INVALID_ARG, "plan is NULL");
  cn_status st;
  if ((st = check_records(pos_i, plan->n_total, "pos_i")) != CN_OK) return st;
  if ((st = check_records(pos_j, plan->n_j_total, "pos_mass_j")) != CN_OK) return st;
  if (plan->n_total > 0 && !acc_out) return fail(CN_ERR_INVALID_ARG, "acc_out is NULL");
  if ((acc_out && !aligned(acc_out, 4)) || (pot_out && !aligned(pot_out, 4)))
    return fail(CN_ERR_MISALIGNED, "outputs must be 4-byte aligned");
  if (pot_out && !plan->pot) return fail(CN_ERR_INVALID_ARG, "plan was created without the potential form");
  const size_t n = static_cast<size_t>(plan->n_total), nj = static_cast<size_t>(plan->n_j_total);
  if (overlaps(acc_out, n * 12, pos_i, n * 16) || overlaps(pot_out, n * 4, pos_i, n * 16) ||
      overlaps(acc_out, n * 12, pos_j, nj * 16) || overlaps(pot_out, n * 4, pos_j, nj * 16) ||
      overlaps(acc_out, n * 12, pot_out, n * 4))
    return fail(CN_ERR_INVALID_ARG, "outputs overlap inputs or each other");
  int dev = 0;
  DeviceInfo* d = nullptr;
  if ((st = current_device(&dev, &d)) != CN_OK) return st;
  if (dev != plan->dev) return fail(CN_ERR_INVALID_ARG, "plan was built on another device");
  cudaError_t e;
  if (plan->units == 0 || plan->zero_first) {
    if (n && (e = cudaMemsetAsync(acc_out, 0, n * 12, s)) != cudaSuccess) return fail_cuda(e, "cudaMemsetAsync");
    if (n && pot_out && (e = cudaMemsetAsync(pot_out, 0, n * 4, s)) != cudaSuccess)
      return fail_cuda(e, "cudaMemsetAsync");
    if (plan->units == 0) return CN_OK;
  }
  Geometry g;
  g.units = plan->units;
  g.n_chunks = plan->n_chunks;
  g.n_tiles = plan->n_tiles;
  g.ctrl_bytes = plan->ctrl_bytes;
  g.data_bytes = plan->data_bytes;
  g.ws_bytes = plan->ws_bytes;
  char *ctrl = nullptr, *data = nullptr;
  if ((st = launch_workspace(s, g, ws, ws_bytes, ws == nullptr, &ctrl, &data)) != CN_OK) return st;
  PairArgs a = base_args(ctrl, data, g, plan->plan, d->status);
  a.pos_i = reinterpret_cast<const float4*>(pos_i);
  a.pos_j = reinterpret_cast<const float4*>(pos_j);
  a.acc_out = acc_out;
  a.pot_out = pot_out;
  a.tiles = plan->d_tiles;
  a.n_i = plan->n_total;
  a.n_j = plan->n_j_total;
  a.j_index = plan->d_index;
  a.n_index = plan->n_index;
  if (log_enabled()) {
    Geometry lg = g;
    lg.grid = plan->grid;
    lg.smem = plan->d_index ? cn::gather_smem_bytes(plan->plan) : cn::ring_smem_bytes(plan->plan);
    log_plan(plan->lists ? (plan->d_index ? "cn_force_lists (index lists)" : "cn_force_lists") : "cn_force_batched",
             plan->pot ? cn::kBatchedPot : cn::kBatched, plan->n_total, plan->n_j_total, plan->guard, plan->plan, lg,
             0);
  }
  if (inject("launch")) return fail(CN_ERR_CUDA, "kernel launch: injected launch failure");
  e = plan->d_index ? cn::launch_f32_gather(a, plan->plan, plan->pot, plan->guard, plan->grid, s)
                    : cn::launch_f32(a, plan->plan, plan->pot, plan->guard, true, plan->grid, s);
  if (e != cudaSuccess) return fail_cuda(e, "batched pair kernel launch");
  return CN_OK;
}

// One group of the work: i-particles [i_begin, i_begin + ni) against the j
// records [j_begin, j_begin + nj) with softening eps2.
struct Group {
  int64_t i_begin, ni, j_begin, nj;
  float eps2;
};

// Builds the (group, i-tile, j-tile) unit table of a plan and uploads it.
// index_host (gathering list plans): n_index list entries, each the index of
// a j record; the groups' j ranges then count entries of this array.
cn_status build_group_plan(const std::vector<Group>& groups, bool lists, int64_t n_i_total, int64_t n_j_total,
                           const cn_tune* tune, int with_pot, cn_batch_plan** out, const int32_t* index_host = nullptr,
                           int64_t n_index = 0) {
  const bool gather = index_host != nullptr;
  bool guard = false, zero_first = false;
  double pairs = 0.0;
  for (const Group& gr : groups) {
    cn_status st = check_eps2(gr.eps2);
    if (st != CN_OK) return st;
    if (gr.ni > 0 && gr.nj > 0 && needs_guard(gr.eps2)) guard = true;
    if (gr.ni > 0 && gr.nj == 0) zero_first = true;
    pairs += static_cast<double>(gr.ni) * static_cast<double>(gr.nj);
  }
  int dev = 0;
  DeviceInfo* d = nullptr;
  cn_status st = current_device(&dev, &d);
  if (st != CN_OK) return st;
  const int variant = with_pot ? cn::kBatchedPot : cn::kBatched;
  const int64_t key_i = static_cast<int64_t>(groups.size());
  cn_tune fitted{};
  if (!tune && !registered_tune(dev, variant, key_i, n_i_total)) {
    // i-tile fitted to the group sizes: every group is cut into whole i-tiles,
    // so a tile larger than the typical group leaves lanes idle, and every
    // j range into whole j-tiles (padded with zero masses). Among the
    // shapes below take the one with the least evaluated-but-padded work,
    // weighted by each shape's relative pair rate, measured on GB300: the
    // packed K = 8 kernel 1.0, its split-j forms 0.95, K = 4 0.99, K = 2 x
    // 128 0.93, one particle per thread 0.80. Ensembles (eight of them, 64 ..
    // 65536 particles per cluster) add K = 4 x 64 at 0.99, ahead of 4 x 128
    // (the same rate with half the i-tile), K = 2 x 64 with 128-record
    // j-tiles at 0.93 (clusters of a few hundred), and rate the 128-thread split-j
    // form 0.75 (0.29 against 0.67 of the FP32 bound for 4096 clusters of
    // 256); interaction lists keep their measured set (groups of 256 against
    // 4096-record lists: the 256-thread split-j form 0.72, 4 x 64 below 0.70).
    struct Cand {
      int k, threads, j_lanes, j_tile;
      double rate;
      int use;  // 1: ensembles, 2: lists, 3: both
    };
    static const Cand cands[] = {{8, 256, 1, 512, 1.0, 3},   {8, 256, 2, 512, 0.95, 3}, {8, 256, 4, 512, 0.95, 3},
                                 {8, 256, 8, 512, 0.95, 3},  {8, 128, 8, 512, 0.94, 2}, {8, 128, 8, 512, 0.75, 1},
                                 {4, 64, 1, 256, 0.99, 1},   {4, 128, 1, 256, 0.99, 3}, {2, 128, 1, 256, 0.93, 3},
                                 {2, 64, 1, 128, 0.93, 1},   {1, 128, 1, 256, 0.80, 3}};
    double best = -1.0;
    for (const Cand& c : cands) {
      if (!(c.use & (lists ? 2 : 1))) continue;
      if (guard && (c.j_lanes > 1 || c.k > 1)) continue;  // the guarded kernels hold one particle, no split-j
      const int64_t it = static_cast<int64_t>(c.k) * c.threads / c.j_lanes;
      double padded = 0.0;
      for (const Group& gr : groups)
        padded += static_cast<double>(ceil_div(gr.ni, it) * it) * static_cast<double>(ceil_div(gr.nj, c.j_tile) * c.j_tile);
      const double score = padded > 0.0 ? pairs / padded * c.rate : c.rate;
      if (score > best) {
        best = score;
        fitted = default_tune(variant, key_i, n_i_total, d->sms);
        fitted.i_per_thread = c.k;
        fitted.threads = c.threads;
        fitted.j_lanes = c.j_lanes;
        fitted.j_tile = c.j_tile;
      }
    }
    // with the potential the K = 8 split-j kernel runs short of registers:
    // K = 4 with half the lane groups keeps the i-tile (lists of 4096 records
    // for groups of 256: 0.525 -> 0.712 of the 14-operation bound); the
    // gathering kernel, whose threads also stage records, does the same
    // (0.651 -> 0.673 of the FP32 bound on those lists as index arrays)
    if ((with_pot || gather) && fitted.i_per_thread == 8 && fitted.j_lanes > 1) {
      fitted.i_per_thread = 4;
      fitted.j_lanes /= 2;
      if (fitted.j_lanes < 2) fitted.j_lanes = 0;
    }
    tune = &fitted;
  }
  Plan p;
  if ((st = resolve_plan(dev, variant, key_i, n_i_total, guard, tune, &p)) != CN_OK) return st;
  // split-j batched kernels exist for K = 2, 4, 8 without the s = 0 guard
  if (p.j_lanes > 1 && (guard || p.k < 2)) p.j_lanes = 1;
  // tiles in order of decreasing work (largest first for the dynamic queue)
  std::vector<size_t> order(groups.size());
  for (size_t c = 0; c < groups.size(); ++c) order[c] = c;
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
    return groups[x].ni * groups[x].nj > groups[y].ni * groups[y].nj;
  });
  std::vector<cn::TileDesc> tiles;
  int64_t units = 0;
  const int it = p.i_tile();
  for (size_t c : order) {
    const Group& gr = groups[c];
    if (gr.ni == 0 || gr.nj == 0) continue;
    const int64_t njt = ceil_div(gr.nj, p.j_tile);
    if (njt > INT32_MAX) return fail(CN_ERR_INVALID_ARG, "a j set is too large");
    for (int64_t i0 = 0; i0 < gr.ni; i0 += it) {
      cn::TileDesc t{};
      t.i0 = gr.i_begin + i0;
      t.j0 = gr.j_begin;
      t.nj = gr.nj;
      t.unit0 = units;
      t.ni = static_cast<int32_t>(std::min<int64_t>(it, gr.ni - i0));
      t.njt = static_cast<int32_t>(njt);
      t.eps2 = gr.eps2;
      tiles.push_back(t);
      units += njt;
    }
  }
  Geometry g;
  if (!tiles.empty() &&
      (st = layout(dev, *d, variant, guard, p, static_cast<int64_t>(tiles.size()), units, 0, &g, gather)) != CN_OK)
    return st;
  // Ragged ensembles (cluster sizes spanning 4x or more) with the fitted
  // shape and many units per resident CTA take the dynamic queue in chunks
  // of 32 units (measured: 0.74 -> 0.78 of the FP32 bound on 512 clusters
  // of 256 .. 16384, 0.60 -> 0.63 on 2048 of 256 .. 2048, 0.77 -> 0.81 on
  // 256 of 128 .. 65536). Equal clusters keep the static schedule (1000 of
  // 1024: 0.73 static, 0.62 dynamic; 64 of 16384: 0.83 static, 0.72
  // dynamic), and so do launches with few units per slot, where the chunks
  // leave CTAs idle.
  int64_t ni_min = INT64_MAX, ni_max = 0;
  for (const Group& gr : groups)
    if (gr.ni > 0 && gr.nj > 0) {
      ni_min = std::min(ni_min, gr.ni);
      ni_max = std::max(ni_max, gr.ni);
    }
  if (!lists && tune == &fitted && !tiles.empty() && p.chunk_units == 0 && ni_max >= 4 * ni_min &&
      units >= 20 * static_cast<int64_t>(g.grid)) {
    p.chunk_units = 32;
    if ((st = layout(dev, *d, variant, guard, p, static_cast<int64_t>(tiles.size()), units, 0, &g, gather)) != CN_OK)
      return st;
  }
  auto* plan = new cn_batch_plan();
  plan->dev = dev;
  plan->lists = lists;
  plan->zero_first = zero_first;
  plan->n_clusters = static_cast<int32_t>(groups.size());
  plan->n_total = n_i_total;
  plan->n_j_total = n_j_total;
  plan->pairs = pairs;
  plan->plan = p;
  plan->guard = guard;
  plan->pot = with_pot != 0;
  plan->n_tiles = static_cast<int32_t>(tiles.size());
  plan->units = units;
  plan->n_chunks = g.n_chunks;
  plan->grid = g.grid;
  plan->ws_bytes = tiles.empty() ? 0 : g.ws_bytes;
  plan->ctrl_bytes = g.ctrl_bytes;
  plan->data_bytes = g.data_bytes;
  if (!tiles.empty()) {
    if (inject("alloc")) {
      delete plan;
      return fail(CN_ERR_CUDA, "cudaMalloc: injected allocation failure");
    }
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&plan->d_tiles), tiles.size() * sizeof(cn::TileDesc));
    if (e == cudaSuccess)
      e = cudaMemcpy(plan->d_tiles, tiles.data(), tiles.size() * sizeof(cn::TileDesc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && gather) {
      plan->n_index = n_index;
      e = cudaMalloc(reinterpret_cast<void**>(&plan->d_index), static_cast<size_t>(n_index) * sizeof(int32_t));
      if (e == cudaSuccess)
        e = cudaMemcpy(plan->d_index, index_host, static_cast<size_t>(n_index) * sizeof(int32_t),
                       cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
      cudaFree(plan->d_tiles);
      cudaFree(plan->d_index);
      delete plan;
      return fail_cuda(e, "uploading the batched unit table");
    }
  }
  *out = plan;
  return CN_OK;
}

cn_status build_batch_plan(int32_t n_clusters, const int64_t* offsets, const float* eps2, const cn_tune* tune,
                           int with_pot, cn_batch_plan** out) {
  if (!out) return fail(CN_ERR_INVALID_ARG, "plan_out is NULL");
  *out = nullptr;
  if (n_clusters < 0 || (n_clusters > 0 && (!offsets || !eps2)))
    return fail(CN_ERR_INVALID_ARG, "n_clusters < 0 or NULL offsets/eps2");
  if (n_clusters > 0 && offsets[0] != 0) return fail(CN_ERR_INVALID_ARG, "offsets[0] must be 0");
  std::vector<Group> groups(static_cast<size_t>(n_clusters));
  for (int32_t c = 0; c < n_clusters; ++c) {
    if (offsets[c + 1] < offsets[c]) return fail(CN_ERR_INVALID_ARG, "offsets must be non-decreasing");
    const int64_t nc = offsets[c + 1] - offsets[c];
    groups[c] = Group{offsets[c], nc, offsets[c], nc, eps2[c]};
  }
  const int64_t n_total = n_clusters > 0 ? offsets[n_clusters] : 0;
  if (inject("hostmem")) throw std::bad_alloc();
  return build_group_plan(groups, false, n_total, n_total, tune, with_pot, out);
}

cn_status build_list_plan(int32_t n_groups, const int64_t* i_offsets, const int64_t* j_begin, const int64_t* j_count,
                          const float* eps2, const cn_tune* tune, int with_pot, cn_batch_plan** out) {
  if (!out) return fail(CN_ERR_INVALID_ARG, "plan_out is NULL");
  *out = nullptr;
  if (n_groups < 0 || (n_groups > 0 && (!i_offsets || !j_begin || !j_count || !eps2)))
    return fail(CN_ERR_INVALID_ARG, "n_groups < 0 or a NULL array");
  if (n_groups > 0 && i_offsets[0] != 0) return fail(CN_ERR_INVALID_ARG, "i_offsets[0] must be 0");
  std::vector<Group> groups(static_cast<size_t>(n_groups));
  int64_t n_j_total = 0;
  for (int32_t c = 0; c < n_groups; ++c) {
    if (i_offsets[c + 1] < i_offsets[c]) return fail(CN_ERR_INVALID_ARG, "i_offsets must be non-decreasing");
    if (j_begin[c] < 0 || j_count[c] < 0) return fail(CN_ERR_INVALID_ARG, "negative list begin or count");
    groups[c] = Group{i_offsets[c], i_offsets[c + 1] - i_offsets[c], j_begin[c], j_count[c], eps2[c]};
    if (j_count[c] > 0) n_j_total = std::max(n_j_total, j_begin[c] + j_count[c]);
  }
  const int64_t n_i_total = n_groups > 0 ? i_offsets[n_groups] : 0;
  if (inject("hostmem")) throw std::bad_alloc();
  return build_group_plan(groups, true, n_i_total, n_j_total, tune, with_pot, out);
}

// Gathering list plan: group g's list is the entries j_begin[g] ..
// j_begin[g] + j_count[g] - 1 of j_index, each the index of one of n_src
// records. Every entry a list reaches is checked here, on the host.
cn_status build_list_plan_indexed(int32_t n_groups, const int64_t* i_offsets, const int64_t* j_begin,
                                  const int64_t* j_count, const float* eps2, const int32_t* j_index, int64_t n_index,
                                  int64_t n_src, const cn_tune* tune, int with_pot, cn_batch_plan** out) {
  if (!out) return fail(CN_ERR_INVALID_ARG, "plan_out is NULL");
  *out = nullptr;
  if (n_groups < 0 || (n_groups > 0 && (!i_offsets || !j_begin || !j_count || !eps2)))
    return fail(CN_ERR_INVALID_ARG, "n_groups < 0 or a NULL array");
  if (n_index < 0 || n_src < 0 || (n_index > 0 && !j_index))
    return fail(CN_ERR_INVALID_ARG, "n_index < 0, n_src < 0 or a NULL j_index");
  if (n_src > INT32_MAX) return fail(CN_ERR_INVALID_ARG, "n_src exceeds the 32-bit index range");
  if (n_groups > 0 && i_offsets[0] != 0) return fail(CN_ERR_INVALID_ARG, "i_offsets[0] must be 0");
  std::vector<Group> groups(static_cast<size_t>(n_groups));
  std::vector<char> reached(static_cast<size_t>(n_index), 0);
  for (int32_t c = 0; c < n_groups; ++c) {
    if (i_offsets[c + 1] < i_offsets[c]) return fail(CN_ERR_INVALID_ARG, "i_offsets must be non-decreasing");
    if (j_begin[c] < 0 || j_count[c] < 0) return fail(CN_ERR_INVALID_ARG, "negative list begin or count");
    if (j_count[c] > 0 && j_begin[c] + j_count[c] > n_index)
      return fail(CN_ERR_INVALID_ARG, "a list runs past the end of j_index");
    groups[c] = Group{i_offsets[c], i_offsets[c + 1] - i_offsets[c], j_begin[c], j_count[c], eps2[c]};
    if (groups[c].ni > 0)
      for (int64_t e = j_begin[c]; e < j_begin[c] + j_count[c]; ++e) reached[static_cast<size_t>(e)] = 1;
  }
  for (int64_t e = 0; e < n_index; ++e)
    if (reached[static_cast<size_t>(e)] && (j_index[e] < 0 || j_index[e] >= n_src))
      return fail(CN_ERR_INVALID_ARG, "a j_index entry lies outside 0 .. n_src - 1");
  const int64_t n_i_total = n_groups > 0 ? i_offsets[n_groups] : 0;
  if (inject("hostmem")) throw std::bad_alloc();
  return build_group_plan(groups, true, n_i_total, n_src, tune, with_pot, out, j_index != nullptr ? j_index : &kNoIndex,
                          n_index);
}

// Host staging buffers of cn_force_host, per (device, stream).
struct HostStage {
  void* buf = nullptr;
  size_t bytes = 0;
};
std::map<std::pair<int, cudaStream_t>, HostStage> g_stage;

cn_status stage_buffer(cudaStream_t s, size_t need, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(g_mu);
  HostStage& h = g_stage[{dev, s}];
  if (h.bytes < need) {
    if (inject("alloc")) return fail(CN_ERR_CUDA, "cudaMalloc: injected allocation failure");
    if (h.buf) {
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail_cuda(e, "cudaStreamSynchronize");
      cudaFree(h.buf);
      h.buf = nullptr;
      h.bytes = 0;
    }
    const size_t nb = align_up(need, static_cast<size_t>(1) << 20);
    if ((e = cudaMalloc(&h.buf, nb)) != cudaSuccess) return fail_cuda(e, "cudaMalloc(staging)");
    h.bytes = nb;
  }
  *out = h.buf;
  return CN_OK;
}

cn_status energy_common(int64_t n, const float* pos_mass, const float* pot_f, const double* pot_d, double* w_out,
                        cudaStream_t s) {
  if (n < 0) return fail(CN_ERR_INVALID_ARG, "n must be >= 0");
  if (!w_out || !aligned(w_out, 8)) return fail(CN_ERR_INVALID_ARG, "w_out must be a non-NULL aligned double pointer");
  cn_status st = check_records(pos_mass, n, "pos_mass");
  if (st != CN_OK) return st;
  if (n > 0 && !pot_f && !pot_d) return fail(CN_ERR_INVALID_ARG, "pot is NULL");
  int dev = 0;
  DeviceInfo* d = nullptr;
  if ((st = current_device(&dev, &d)) != CN_OK) return st;
  if (n == 0) {
    cudaError_t e = cudaMemsetAsync(w_out, 0, sizeof(double), s);
    return e == cudaSuccess ? CN_OK : fail_cuda(e, "cudaMemsetAsync");
  }
  double* aux = nullptr;
  if ((st = library_aux(s, &aux)) != CN_OK) return st;
  const size_t nb = cn::energy_workspace_doubles();
  if (inject("launch")) return fail(CN_ERR_CUDA, "kernel launch: injected launch failure");
  cudaError_t e = cn::launch_energy(n, reinterpret_cast<const float4*>(pos_mass), pot_f, pot_d, aux,
                                    reinterpret_cast<int*>(aux + nb), w_out, s);
  return e == cudaSuccess ? CN_OK : fail_cuda(e, "potential-energy kernel launch");
}

// ------------------------------------------------------------------ tuning file
// A small reader for the JSON the library writes (objects, arrays, strings
// without escapes other than \" and \\, integers, true/false/null).
struct JsonValue {
  enum Kind { kNull, kBool, kNumber, kString, kArray, kObject } kind = kNull;
  double number = 0.0;
  bool boolean = false;
  std::string text;
  std::vector<JsonValue> items;
  std::vector<std::pair<std::string, JsonValue>> fields;
  const JsonValue* get(const char* key) const {
    for (const auto& f : fields)
      if (f.first == key) return &f.second;
    return nullptr;
  }
};

struct JsonReader {
  const std::string& src;
  size_t pos = 0;
  int depth = 0;
  void skip() {
    while (pos < src.size() && (src[pos] == ' ' || src[pos] == '\n' || src[pos] == '\r' || src[pos] == '\t')) ++pos;
  }
  bool literal(const char* word) {
    const size_t n = std::strlen(word);
    if (src.compare(pos, n, word) != 0) return false;
    pos += n;
    return true;
  }
  bool string(std::string* out) {
    if (pos >= src.size() || src[pos] != '"') return false;
    ++pos;
    out->clear();
    while (pos < src.size() && src[pos] != '"') {
      char c = src[pos++];
      if (c == '\\') {
        if (pos >= src.size()) return false;
        c = src[pos++];
        if (c != '"' && c != '\\' && c != '/') return false;
      }
      out->push_back(c);
    }
    if (pos >= src.size()) return false;
    ++pos;
    return true;
  }
  bool value(JsonValue* v) {
    if (++depth > 16) return false;
    skip();
    bool ok = false;
    if (pos >= src.size()) {
      ok = false;
    } else if (src[pos] == '{') {
      v->kind = JsonValue::kObject;
      ++pos;
      skip();
      if (pos < src.size() && src[pos] == '}') {
        ++pos;
        ok = true;
      } else {
        for (;;) {
          skip();
          std::pair<std::string, JsonValue> f;
          if (!string(&f.first)) break;
          skip();
          if (pos >= src.size() || src[pos] != ':') break;
          ++pos;
          if (!value(&f.second)) break;
          v->fields.push_back(std::move(f));
          skip();
          if (pos < src.size() && src[pos] == ',') {
            ++pos;
            continue;
          }
          if (pos < src.size() && src[pos] == '}') {
            ++pos;
            ok = true;
          }
          break;
        }
      }
    } else if (src[pos] == '[') {
      v->kind = JsonValue::kArray;
      ++pos;
      skip();
      if (pos < src.size() && src[pos] == ']') {
        ++pos;
        ok = true;
      } else {
        for (;;) {
          JsonValue item;
          if (!value(&item)) break;
          v->items.push_back(std::move(item));
          skip();
          if (pos < src.size() && src[pos] == ',') {
            ++pos;
            continue;
          }
          if (pos < src.size() && src[pos] == ']') {
            ++pos;
            ok = true;
          }
          break;
        }
      }
    } else if (src[pos] == '"') {
      v->kind = JsonValue::kString;
      ok = string(&v->text);
    } else if (literal("true")) {
      v->kind = JsonValue::kBool;
      v->boolean = true;
      ok = true;
    } else if (literal("false")) {
      v->kind = JsonValue::kBool;
      ok = true;
    } else if (literal("null")) {
      ok = true;
    } else {
      const char* start = src.c_str() + pos;
      char* end = nullptr;
      v->number = std::strtod(start, &end);
      if (end != start) {
        v->kind = JsonValue::kNumber;
        pos += static_cast<size_t>(end - start);
        ok = std::isfinite(v->number);
      }
    }
    --depth;
    return ok;
  }
};

int variant_from_name(const std::string& name) {
  for (int v = 0; v < 12; ++v)
    if (name == variant_name(v)) return v;
  return -1;
}

bool json_int(const JsonValue& o, const char* key, int64_t lo, int64_t hi, int64_t* out) {
  const JsonValue* v = o.get(key);
  if (!v || v->kind != JsonValue::kNumber || v->number != std::floor(v->number) || v->number < static_cast<double>(lo) ||
      v->number > static_cast<double>(hi))
    return false;
  *out = static_cast<int64_t>(v->number);
  return true;
}

cn_status device_identity(int dev, std::string* name, std::string* arch, int* sms) {
  cudaDeviceProp prop{};
  const cudaError_t e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return fail_cuda(e, "cudaGetDeviceProperties");
  *name = prop.name;
  *arch = "sm_" + std::to_string(prop.major) + std::to_string(prop.minor);
  *sms = prop.multiProcessorCount;
  return CN_OK;
}

}  // namespace

namespace cn {
// cn_force on a workspace the caller supplies, without touching the
// library-owned workspaces (used by the static-scratch entry point).
cn_status force_f32_on_workspace(int64_t n_i, const float* pos_i, int64_t n_j, const float* pos_mass_j, float eps2,
                                 float* acc_out, float* pot_out, void* ws, size_t ws_bytes, cudaStream_t s) {
  return force_common(false, n_i, pos_i, n_j, pos_mass_j, eps2, acc_out, pot_out, ws, ws_bytes, false, s);
}
cn_status set_error(cn_status st, const std::string& msg) { return fail(st, msg); }

cn_status fail_nothrow(cn_status st, const char* msg) noexcept {
  try {
    g_last_error = msg;
  } catch (...) {
    g_last_error.clear();  // no room even for the message
  }
  return st;
}
}  // namespace cn

// ====================================================================== C ABI
extern "C" {

cn_status cn_force(int64_t n_i, const float* pos_i, int64_t n_j, const float* pos_mass_j, float eps2, float* acc_out,
                   float* pot_out, cn_stream stream) {
  NvtxRange nvtx_range("cn_force");
  return cn::guard([&]() -> cn_status {
    return force_common(false, n_i, pos_i, n_j, pos_mass_j, eps2, acc_out, pot_out, nullptr, 0, true,
                        reinterpret_cast<cudaStream_t>(stream));
  });
}

cn_status cn_force_eps_i(int64_t n_i, const float* pos_eps_i, int64_t n_j, const float* pos_mass_j, float* acc_out,
                         float* pot_out, cn_stream stream) {
  NvtxRange nvtx_range("cn_force_eps_i");
  return cn::guard([&]() -> cn_status {
    return force_common(false, n_i, pos_eps_i, n_j, pos_mass_j, 0.f, acc_out, pot_out, nullptr, 0, true,
                        reinterpret_cast<cudaStream_t>(stream), true);
  });
}

cn_status cn_force_ws(int64_t n_i, const float* pos_i, int64_t n_j, const float* pos_mass_j, float eps2,
                      float* acc_out, float* pot_out, void* workspace, size_t ws_bytes, cn_stream stream) {
  NvtxRange nvtx_range("cn_force_ws");
  return cn::guard([&]() -> cn_status {
    return force_common(false, n_i, pos_i, n_j, pos_mass_j, eps2, acc_out, pot_out, workspace, ws_bytes, false,
                        reinterpret_cast<cudaStream_t>(stream));
  });
}

cn_status cn_force_dd(int64_t n_i, const float* pos_i, int64_t n_j, const float* pos_mass_j, float eps2,
                      double* acc_out, double* pot_out, cn_stream stream) {
  NvtxRange nvtx_range("cn_force_dd");
  return cn::guard([&]() -> cn_status {
    return force_common(true, n_i, pos_i, n_j, pos_mass_j, eps2, acc_out, pot_out, nullptr, 0, true,
                        reinterpret_cast<cudaStream_t>(stream));
  });
}

cn_status cn_force_dd_ws(int64_t n_i, const float* pos_i, int64_t n_j, const float* pos_mass_j, float eps2,
                         double* acc_out, double* pot_out, void* workspace, size_t ws_bytes, cn_stream stream) {
  NvtxRange nvtx_range("cn_force_dd_ws");
  return cn::guard([&]() -> cn_status {
    return force_common(true, n_i, pos_i, n_j, pos_mass_j, eps2, acc_out, pot_out, workspace, ws_bytes, false,
                        reinterpret_cast<cudaStream_t>(stream));
  });
}

size_t cn_workspace_bytes(int variant, int64_t n_i, int64_t n_j) {
  return cn::guard_value<size_t>(0, [&]() -> size_t {
    if (n_i <= 0 || n_j <= 0 || variant < cn::kF32 || variant > cn::kF32EpsIPot || variant == cn::kBatched ||
        variant == cn::kBatchedPot || variant == cn::kSym)
      return 0;
    int dev = 0;
    DeviceInfo* d = nullptr;
    if (current_device(&dev, &d) != CN_OK) return 0;
    Plan p;
    if (resolve_plan(dev, variant, n_i, n_j, false, nullptr, &p) != CN_OK) return 0;
    Geometry g;
    if (single_geometry(dev, *d, variant, false, p, n_i, n_j, &g) != CN_OK) return 0;
    // the guarded (eps2 = 0) shape uses one i-particle per thread: size for the larger of the two
    Plan pg = p;
    pg.k = 1;
    Geometry gg;
    if (single_geometry(dev, *d, variant, true, pg, n_i, n_j, &gg) != CN_OK) return g.ws_bytes;
    return std::max(g.ws_bytes, gg.ws_bytes);
  });
}

cn_status cn_batch_plan_create(int32_t n_clusters, const int64_t* offsets_host, const float* eps2_host,
                               const cn_tune* tune, int with_potential, cn_batch_plan** plan_out) {
  NvtxRange nvtx_range("cn_batch_plan_create");
  return cn::guard([&]() -> cn_status {
    return build_batch_plan(n_clusters, offsets_host, eps2_host, tune, with_potential, plan_out);
  });
}

cn_status cn_batch_plan_destroy(cn_batch_plan* plan) {
  return cn::guard([&]() -> cn_status {
    if (!plan) return CN_OK;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->d_tiles) cudaFree(plan->d_tiles);
    if (plan->d_index) cudaFree(plan->d_index);
    delete plan;
    return CN_OK;
  });
}

size_t cn_batch_plan_workspace_bytes(const cn_batch_plan* plan) { return plan ? plan->ws_bytes : 0; }

cn_status cn_batch_plan_info(const cn_batch_plan* plan, int64_t* n_total, double* pairs) {
  return cn::guard([&]() -> cn_status {
    if (!plan) return fail(CN_ERR_INVALID_ARG, "plan is NULL");
    if (n_total) *n_total = plan->n_total;
    if (pairs) *pairs = plan->pairs;
    return CN_OK;
  });
}

cn_status cn_force_batched(const cn_batch_plan* plan, const float* pos_mass, float* acc_out, float* pot_out,
                           void* workspace, size_t ws_bytes, cn_stream stream) {
  NvtxRange nvtx_range("cn_force_batched");
  return cn::guard([&]() -> cn_status {
    if (plan && plan->lists) return fail(CN_ERR_INVALID_ARG, "an interaction-list plan runs with cn_force_lists");
    return run_batched(plan, pos_mass, pos_mass, acc_out, pot_out, workspace, ws_bytes,
                       reinterpret_cast<cudaStream_t>(stream));
  });
}

cn_status cn_list_plan_create(int32_t n_groups, const int64_t* i_offsets_host, const int64_t* j_begin_host,
                              const int64_t* j_count_host, const float* eps2_host, const cn_tune* tune,
                              int with_potential, cn_batch_plan** plan_out) {
  NvtxRange nvtx_range("cn_list_plan_create");
  return cn::guard([&]() -> cn_status {
    return build_list_plan(n_groups, i_offsets_host, j_begin_host, j_count_host, eps2_host, tune, with_potential,
                           plan_out);
  });
}

cn_status cn_list_plan_create_indexed(int32_t n_groups, const int64_t* i_offsets_host, const int64_t* j_begin_host,
                                      const int64_t* j_count_host, const float* eps2_host,
                                      const int32_t* j_index_host, int64_t n_index, int64_t n_src,
                                      const cn_tune* tune, int with_potential, cn_batch_plan** plan_out) {
  NvtxRange nvtx_range("cn_list_plan_create_indexed");
  return cn::guard([&]() -> cn_status {
    return build_list_plan_indexed(n_groups, i_offsets_host, j_begin_host, j_count_host, eps2_host, j_index_host,
                                   n_index, n_src, tune, with_potential, plan_out);
  });
}

cn_status cn_force_lists(const cn_batch_plan* plan, const float* pos_i, const float* pos_mass_j, float* acc_out,
                         float* pot_out, void* workspace, size_t ws_bytes, cn_stream stream) {
  NvtxRange nvtx_range("cn_force_lists");
  return cn::guard([&]() -> cn_status {
    if (plan && !plan->lists) return fail(CN_ERR_INVALID_ARG, "a cluster plan runs with cn_force_batched");
    return run_batched(plan, pos_i, pos_mass_j, acc_out, pot_out, workspace, ws_bytes,
                       reinterpret_cast<cudaStream_t>(stream));
  });
}

cn_status capture_plan(cn_batch_plan* plan, const float* pos_i, const float* pos_j, float* acc_out, float* pot_out,
                       void* workspace, size_t ws_bytes, cn_stream stream) {
  if (!plan) return fail(CN_ERR_INVALID_ARG, "plan is NULL");
  auto s = reinterpret_cast<cudaStream_t>(stream);
  if (!s) return fail(CN_ERR_INVALID_ARG, "graph capture needs a non-default stream");
  if (!workspace && plan->ws_bytes) return fail(CN_ERR_WORKSPACE, "graph capture needs a caller workspace");
  if (inject("capture")) return fail(CN_ERR_CUDA, "cudaStreamBeginCapture: injected capture failure");
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail_cuda(e, "cudaStreamBeginCapture");
  cn_status st = run_batched(plan, pos_i, pos_j, acc_out, pot_out, workspace, ws_bytes, s);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(s, &graph);
  if (st != CN_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail_cuda(e, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail_cuda(e, "cudaGraphInstantiate");
  }
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  plan->graph = graph;
  plan->exec = exec;
  return CN_OK;
}

cn_status cn_batch_plan_capture(cn_batch_plan* plan, const float* pos_mass, float* acc_out, float* pot_out,
                                void* workspace, size_t ws_bytes, cn_stream stream) {
  NvtxRange nvtx_range("cn_batch_plan_capture");
  return cn::guard([&]() -> cn_status {
    if (plan && plan->lists) return fail(CN_ERR_INVALID_ARG, "an interaction-list plan is captured with cn_list_plan_capture");
    return capture_plan(plan, pos_mass, pos_mass, acc_out, pot_out, workspace, ws_bytes, stream);
  });
}

cn_status cn_list_plan_capture(cn_batch_plan* plan, const float* pos_i, const float* pos_mass_j, float* acc_out,
                               float* pot_out, void* workspace, size_t ws_bytes, cn_stream stream) {
  NvtxRange nvtx_range("cn_list_plan_capture");
  return cn::guard([&]() -> cn_status {
    if (plan && !plan->lists) return fail(CN_ERR_INVALID_ARG, "a cluster plan is captured with cn_batch_plan_capture");
    return capture_plan(plan, pos_i, pos_mass_j, acc_out, pot_out, workspace, ws_bytes, stream);
  });
}

cn_status cn_batch_plan_launch(const cn_batch_plan* plan, cn_stream stream) {
  NvtxRange nvtx_range("cn_batch_plan_launch");
  return cn::guard([&]() -> cn_status {
    if (!plan || !plan->exec) return fail(CN_ERR_INVALID_ARG, "plan has no captured graph");
    if (inject("launch")) return fail(CN_ERR_CUDA, "cudaGraphLaunch: injected launch failure");
    cudaError_t e = cudaGraphLaunch(plan->exec, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? CN_OK : fail_cuda(e, "cudaGraphLaunch");
  });
}

cn_status cn_force_adjoint(int64_t n, const float* pos_mass, float eps2, const float* w, float* grad_pos,
                           float* grad_mass, cn_stream stream) {
  NvtxRange nvtx_range("cn_force_adjoint");
  return cn::guard([&]() -> cn_status {
    auto s = reinterpret_cast<cudaStream_t>(stream);
    if (n < 0) return fail(CN_ERR_INVALID_ARG, "n must be >= 0");
    cn_status st;
    if ((st = check_eps2(eps2)) != CN_OK) return st;
    if ((st = check_records(pos_mass, n, "pos_mass")) != CN_OK) return st;
    if (n > 0 && (!w || !grad_pos || !grad_mass)) return fail(CN_ERR_INVALID_ARG, "w, grad_pos and grad_mass are required");
    if ((w && !aligned(w, 4)) || (grad_pos && !aligned(grad_pos, 4)) || (grad_mass && !aligned(grad_mass, 4)))
      return fail(CN_ERR_MISALIGNED, "w and the gradients must be 4-byte aligned");
    const size_t un = static_cast<size_t>(n);
    if (overlaps(grad_pos, un * 12, pos_mass, un * 16) || overlaps(grad_pos, un * 12, w, un * 12) ||
        overlaps(grad_mass, un * 4, pos_mass, un * 16) || overlaps(grad_mass, un * 4, w, un * 12) ||
        overlaps(grad_pos, un * 12, grad_mass, un * 4))
      return fail(CN_ERR_INVALID_ARG, "outputs overlap inputs or each other");
    if (n == 0) return CN_OK;
    int dev = 0;
    DeviceInfo* d = nullptr;
    if ((st = current_device(&dev, &d)) != CN_OK) return st;
    const bool guard = needs_guard(eps2);
    Plan p;
    if ((st = resolve_plan(dev, cn::kAdjoint, n, n, guard, nullptr, &p)) != CN_OK) return st;
    Geometry g;
    if ((st = single_geometry(dev, *d, cn::kAdjoint, guard, p, n, n, &g)) != CN_OK) return st;
    char *ctrl = nullptr, *data = nullptr;
    if ((st = library_workspace(s, g.ctrl_bytes, g.data_bytes, &ctrl, &data)) != CN_OK) return st;
    float4* wrec = reinterpret_cast<float4*>(data + g.off_wrec);
    if (inject("launch")) return fail(CN_ERR_CUDA, "kernel launch: injected launch failure");
    cudaError_t e = cn::launch_pack_w(w, wrec, n, s);
    if (e != cudaSuccess) return fail_cuda(e, "weight packing launch");
    PairArgs a = base_args(ctrl, data, g, p, d->status);
    a.pos_i = reinterpret_cast<const float4*>(pos_mass);
    a.pos_j = reinterpret_cast<const float4*>(pos_mass);
    a.pos_i2 = wrec;
    a.pos_j2 = wrec;
    a.acc_out = grad_pos;
    a.pot_out = grad_mass;
    a.n_i = n;
    a.n_j = n;
    a.eps2 = eps2;
    log_plan("cn_force_adjoint", cn::kAdjoint, n, n, guard, p, g, g.njt);
    e = cn::launch_adjoint(a, p, guard, g.grid, s);
    return e == cudaSuccess ? CN_OK : fail_cuda(e, "adjoint kernel launch");
  });
}

cn_status cn_force_jerk(int64_t n_i, const float* pos_i, const float* vel_i, int64_t n_j, const float* pos_mass_j,
                        const float* vel_j, float eps2, float* acc_out, float* jerk_out, float* pot_out,
                        cn_stream stream) {
  NvtxRange nvtx_range("cn_force_jerk");
  return cn::guard([&]() -> cn_status {
    return jerk_common(n_i, pos_i, vel_i, n_j, pos_mass_j, vel_j, eps2, acc_out, jerk_out, pot_out,
                       reinterpret_cast<cudaStream_t>(stream));
  });
}

cn_status cn_force_symmetric(int64_t n, const float* pos_mass, float eps2, float* acc_out, float* pot_out,
                             cn_stream stream) {
  NvtxRange nvtx_range("cn_force_symmetric");
  return cn::guard([&]() -> cn_status {
    return symmetric_common(n, pos_mass, eps2, acc_out, pot_out, reinterpret_cast<cudaStream_t>(stream));
  });
}

cn_status cn_potential_energy(int64_t n, const float* pos_mass, const float* pot, double* w_out, cn_stream stream) {
  NvtxRange nvtx_range("cn_potential_energy");
  return cn::guard([&]() -> cn_status {
    return energy_common(n, pos_mass, pot, nullptr, w_out, reinterpret_cast<cudaStream_t>(stream));
  });
}

cn_status cn_potential_energy_dd(int64_t n, const float* pos_mass, const double* pot, double* w_out,
                                 cn_stream stream) {
  NvtxRange nvtx_range("cn_potential_energy_dd");
  return cn::guard([&]() -> cn_status {
    return energy_common(n, pos_mass, nullptr, pot, w_out, reinterpret_cast<cudaStream_t>(stream));
  });
}

cn_status cn_force_host(int64_t n_i, const float* pos_i_host, int64_t n_j, const float* pos_mass_j_host, float eps2,
                        float* acc_host, float* pot_host, cn_stream stream) {
  NvtxRange nvtx_range("cn_force_host");
  return cn::guard([&]() -> cn_status {
    auto s = reinterpret_cast<cudaStream_t>(stream);
    if (n_i < 0 || n_j < 0) return fail(CN_ERR_INVALID_ARG, "n_i and n_j must be >= 0");
    if ((n_i > 0 && (!pos_i_host || !acc_host)) || (n_j > 0 && !pos_mass_j_host))
      return fail(CN_ERR_INVALID_ARG, "NULL host buffer");
    cn_status st = check_eps2(eps2);
    if (st != CN_OK) return st;
    if (n_i == 0) return CN_OK;
    int dev = 0;
    DeviceInfo* d = nullptr;
    if ((st = current_device(&dev, &d)) != CN_OK) return st;
    // i = j when the caller passes the same host array for both sets: copy it once
    const bool same = pos_i_host == pos_mass_j_host && n_i == n_j;
    const size_t bi = align_up(static_cast<size_t>(n_i) * 16, 256);
    const size_t bj = same ? 0 : align_up(static_cast<size_t>(n_j) * 16, 256);
    const size_t ba = align_up(static_cast<size_t>(n_i) * 12, 256);
    const size_t bp = pot_host ? align_up(static_cast<size_t>(n_i) * 4, 256) : 0;
    void* buf = nullptr;
    if ((st = stage_buffer(s, bi + bj + ba + bp, &buf)) != CN_OK) return st;
    char* base = static_cast<char*>(buf);
    float* d_pi = reinterpret_cast<float*>(base);
    float* d_pj = same ? d_pi : reinterpret_cast<float*>(base + bi);
    float* d_acc = reinterpret_cast<float*>(base + bi + bj);
    float* d_pot = pot_host ? reinterpret_cast<float*>(base + bi + bj + ba) : nullptr;
    cudaError_t e = cudaMemcpyAsync(d_pi, pos_i_host, static_cast<size_t>(n_i) * 16, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !same && n_j > 0)
      e = cudaMemcpyAsync(d_pj, pos_mass_j_host, static_cast<size_t>(n_j) * 16, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_cuda(e, "cudaMemcpyAsync(host to device)");
    if ((st = cn_force(n_i, d_pi, n_j, d_pj, eps2, d_acc, d_pot, stream)) != CN_OK) return st;
    e = cudaMemcpyAsync(acc_host, d_acc, static_cast<size_t>(n_i) * 12, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && pot_host)
      e = cudaMemcpyAsync(pot_host, d_pot, static_cast<size_t>(n_i) * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return fail_cuda(e, "cudaMemcpyAsync(device to host)");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail_cuda(e, "cudaStreamSynchronize");
    return CN_OK;
  });
}

cn_status cn_force_host_f64(const double* xj, const double* mj, const double* xi, double eps2, double* a, int ni,
                            int nj) {
  NvtxRange nvtx_range("cn_force_host_f64");
  return cn::guard([&]() -> cn_status {
    if (ni < 0 || nj < 0) return fail(CN_ERR_INVALID_ARG, "ni and nj must be >= 0");
    if ((ni > 0 && (!xi || !a)) || (nj > 0 && (!xj || !mj))) return fail(CN_ERR_INVALID_ARG, "NULL host array");
    if (!std::isfinite(eps2) || eps2 < 0.0) return fail(CN_ERR_INVALID_ARG, "eps2 must be finite and >= 0");
    if (ni == 0) return CN_OK;
    std::vector<float> pi(static_cast<size_t>(ni) * 4), pj(static_cast<size_t>(nj) * 4), acc(static_cast<size_t>(ni) * 3);
    for (int i = 0; i < ni; ++i) {
      for (int c = 0; c < 3; ++c) pi[4 * i + c] = static_cast<float>(xi[3 * i + c]);
      pi[4 * i + 3] = 0.f;
    }
    for (int j = 0; j < nj; ++j) {
      for (int c = 0; c < 3; ++c) pj[4 * j + c] = static_cast<float>(xj[3 * j + c]);
      pj[4 * j + 3] = static_cast<float>(mj[j]);
    }
    cn_status st = cn_force_host(ni, pi.data(), nj, nj ? pj.data() : nullptr, static_cast<float>(eps2), acc.data(),
                                 nullptr, nullptr);
    if (st != CN_OK) return st;
    for (size_t k = 0; k < acc.size(); ++k) a[k] = acc[k];
    return CN_OK;
  });
}

cn_status cn_tune_get(int variant, int64_t n_i, int64_t n_j, cn_tune* out) {
  return cn::guard([&]() -> cn_status {
    if (!out || variant < cn::kF32 || variant > cn::kF32EpsIPot || n_i < 0 || n_j < 0)
      return fail(CN_ERR_INVALID_ARG, "bad variant, size or NULL output");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
    Plan p;
    cn_status st = resolve_plan(dev, variant, n_i, n_j, false, nullptr, &p);
    if (st != CN_OK) return st;
    out->i_per_thread = p.k;
    out->threads = p.threads;
    out->j_tile = p.j_tile;
    out->stages = p.stages;
    out->ctas_per_sm = p.ctas_per_sm;
    out->chunk_units = static_cast<int32_t>(p.chunk_units);
    out->j_lanes = p.j_lanes;
    return CN_OK;
  });
}

cn_status cn_tune_set(int variant, int64_t n_i, int64_t n_j, const cn_tune* tune) {
  return cn::guard([&]() -> cn_status {
    if (variant < cn::kF32 || variant > cn::kF32EpsIPot || n_i < 0 || n_j < 0)
      return fail(CN_ERR_INVALID_ARG, "bad variant or size");
    if (tune) {
      cn_status st = check_tune(variant, *tune);
      if (st != CN_OK) return st;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_mu);
    const auto key = std::make_tuple(dev, variant, bucket(n_i), bucket(n_j));
    if (tune)
      g_tune[key] = *tune;
    else
      g_tune.erase(key);
    g_plan_gen.fetch_add(1, std::memory_order_acq_rel);
    return CN_OK;
  });
}

cn_status cn_tune_save(const char* path) {
  return cn::guard([&]() -> cn_status {
    if (!path) return fail(CN_ERR_INVALID_ARG, "path is NULL");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
    std::string name, arch;
    int sms = 0;
    cn_status st = device_identity(dev, &name, &arch, &sms);
    if (st != CN_OK) return st;
    std::string out = "{\"format\": \"cunbody-tune-1\", \"device\": \"";
    for (char c : name) {
      if (c == '"' || c == '\\') out.push_back('\\');
      out.push_back(c);
    }
    out += "\", \"arch\": \"" + arch + "\", \"sms\": " + std::to_string(sms) + ", \"entries\": [";
    {
      std::lock_guard<std::mutex> lock(g_mu);
      bool first = true;
      for (const auto& kv : g_tune) {
        if (std::get<0>(kv.first) != dev) continue;
        const cn_tune& t = kv.second;
        char line[512];
        std::snprintf(line, sizeof(line),
                      "%s\n  {\"variant\": \"%s\", \"n_i_class\": %d, \"n_j_class\": %d, \"i_per_thread\": %d, "
                      "\"threads\": %d, \"j_tile\": %d, \"stages\": %d, \"ctas_per_sm\": %d, \"chunk_units\": %d, "
                      "\"j_lanes\": %d}",
                      first ? "" : ",", variant_name(std::get<1>(kv.first)), std::get<2>(kv.first), std::get<3>(kv.first),
                      t.i_per_thread, t.threads, t.j_tile, t.stages, t.ctas_per_sm, t.chunk_units, t.j_lanes);
        out += line;
        first = false;
      }
    }
    out += "\n]}\n";
    FILE* f = std::fopen(path, "w");
    if (!f) return fail(CN_ERR_INVALID_ARG, std::string("cannot write ") + path);
    const bool ok = std::fwrite(out.data(), 1, out.size(), f) == out.size();
    if (std::fclose(f) != 0 || !ok) return fail(CN_ERR_INVALID_ARG, std::string("writing ") + path + " failed");
    return CN_OK;
  });
}

cn_status cn_tune_load(const char* path, int32_t* n_loaded) {
  return cn::guard([&]() -> cn_status {
    if (n_loaded) *n_loaded = 0;
    if (!path) return fail(CN_ERR_INVALID_ARG, "path is NULL");
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(CN_ERR_INVALID_ARG, std::string("cannot read ") + path);
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0 && text.size() < (static_cast<size_t>(1) << 24))
      text.append(buf, got);
    std::fclose(f);
    JsonValue root;
    JsonReader rd{text};
    if (!rd.value(&root) || root.kind != JsonValue::kObject) return fail(CN_ERR_INVALID_ARG, "tuning file: not a JSON object");
    rd.skip();
    if (rd.pos != text.size()) return fail(CN_ERR_INVALID_ARG, "tuning file: trailing characters");
    const JsonValue* fmt = root.get("format");
    const JsonValue* dname = root.get("device");
    const JsonValue* darch = root.get("arch");
    const JsonValue* entries = root.get("entries");
    int64_t file_sms = 0;
    if (!fmt || fmt->kind != JsonValue::kString || fmt->text != "cunbody-tune-1")
      return fail(CN_ERR_INVALID_ARG, "tuning file: unknown format");
    if (!dname || dname->kind != JsonValue::kString || !darch || darch->kind != JsonValue::kString ||
        !json_int(root, "sms", 1, 1 << 20, &file_sms) || !entries || entries->kind != JsonValue::kArray)
      return fail(CN_ERR_INVALID_ARG, "tuning file: device, arch, sms or entries missing");
    struct Entry {
      int variant, ci, cj;
      cn_tune t;
    };
    std::vector<Entry> parsed;
    for (const JsonValue& e : entries->items) {
      if (e.kind != JsonValue::kObject) return fail(CN_ERR_INVALID_ARG, "tuning file: an entry is not an object");
      const JsonValue* vn = e.get("variant");
      const int variant = (vn && vn->kind == JsonValue::kString) ? variant_from_name(vn->text) : -1;
      int64_t ci, cj, k, th, jt, stg, cps, ch, jl;
      if (variant < 0 || !json_int(e, "n_i_class", 0, 62, &ci) || !json_int(e, "n_j_class", 0, 62, &cj) ||
          !json_int(e, "i_per_thread", 0, 8, &k) || !json_int(e, "threads", 0, 1024, &th) ||
          !json_int(e, "j_tile", 0, 4096, &jt) || !json_int(e, "stages", 0, 8, &stg) ||
          !json_int(e, "ctas_per_sm", 0, 64, &cps) || !json_int(e, "chunk_units", 0, INT32_MAX, &ch) ||
          !json_int(e, "j_lanes", 0, 32, &jl))
        return fail(CN_ERR_INVALID_ARG, "tuning file: an entry has a missing or out-of-range field");
      Entry en{variant, static_cast<int>(ci), static_cast<int>(cj),
               cn_tune{static_cast<int32_t>(k), static_cast<int32_t>(th), static_cast<int32_t>(jt),
                       static_cast<int32_t>(stg), static_cast<int32_t>(cps), static_cast<int32_t>(ch),
                       static_cast<int32_t>(jl)}};
      const cn_status st = check_tune(variant, en.t);
      if (st != CN_OK) return st;
      parsed.push_back(en);
    }
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return fail_cuda(ce, "cudaGetDevice");
    std::string name, arch;
    int sms = 0;
    cn_status st = device_identity(dev, &name, &arch, &sms);
    if (st != CN_OK) return st;
    if (name != dname->text || arch != darch->text || sms != file_sms)
      return fail(CN_ERR_UNSUPPORTED_DEVICE, "tuning file was written on " + dname->text + " (" + darch->text + ", " +
                                                 std::to_string(file_sms) + " SMs), this device is " + name + " (" +
                                                 arch + ", " + std::to_string(sms) + " SMs)");
    {
      std::lock_guard<std::mutex> lock(g_mu);
      for (const Entry& en : parsed) g_tune[std::make_tuple(dev, en.variant, en.ci, en.cj)] = en.t;
      g_plan_gen.fetch_add(1, std::memory_order_acq_rel);
    }
    if (n_loaded) *n_loaded = static_cast<int32_t>(parsed.size());
    return CN_OK;
  });
}

cn_status cn_autotune(int variant, int64_t n_i, const float* pos_i, int64_t n_j, const float* pos_mass_j, float eps2,
                      void* acc_out, void* pot_out, int reps, cn_stream stream, cn_tune* best_out) {
  NvtxRange nvtx_range("cn_autotune");
  return cn::guard([&]() -> cn_status {
    if (variant < cn::kF32 || variant > cn::kDDPot) return fail(CN_ERR_INVALID_ARG, "cn_autotune covers the F32 and DD variants");
    if (n_i <= 0 || n_j <= 0) return fail(CN_ERR_INVALID_ARG, "autotuning needs n_i > 0 and n_j > 0");
    const bool dd = variant == cn::kDD || variant == cn::kDDPot;
    const bool pot = variant == cn::kF32Pot || variant == cn::kDDPot;
    if (pot && !pot_out) return fail(CN_ERR_INVALID_ARG, "the potential variants need pot_out");
    auto s = reinterpret_cast<cudaStream_t>(stream);
    if (reps < 1) reps = 1;
    const int ks[] = {1, 2, 4, 8};
    const int ths[] = {64, 128, 256};
    const int tiles[] = {128, 256, 512, 1024};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    cn_tune best{};
    cn_status result = CN_OK;
    std::vector<cn_tune> cands;
    {
      // the default shape of these sizes first (its j-tile fitted to the
      // schedule, which the grid below does not contain), so that the result
      // is never slower than the default by more than the timing noise
      int dev = 0;
      DeviceInfo* d = nullptr;
      cn_status st = current_device(&dev, &d);
      if (st != CN_OK) return st;
      cands.push_back(default_tune(variant, n_i, n_j, d->sms));
    }
    for (int k : ks) {
      if (!valid_k(variant, k)) continue;
      for (int th : ths) {
        if (static_cast<int64_t>(k) * th > 4 * std::max<int64_t>(n_i, 256)) continue;  // tile far larger than the i set
        for (int jt : tiles) {
          if (jt > 4 * std::max<int64_t>(n_j, 64)) continue;
          cands.push_back(cn_tune{k, th, jt, 4, 0, 0, 1});
        }
      }
    }
    if (!dd && n_i <= 16384) {  // split-j shapes for small systems
      for (int jl : {2, 4, 8, 16, 32}) {
        if (n_i * jl > 262144) continue;
        for (int th : {128, 256})
          for (int64_t jt : {static_cast<int64_t>(512), static_cast<int64_t>(2048), round_up(std::max<int64_t>(n_j, 1), 8 * jl),
                             static_cast<int64_t>(4096)}) {
            if (jt % (8 * jl) || jt > 4096 || jt < 8 * jl) continue;
            for (int k : {1, 2, 4, 8}) {  // i-particles per lane group (packed for K >= 2)
              if (static_cast<int64_t>(k) * th / jl > 4 * std::max<int64_t>(n_i, 64)) continue;
              cands.push_back(cn_tune{k, th, static_cast<int32_t>(jt), jt >= n_j ? 1 : 3, 0, 0, jl});
            }
          }
      }
    }
    // Candidates are timed as one CUDA graph of `reps` calls, so that the host
    // cost of a call does not hide the device time of small problems. Capture
    // needs a non-default stream: the legacy stream gets a private one.
    cudaStream_t ts = s;
    const bool own_stream = (s == nullptr);
    if (own_stream && cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return fail(CN_ERR_CUDA, "autotune: cudaStreamCreate failed");
    }
    auto call = [&]() {
      return force_common(dd, n_i, pos_i, n_j, pos_mass_j, eps2, acc_out, pot ? pot_out : nullptr, nullptr, 0, true,
                          ts);
    };
    for (const cn_tune& t : cands) {
      if (check_tune(variant, t) != CN_OK) continue;
      cn_tune_set(variant, n_i, n_j, &t);
      cn_status st = call();  // warm-up (and workspace growth)
      if (st == CN_ERR_INVALID_ARG) continue;  // shape does not fit
      if (st != CN_OK) {
        result = st;
        break;
      }
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      if (cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        result = fail(CN_ERR_CUDA, "autotune: cudaStreamBeginCapture failed");
        break;
      }
      for (int r = 0; r < reps && st == CN_OK; ++r) st = call();
      cudaError_t e = cudaStreamEndCapture(ts, &graph);
      if (st == CN_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      if (st == CN_OK && e == cudaSuccess) e = cudaGraphLaunch(exec, ts);  // warm
      if (st == CN_OK && e == cudaSuccess) e = cudaEventRecord(e0, ts);
      if (st == CN_OK && e == cudaSuccess) e = cudaGraphLaunch(exec, ts);
      if (st == CN_OK && e == cudaSuccess) e = cudaEventRecord(e1, ts);
      if (st == CN_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (st == CN_OK && e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      if (st != CN_OK) {
        result = st;
        break;
      }
      if (e != cudaSuccess) {
        result = fail_cuda(e, "autotune: timing a candidate");
        break;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
    if (own_stream) {
      cudaStreamSynchronize(ts);
      release_library_workspace(ts);
      cudaStreamDestroy(ts);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != CN_OK) {
      cn_tune_set(variant, n_i, n_j, nullptr);
      return result;
    }
    if (best_ms >= 1e30f) {
      cn_tune_set(variant, n_i, n_j, nullptr);
      return fail(CN_ERR_INVALID_ARG, "no candidate launch shape fits");
    }
    cn_tune_set(variant, n_i, n_j, &best);
    if (best_out) *best_out = best;
    return CN_OK;
  });
}

cn_status cn_autotune_batched(int32_t n_clusters, const int64_t* offsets_host, const float* eps2_host,
                              const float* pos_mass, float* acc_out, float* pot_out, int reps, cn_stream stream,
                              cn_tune* best_out) {
  NvtxRange nvtx_range("cn_autotune_batched");
  return cn::guard([&]() -> cn_status {
    if (n_clusters <= 0 || !offsets_host) return fail(CN_ERR_INVALID_ARG, "empty ensemble");
    auto s = reinterpret_cast<cudaStream_t>(stream);
    if (reps < 1) reps = 1;
    const int variant = pot_out ? cn::kBatchedPot : cn::kBatched;
    const int ks[] = {2, 4, 8};
    const int ths[] = {64, 128, 256};
    const int tiles[] = {128, 256, 512};
    const int chunks[] = {0, 8, 32};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    cn_tune best{};
    cn_status result = CN_OK;
    std::vector<cn_tune> cands;
    for (int k : ks)
      for (int th : ths)
        for (int jt : tiles)
          for (int ch : chunks) cands.push_back(cn_tune{k, th, jt, 4, 0, ch, 1});
    // split-j shapes: eight i-particles per lane group, small i-tiles
    for (int jl : {2, 4, 8})
      for (int jt : {256, 512})
        for (int ch : {0, 8}) cands.push_back(cn_tune{8, 256, jt, 4, 0, ch, jl});
    for (const cn_tune& t : cands) {
      if (result != CN_OK) break;
      cn_batch_plan* plan = nullptr;
      cn_status st = build_batch_plan(n_clusters, offsets_host, eps2_host, &t, pot_out != nullptr, &plan);
      if (st != CN_OK) {
        if (st == CN_ERR_INVALID_ARG) continue;
        result = st;
        break;
      }
      st = run_batched(plan, pos_mass, pos_mass, acc_out, pot_out, nullptr, 0, s);
      if (st == CN_OK) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; ++r) run_batched(plan, pos_mass, pos_mass, acc_out, pot_out, nullptr, 0, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) == cudaSuccess) {
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best_ms) {
            best_ms = ms;
            best = t;
          }
        } else {
          st = fail(CN_ERR_CUDA, "autotune: event synchronisation failed");
        }
      }
      cn_batch_plan_destroy(plan);
      if (st != CN_OK) result = st;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != CN_OK) return result;
    if (best_ms >= 1e30f) return fail(CN_ERR_INVALID_ARG, "no candidate launch shape fits");
    const int64_t n_total = offsets_host[n_clusters];
    cn_tune_set(variant, n_clusters, n_total, &best);
    if (best_out) *best_out = best;
    return CN_OK;
  });
}

cn_status cn_get_device_status(cn_stream stream) {
  NvtxRange nvtx_range("cn_get_device_status");
  return cn::guard([&]() -> cn_status {
    auto s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    DeviceInfo* d = nullptr;
    cn_status st = current_device(&dev, &d);
    if (st != CN_OK) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "cudaStreamSynchronize");
    int flag = 0;
    if ((e = cudaMemcpy(&flag, d->status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return fail_cuda(e, "reading the device status word");
    if (flag == 0) return CN_OK;
    const int zero = 0;
    cudaMemcpy(d->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    {
      // arrival counters may have been left mid-protocol: clear every library workspace of this device
      std::lock_guard<std::mutex> lock(g_mu);
      for (auto& kv : g_ws)
        if (kv.first.first == dev) {
          if (kv.second.ctrl) cudaMemset(kv.second.ctrl, 0, kv.second.ctrl_bytes);
          if (kv.second.aux) cudaMemset(kv.second.aux, 0, (cn::energy_workspace_doubles() + 1) * sizeof(double));
        }
    }
    cudaDeviceSynchronize();
    return fail(CN_ERR_TIMEOUT, "a kernel wait timed out (device status bits " + std::to_string(flag) + ")");
  });
}

cn_status cn_set_wait_limit_ns(uint64_t ns) {
  return cn::guard([&]() -> cn_status {
    g_wait_ns.store(ns ? ns : kDefaultWaitNs);
    return CN_OK;
  });
}

cn_status cn_debug_timeout_probe(cn_stream stream) {
  return cn::guard([&]() -> cn_status {
    int dev = 0;
    DeviceInfo* d = nullptr;
    cn_status st = current_device(&dev, &d);
    if (st != CN_OK) return st;
    cudaError_t e = cn::launch_timeout_probe(d->status, g_wait_ns.load(), reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? CN_OK : fail_cuda(e, "timeout probe launch");
  });
}

cn_status cn_probe_peaks(cn_stream stream, double* out5) {
  return cn::guard([&]() -> cn_status {
    if (!out5) return fail(CN_ERR_INVALID_ARG, "out is NULL");
    int dev = 0;
    DeviceInfo* d = nullptr;
    cn_status st = current_device(&dev, &d);
    if (st != CN_OK) return st;
    cudaError_t e = cn::run_probes(reinterpret_cast<cudaStream_t>(stream), out5);
    return e == cudaSuccess ? CN_OK : fail_cuda(e, "issue-rate probes");
  });
}

const char* cn_status_string(cn_status status) {
  switch (status) {
    case CN_OK: return "CN_OK";
    case CN_ERR_INVALID_ARG: return "CN_ERR_INVALID_ARG";
    case CN_ERR_MISALIGNED: return "CN_ERR_MISALIGNED";
    case CN_ERR_CUDA: return "CN_ERR_CUDA";
    case CN_ERR_TIMEOUT: return "CN_ERR_TIMEOUT";
    case CN_ERR_UNSUPPORTED_DEVICE: return "CN_ERR_UNSUPPORTED_DEVICE";
    case CN_ERR_WORKSPACE: return "CN_ERR_WORKSPACE";
    case CN_ERR_HOST: return "CN_ERR_HOST";
  }
  return "CN_ERR_UNKNOWN";
}

const char* cn_last_error_message(void) { return g_last_error.c_str(); }

const char* cn_version(void) { return "cunbody 0.1.0 (sm_103a)"; }

}  // extern "C"
