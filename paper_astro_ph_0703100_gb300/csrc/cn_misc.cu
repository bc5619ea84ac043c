// Auxiliary kernels: the device status word, the FP64 potential-energy
// reduction, the issue-rate probes and the timeout probe.
#include "cn_device.cuh"
#include "cn_kernels.h"

namespace cn {

// One status word per device (bits of the kStatus* enum), set by kernels
// whose bounded waits ran out; read and cleared by cn_get_device_status.
__device__ int g_device_status = 0;

cudaError_t device_status_address(int** p) {
  return cudaGetSymbolAddress(reinterpret_cast<void**>(p), g_device_status);
}

namespace {

constexpr int kEnergyBlocks = 128;
constexpr int kEnergyThreads = 256;

// W = 1/2 sum_i m_i phi_i in FP64: each block sums a contiguous range in a
// fixed order and a fixed-shape tree; the last block to finish adds the
// block sums in block order. Deterministic for a given n.
__global__ void __launch_bounds__(kEnergyThreads) energy_kernel(int64_t n, const float4* __restrict__ pm,
                                                                 const float* __restrict__ pot_f,
                                                                 const double* __restrict__ pot_d,
                                                                 double* partials, int* counter, double* w_out) {
  __shared__ double red[kEnergyThreads];
  __shared__ int last;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * per;
  const int64_t hi = lo + per < n ? lo + per : n;
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double phi = pot_f ? static_cast<double>(pot_f[i]) : pot_d[i];
    s += 0.5 * static_cast<double>(pm[i].w) * phi;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kEnergyThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = red[0];
    __threadfence();
    last = (atomicAdd(counter, 1) == static_cast<int>(gridDim.x) - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double tot = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) tot += __ldcg(partials + b);
    *w_out = tot;
    *counter = 0;
  }
}

// ---- issue-rate probes
constexpr int kProbeIters = 4096;

__global__ void probe_ffma_kernel(float* sink, float seed, unsigned long long* clk) {
  float a0 = seed + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  float a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  const float b = 0.999999f, c = 1e-7f;
  const unsigned long long c0 = clock64();
  const uint64_t t0 = global_ns();
#pragma unroll 16
  for (int it = 0; it < kProbeIters; ++it) {
    a0 = fmaf(a0, b, c); a1 = fmaf(a1, b, c); a2 = fmaf(a2, b, c); a3 = fmaf(a3, b, c);
    a4 = fmaf(a4, b, c); a5 = fmaf(a5, b, c); a6 = fmaf(a6, b, c); a7 = fmaf(a7, b, c);
  }
  const unsigned long long c1 = clock64();
  const uint64_t t1 = global_ns();
  const float r = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (r == 12345.678f) sink[threadIdx.x] = r;
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    clk[0] = c1 - c0;
    clk[1] = t1 - t0;
  }
}

__global__ void probe_mufu_kernel(float* sink, float seed) {
  float a0 = seed + 1 + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  float a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
#pragma unroll 16
  for (int it = 0; it < kProbeIters; ++it) {
    a0 = rsqrt_mufu(a0); a1 = rsqrt_mufu(a1); a2 = rsqrt_mufu(a2); a3 = rsqrt_mufu(a3);
    a4 = rsqrt_mufu(a4); a5 = rsqrt_mufu(a5); a6 = rsqrt_mufu(a6); a7 = rsqrt_mufu(a7);
  }
  const float r = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (r == 12345.678f) sink[threadIdx.x] = r;
}

// A register-only loop with the pair kernel's instruction mix: per pair
// 3 FADD, 3 FFMA, 1 MUFU, 3 FMUL, 3 FFMA; four independent i chains and
// three FADDs per iteration (four pairs) to move the j position.
__global__ void probe_pair_kernel(float* sink, float seed, float dj) {
  float xi[4], ax[4], ay[4], az[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    xi[k] = seed * (k + 1) + threadIdx.x * 1e-3f;
    ax[k] = ay[k] = az[k] = 0.f;
  }
  float jx = 0.5f, jy = -0.25f, jz = 0.125f;
  const float m = 1e-3f, eps2 = 1e-2f;
#pragma unroll 4
  for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float dx = jx - xi[k], dy = jy - xi[k], dz = jz - xi[k];
      const float s = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
      const float r = rsqrt_mufu(s);
      const float q = (m * r) * (r * r);
      ax[k] = fmaf(q, dx, ax[k]);
      ay[k] = fmaf(q, dy, ay[k]);
      az[k] = fmaf(q, dz, az[k]);
    }
    jx += dj;  // a moving j position, so no pair term is loop-invariant
    jy -= dj;
    jz += dj;
  }
  float r = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) r += ax[k] + ay[k] + az[k];
  if (r == 12345.678f) sink[threadIdx.x] = r;
}

__global__ void timeout_probe_kernel(int* status, uint64_t wait_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // nothing ever arrives on this barrier: the bounded wait must give up
    if (!mbar_wait(&bar, 0, wait_ns)) set_status(status, kStatusTimeoutFull);
    // complete the phase so that no thread is left waiting on it
    mbar_arrive(&bar);
  }
  __syncthreads();
}

}  // namespace

cudaError_t launch_energy(int64_t n, const float4* pos_mass, const float* pot_f, const double* pot_d,
                          double* partials, int* counter, double* w_out, cudaStream_t s) {
  energy_kernel<<<kEnergyBlocks, kEnergyThreads, 0, s>>>(n, pos_mass, pot_f, pot_d, partials, counter, w_out);
  return cudaGetLastError();
}
size_t energy_workspace_doubles() { return kEnergyBlocks; }

cudaError_t launch_timeout_probe(int* status, uint64_t wait_ns, cudaStream_t s) {
  timeout_probe_kernel<<<1, 32, 0, s>>>(status, wait_ns);
  return cudaGetLastError();
}

// Runs the three probes; out[0..4] as documented for cn_probe_peaks.
cudaError_t run_probes(cudaStream_t s, double* out) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  float* sink = nullptr;
  unsigned long long* clk = nullptr;
  e = cudaMalloc(&sink, 1024 * sizeof(float));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&clk, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaFree(sink);
    return e;
  }
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  const int threads = 256;
  const int blocks = sms * 8;
  const double lanes = static_cast<double>(threads) * blocks;
  float ms = 0.f;
  double best[3] = {0, 0, 0};
  unsigned long long hclk[2] = {0, 0};
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    cudaEventRecord(ev0, s);
    probe_ffma_kernel<<<blocks, threads, 0, s>>>(sink, 1.0f + rep, clk);
    cudaEventRecord(ev1, s);
    e = cudaEventSynchronize(ev1);
    cudaEventElapsedTime(&ms, ev0, ev1);
    best[0] = fmax(best[0], lanes * kProbeIters * 8 / (ms * 1e-3));
    cudaMemcpy(hclk, clk, sizeof(hclk), cudaMemcpyDeviceToHost);
    cudaEventRecord(ev0, s);
    probe_mufu_kernel<<<blocks, threads, 0, s>>>(sink, 2.0f + rep);
    cudaEventRecord(ev1, s);
    e = cudaEventSynchronize(ev1);
    cudaEventElapsedTime(&ms, ev0, ev1);
    best[1] = fmax(best[1], lanes * kProbeIters * 8 / (ms * 1e-3));
    cudaEventRecord(ev0, s);
    probe_pair_kernel<<<blocks, threads, 0, s>>>(sink, 3.0f + rep, 1e-6f);
    cudaEventRecord(ev1, s);
    e = cudaEventSynchronize(ev1);
    cudaEventElapsedTime(&ms, ev0, ev1);
    best[2] = fmax(best[2], lanes * kProbeIters * 4 / (ms * 1e-3));  // pairs per second
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  out[0] = best[0];
  out[1] = best[1];
  out[2] = best[2];
  out[3] = hclk[1] ? static_cast<double>(hclk[0]) * 1e3 / static_cast<double>(hclk[1]) : 0.0;
  out[4] = sms;
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  cudaFree(sink);
  cudaFree(clk);
  return e;
}

}  // namespace cn
