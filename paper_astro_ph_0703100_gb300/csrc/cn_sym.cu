// Symmetric (Newton's third law) evaluation for an i set equal to the j set:
// every unordered pair is evaluated once and its term is added to both
// particles. The paper's kernel evaluates every ordered pair; this form does
// about half the pair work.
//
// The particles are cut into square tiles of B = threads x K. A unit is a
// tile pair (I, J) with I <= J. For I < J the CTA holds tile I in registers
// (K particles per thread) and streams tile J through a shared-memory ring
// (bulk copies, mbarriers). Per j record each lane adds m_j r^-3 d to its K
// i-particles and collects -m_i r^-3 d over them; the collected j-side terms
// of a batch of 8 j records are summed across the warp by a reduce-scatter
// (each lane visits the batch in an order permuted by its lane bits, so
// every exchange reads a fixed register: 24 shuffles and 24 adds per batch)
// and each warp's sums go to its own shared-memory row; at the end of the
// unit the rows are added in warp order. Diagonal units (I = J) use the
// one-sided loop. A CTA adds the i-side (tile I) sums of its consecutive
// units of row I, by TwoSum, into one (hi, lo) slot pair per (CTA, row)
// segment in a small buffer that stays in L2; each off-diagonal unit writes
// its j-side sums to slot (J, I) of a
// [tiles][n_pad] float4 array. A second kernel adds, per particle and in
// FP64, the j-side slots in partner order and then the i-side segments of
// its row in CTA order - a deterministic result with no atomics on data. The
// j-side array grows as N^2 / (2B) (it stays in L2 up to N ~ 2^17 with 2048
// particle tiles); when it would be too large the rows of tiles are
// processed in bands, each band merged into FP64 running sums.
//
// The i-particles of a thread are held in pairs and the pair terms are
// evaluated with packed f32x2 instructions (two i-particles per 64-bit
// register pair; the rsqrt stays two MUFU operations): 8 packed FP32
// instructions and 2 MUFU per two unordered pairs. The two halves of a
// thread's j-side sum are added before the warp reduction.
#include "cn_device.cuh"
#include "cn_sym.h"

namespace cn {

__device__ __forceinline__ void sym_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

namespace {

constexpr int kSymBatch = 8;  // j records per reduce-scatter batch

// Unit u of the upper triangle (row-major: (0,0), (0,1), ..., (0,T-1), (1,1), ...).
__device__ __forceinline__ void unit_tiles(int64_t u, int32_t T, int32_t* I, int32_t* J) {
  // row I starts at I*T - I*(I-1)/2; find the last row start <= u
  int32_t lo = 0, hi = T - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    const int64_t start = static_cast<int64_t>(mid) * T - static_cast<int64_t>(mid) * (mid - 1) / 2;
    if (start <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int64_t start = static_cast<int64_t>(lo) * T - static_cast<int64_t>(lo) * (lo - 1) / 2;
  *I = lo;
  *J = lo + static_cast<int32_t>(u - start);
}

// Resident CTAs per SM the register budget is sized for, by block size:
// 64-thread blocks 8 (<= 128 registers), 128-thread blocks 3 (<= 170),
// 256-thread blocks 1. The shared-memory rows of the j-side sums grow with
// the tile, so larger blocks cannot hold more CTAs anyway.
constexpr int sym_min_blocks(int nt_max) { return nt_max <= 64 ? 8 : (nt_max <= 128 ? 3 : 1); }

// POT: the potential rides along as a fourth sum (each pair's -m r to both
// sides, skipping pairs whose separation is exactly zero); the warp
// reduce-scatter then runs over 32 values per lane and ends with every lane
// owning one (j record, component) sum.
template <int K, bool GUARD, int NTMAX, bool POT>
__global__ void __launch_bounds__(NTMAX, sym_min_blocks(NTMAX)) sym_kernel(const __grid_constant__ SymArgs a) {
  constexpr int NCJ = POT ? 4 : 3;  // sums per particle
  extern __shared__ __align__(128) unsigned char smem[];
  const int NT = blockDim.x;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int NW = NT >> 5;
  const int B = NT * K;          // particles per tile
  const int JS = a.sub_tile;     // j records per ring stage (divides B, multiple of 8)
  const int S = a.stages;
  const int subs = B / JS;       // ring stages per unit
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + S;
  volatile int* ctl = reinterpret_cast<volatile int*>(smem + 16 * S);  // [0] abort
  float4* ring = reinterpret_cast<float4*>(smem + 256);
  float* jrows = reinterpret_cast<float*>(ring + static_cast<size_t>(S) * JS);  // [NW][B][NCJ]

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NW);
    }
    ctl[0] = 0;
    mbar_init_fence();
  }
  __syncthreads();
  // only shared memory so far: global memory after the previous kernel ends.
  // No early grid_launch_dependents() here: the merge kernel's CTAs would
  // then be placed on the SMs beside this one and wait there, which cost
  // 1.1% at N = 131072; the implicit trigger at exit is enough.
  grid_dependency_wait();

  const int64_t U = a.units;
  const int64_t G = gridDim.x;
  const int64_t ub = a.unit_base + (static_cast<int64_t>(blockIdx.x) * U) / G;
  const int64_t ue = a.unit_base + (static_cast<int64_t>(blockIdx.x + 1) * U) / G;
  const uint32_t n_loads = static_cast<uint32_t>((ue - ub) * subs);
  const uint32_t D = S > 2 ? static_cast<uint32_t>(S - 2) : static_cast<uint32_t>(S - 1);
  uint32_t issued = 0, consumed = 0;
  // lane permutation of a batch: lane visits j = t ^ perm
  const int perm = (((lane >> 4) & 1) << 2) | (((lane >> 3) & 1) << 1) | ((lane >> 2) & 1);

  // i-particles in pairs (packed f32x2 arithmetic, as in the plain kernel's
  // packed form): negated coordinates and negated masses
  static_assert(K == 1 || K % 2 == 0, "K is 1 or even");
  constexpr int P = (K + 1) / 2;
  float2 nxi[P][3], nmi[P], acc[P][3], pacc[P];
  auto half = [](float2& v, int k) -> float& { return (k & 1) ? v.y : v.x; };
  int32_t cur_I = -1;
  for (int64_t u = ub; u < ue; ++u) {
    int32_t I, J;
    unit_tiles(u, a.n_tiles, &I, &J);
#ifdef CN_DEBUG_BOUNDS
    // debug build: the unit must lie in the launch's band of the triangle and
    // its segment slot inside the allocation; otherwise flag and stop
    if (I < a.row0 || J < I || J >= a.n_tiles ||
        static_cast<int64_t>(blockIdx.x) + (I - a.row0) >= a.n_seg) {
      set_status(a.status, kStatusBadSchedule);
      ctl[0] = 1;  // the exit below waits (bounded) for copies still in flight
      break;
    }
#endif
    const bool diag = (I == J);
    // the first unit of this CTA's segment of row I (a row starts with its
    // diagonal unit), where the segment's running sums start
    const bool seg_first = (u == ub) || diag;
    if (I != cur_I) {
#pragma unroll
      for (int p = 0; p < P; ++p)
#pragma unroll
        for (int c = 0; c < 3; ++c) nxi[p][c] = make_float2(0.f, 0.f);
#pragma unroll
      for (int p = 0; p < P; ++p) nmi[p] = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int64_t p = static_cast<int64_t>(I) * B + k * NT + tid;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p < a.n) v = __ldg(a.pos + p);
        half(nxi[k >> 1][0], k) = -v.x;
        half(nxi[k >> 1][1], k) = -v.y;
        half(nxi[k >> 1][2], k) = -v.z;
        half(nmi[k >> 1], k) = -v.w;
      }
      cur_I = I;
    }
#pragma unroll
    for (int p = 0; p < P; ++p) acc[p][0] = acc[p][1] = acc[p][2] = pacc[p] = make_float2(0.f, 0.f);
    // Every (warp, j record) entry of the rows is written once per unit; the
    // force-only form stores it, the form with the potential adds to a
    // zeroed row (storing measured 2.8% slower there)
    if (POT && !diag)
      for (int e = tid; e < NW * B * NCJ; e += NT) jrows[e] = 0.f;
    __syncthreads();
    for (int sub = 0; sub < subs; ++sub) {
      // ---- producer: keep D loads ahead (thread 0)
      if (tid == 0) {
        while (!ctl[0] && issued < n_loads && issued <= consumed + D) {
          const int slot = static_cast<int>(issued % S);
          if (issued >= static_cast<uint32_t>(S) &&
              !mbar_wait(&empty[slot], ((issued / S) - 1) & 1u, a.wait_ns)) {
            set_status(a.status, kStatusTimeoutEmpty);
            ctl[0] = 1;
            break;
          }
          const int64_t lu = ub + issued / subs;
          const int ls = static_cast<int>(issued % subs);
          int32_t LI, LJ;
          unit_tiles(lu, a.n_tiles, &LI, &LJ);
          const int64_t first = static_cast<int64_t>(LJ) * B + static_cast<int64_t>(ls) * JS;
          const int64_t left = a.n - first;
          const int cnt = static_cast<int>(left <= 0 ? 0 : (left < JS ? left : JS));
          float4* dst = ring + static_cast<size_t>(slot) * JS;
          for (int z = cnt; z < JS; ++z) dst[z] = make_float4(0.f, 0.f, 0.f, 0.f);
          sym_fence_proxy_async();
          mbar_arrive_expect_tx(&full[slot], static_cast<uint32_t>(cnt) * 16u);
          if (cnt > 0) bulk_copy_g2s(dst, a.pos + first, static_cast<uint32_t>(cnt) * 16u, &full[slot]);
          ++issued;
        }
      }
      // ---- consumer
      const int slot = static_cast<int>(consumed % S);
      bool live = !ctl[0];
      if (live && !mbar_wait(&full[slot], (consumed / S) & 1u, a.wait_ns)) {
        set_status(a.status, kStatusTimeoutFull);
        ctl[0] = 1;
        live = false;
      }
      live = __all_sync(0xffffffffu, live);
      if (live) {
        const float4* js = ring + static_cast<size_t>(slot) * JS;
        const float2 e2 = make_float2(a.eps2, a.eps2);
        if (diag) {
#pragma unroll 1
          for (int j = 0; j < JS; j += 8) {
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
              const float4 pj = js[j + jj];
              const float2 jx = make_float2(pj.x, pj.x), jy = make_float2(pj.y, pj.y);
              const float2 jz = make_float2(pj.z, pj.z), jm = make_float2(pj.w, pj.w);
              const float2 njm = make_float2(-pj.w, -pj.w);
#pragma unroll
              for (int p = 0; p < P; ++p) {
                const float2 dx = __fadd2_rn(jx, nxi[p][0]);
                const float2 dy = __fadd2_rn(jy, nxi[p][1]);
                const float2 dz = __fadd2_rn(jz, nxi[p][2]);
                float2 s, d2;
                if constexpr (POT) {
                  d2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                  s = __fadd2_rn(d2, e2);
                } else {
                  s = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
                }
                float2 r = make_float2(rsqrt_mufu(s.x), rsqrt_mufu(s.y));
                if constexpr (GUARD) {
                  r.x = (s.x > 0.f) ? r.x : 0.f;
                  r.y = (s.y > 0.f) ? r.y : 0.f;
                }
                if constexpr (K == 1) r.y = 0.f;  // the unused half of the pair
                const float2 q = __fmul2_rn(jm, __fmul2_rn(r, __fmul2_rn(r, r)));
                acc[p][0] = __ffma2_rn(q, dx, acc[p][0]);
                acc[p][1] = __ffma2_rn(q, dy, acc[p][1]);
                acc[p][2] = __ffma2_rn(q, dz, acc[p][2]);
                if constexpr (POT) {
                  const float2 rp = make_float2(d2.x != 0.f ? r.x : 0.f, d2.y != 0.f ? r.y : 0.f);
                  pacc[p] = __ffma2_rn(njm, rp, pacc[p]);
                }
              }
            }
          }
        } else {
          float* myrow = jrows + static_cast<size_t>(warp) * B * NCJ;
          const int jbase = sub * JS;
#pragma unroll 1
          for (int j = 0; j < JS; j += kSymBatch) {
            float c[kSymBatch][NCJ];
#pragma unroll
            for (int t = 0; t < kSymBatch; ++t) {
              const float4 pj = js[j + (t ^ perm)];
              const float2 jx = make_float2(pj.x, pj.x), jy = make_float2(pj.y, pj.y);
              const float2 jz = make_float2(pj.z, pj.z), jm = make_float2(pj.w, pj.w);
              const float2 njm = make_float2(-pj.w, -pj.w);
              float2 cx = make_float2(0.f, 0.f), cy = cx, cz = cx, cp = cx;
#pragma unroll
              for (int p = 0; p < P; ++p) {
                const float2 dx = __fadd2_rn(jx, nxi[p][0]);
                const float2 dy = __fadd2_rn(jy, nxi[p][1]);
                const float2 dz = __fadd2_rn(jz, nxi[p][2]);
                float2 s, d2;
                if constexpr (POT) {
                  d2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                  s = __fadd2_rn(d2, e2);
                } else {
                  s = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
                }
                float2 r = make_float2(rsqrt_mufu(s.x), rsqrt_mufu(s.y));
                if constexpr (GUARD) {
                  r.x = (s.x > 0.f) ? r.x : 0.f;
                  r.y = (s.y > 0.f) ? r.y : 0.f;
                }
                if constexpr (K == 1) r.y = 0.f;  // the unused half of the pair
                const float2 r3 = __fmul2_rn(r, __fmul2_rn(r, r));
                const float2 qi = __fmul2_rn(jm, r3);      // m_j r^-3 onto particle i
                const float2 qj = __fmul2_rn(nmi[p], r3);  // -m_i r^-3 onto particle j
                acc[p][0] = __ffma2_rn(qi, dx, acc[p][0]);
                acc[p][1] = __ffma2_rn(qi, dy, acc[p][1]);
                acc[p][2] = __ffma2_rn(qi, dz, acc[p][2]);
                cx = __ffma2_rn(qj, dx, cx);
                cy = __ffma2_rn(qj, dy, cy);
                cz = __ffma2_rn(qj, dz, cz);
                if constexpr (POT) {
                  const float2 rp = make_float2(d2.x != 0.f ? r.x : 0.f, d2.y != 0.f ? r.y : 0.f);
                  pacc[p] = __ffma2_rn(njm, rp, pacc[p]);  // -m_j r onto particle i
                  cp = __ffma2_rn(nmi[p], rp, cp);         // -m_i r onto particle j
                }
              }
              c[t][0] = cx.x + cx.y;
              c[t][1] = cy.x + cy.y;
              c[t][2] = cz.x + cz.y;
              if constexpr (POT) c[t][3] = cp.x + cp.y;
            }
            // reduce-scatter over the warp: after the three halving steps
            // lane l holds, in c[0], the sum over the 8 lanes that share
            // l & 3 for j = perm(l); two butterfly steps complete the sum
#pragma unroll
            for (int t = 0; t < 4; ++t)
#pragma unroll
              for (int d = 0; d < NCJ; ++d) c[t][d] += __shfl_xor_sync(0xffffffffu, c[t + 4][d], 16);
#pragma unroll
            for (int t = 0; t < 2; ++t)
#pragma unroll
              for (int d = 0; d < NCJ; ++d) c[t][d] += __shfl_xor_sync(0xffffffffu, c[t + 2][d], 8);
#pragma unroll
            for (int d = 0; d < NCJ; ++d) c[0][d] += __shfl_xor_sync(0xffffffffu, c[1][d], 4);
            if constexpr (POT) {
              // two more halving steps over the four components: lane bit 1
              // keeps components {0, 1} or {2, 3}, lane bit 0 one of those
              const int b1 = (lane >> 1) & 1, b0 = lane & 1;
              float v0 = b1 ? c[0][2] : c[0][0], v1 = b1 ? c[0][3] : c[0][1];
              const float o0 = b1 ? c[0][0] : c[0][2], o1 = b1 ? c[0][1] : c[0][3];
              v0 += __shfl_xor_sync(0xffffffffu, o0, 2);
              v1 += __shfl_xor_sync(0xffffffffu, o1, 2);
              float w = b0 ? v1 : v0;
              w += __shfl_xor_sync(0xffffffffu, b0 ? v0 : v1, 1);
              myrow[static_cast<size_t>(jbase + j + perm) * 4 + 2 * b1 + b0] += w;
            } else {
              // two halving steps over (x, y, z, 0): lane bits 1 and 0
              // select the component the lane ends with; the pad's lane
              // writes nothing
              const int b1 = (lane >> 1) & 1, b0 = lane & 1;
              float v0 = b1 ? c[0][2] : c[0][0], v1 = b1 ? 0.f : c[0][1];
              const float o0 = b1 ? c[0][0] : c[0][2], o1 = b1 ? c[0][1] : 0.f;
              v0 += __shfl_xor_sync(0xffffffffu, o0, 2);
              v1 += __shfl_xor_sync(0xffffffffu, o1, 2);
              float w = b0 ? v1 : v0;
              w += __shfl_xor_sync(0xffffffffu, b0 ? v0 : v1, 1);
              const int comp = 2 * b1 + b0;
              if (comp < 3) myrow[static_cast<size_t>(jbase + j + perm) * 3 + comp] = w;
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
      }
      ++consumed;
    }
    // ---- end of the unit: the unit's i-side sums are folded by TwoSum into
    // the segment's (hi, lo) running sums (each thread reads back only what
    // it wrote; the buffer is small and stays in L2); j-side sums to slot
    // (J, I)
    __syncthreads();
    {
      float4* __restrict__ seg_hi =
          a.slots_seg + (static_cast<size_t>(blockIdx.x) + static_cast<size_t>(I - a.row0)) * 2 * B;
      float4* __restrict__ seg_lo = seg_hi + B;
      // all loads first (one memory latency per unit), then the sums, then
      // the stores
      float4 h[K], l[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        h[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        l[k] = h[k];
        if (!seg_first) {
          h[k] = seg_hi[k * NT + tid];
          l[k] = seg_lo[k * NT + tid];
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float v[4] = {half(acc[k >> 1][0], k), half(acc[k >> 1][1], k), half(acc[k >> 1][2], k),
                            POT ? half(pacc[k >> 1], k) : 0.f};
        float e[4];
        two_sum(h[k].x, v[0], h[k].x, e[0]);
        two_sum(h[k].y, v[1], h[k].y, e[1]);
        two_sum(h[k].z, v[2], h[k].z, e[2]);
        two_sum(h[k].w, v[3], h[k].w, e[3]);
        l[k].x = __fadd_rn(l[k].x, e[0]);
        l[k].y = __fadd_rn(l[k].y, e[1]);
        l[k].z = __fadd_rn(l[k].z, e[2]);
        l[k].w = __fadd_rn(l[k].w, e[3]);
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        seg_hi[k * NT + tid] = h[k];
        seg_lo[k * NT + tid] = l[k];
      }
    }
    if (!diag) {
      for (int jl = tid; jl < B; jl += NT) {
        float sx = 0.f, sy = 0.f, sz = 0.f, sp = 0.f;
        for (int w = 0; w < NW; ++w) {
          const float* r = jrows + (static_cast<size_t>(w) * B + jl) * NCJ;
          sx += r[0];
          sy += r[1];
          sz += r[2];
          if constexpr (POT) sp += r[3];
        }
        const int64_t p = static_cast<int64_t>(J) * B + jl;
        a.slots_j[static_cast<size_t>(I - a.row0) * a.n_pad + p] = make_float4(sx, sy, sz, sp);
      }
    }
    __syncthreads();
  }
  if (tid == 0 && ctl[0]) {
    for (uint32_t c = issued > static_cast<uint32_t>(S) ? issued - S : 0u; c < issued; ++c) {
      if (!mbar_wait(&full[c % S], (c / S) & 1u, a.wait_ns)) {
        set_status(a.status, kStatusTimeoutDrain);
        break;
      }
    }
  }
}

// Per-particle merge of one band (see SymMerge): partners in ascending
// order, FP64 sums carried across bands.
// POT: the potential (slot word 3) is summed too; without it that word is
// skipped, since FP64 additions are the merge's slow part on this GPU.
template <bool POT>
__global__ void sym_merge_kernel(const SymMerge m) {
  grid_dependency_wait();  // the slots are complete once the symmetric kernel has ended
  grid_launch_dependents();
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= m.n) return;
  double sx = 0.0, sy = 0.0, sz = 0.0, sp = 0.0;
  if (!m.first) {
    sx = m.acc64[4 * p + 0];
    sy = m.acc64[4 * p + 1];
    sz = m.acc64[4 * p + 2];
    sp = m.acc64[4 * p + 3];
  }
  const int32_t P = static_cast<int32_t>(p / m.tile);
  // j-side: units (I, P) of the band with I < P
  const int32_t jend = P < m.row1 ? P : m.row1;
  for (int32_t q = m.row0; q < jend; ++q) {
    const float4 v = __ldcs(m.slots_j + static_cast<size_t>(q - m.row0) * m.n_pad + p);
    sx += v.x;
    sy += v.y;
    sz += v.z;
    if constexpr (POT) sp += v.w;
  }
  // i-side: the segments of row P (when it is one of the band's rows), in
  // CTA order: CTA c of the band launch holds units [c U / G, (c + 1) U / G)
  if (P >= m.row0 && P < m.row1) {
    const int64_t T = m.n_tiles;
    const int64_t r0 = static_cast<int64_t>(P) * T - static_cast<int64_t>(P) * (P - 1) / 2 - m.unit_base;
    const int64_t r1 = r0 + (T - P);  // one past the row's last unit
    const int64_t c0 = ((r0 + 1) * m.grid - 1) / m.units;
    const int64_t c1 = (r1 * m.grid - 1) / m.units;
    const int64_t pl = p - static_cast<int64_t>(P) * m.tile;
    for (int64_t c = c0; c <= c1; ++c) {
      const float4* seg = m.slots_seg + (static_cast<size_t>(c) + static_cast<size_t>(P - m.row0)) * 2 * m.tile;
      const float4 h = __ldcs(seg + pl);
      const float4 l = __ldcs(seg + m.tile + pl);
      sx += static_cast<double>(h.x) + static_cast<double>(l.x);
      sy += static_cast<double>(h.y) + static_cast<double>(l.y);
      sz += static_cast<double>(h.z) + static_cast<double>(l.z);
      if constexpr (POT) sp += static_cast<double>(h.w) + static_cast<double>(l.w);
    }
  }
  if (m.last) {
    m.acc_out[3 * p + 0] = static_cast<float>(sx);
    m.acc_out[3 * p + 1] = static_cast<float>(sy);
    m.acc_out[3 * p + 2] = static_cast<float>(sz);
    if constexpr (POT) m.pot_out[p] = static_cast<float>(sp);
  } else {
    m.acc64[4 * p + 0] = sx;
    m.acc64[4 * p + 1] = sy;
    m.acc64[4 * p + 2] = sz;
    m.acc64[4 * p + 3] = sp;
  }
}

template <int K, bool GUARD, bool POT>
const void* sym_fn(int threads) {
  if (threads <= 64) return reinterpret_cast<const void*>(&sym_kernel<K, GUARD, 64, POT>);
  if (threads <= 128) return reinterpret_cast<const void*>(&sym_kernel<K, GUARD, 128, POT>);
  return reinterpret_cast<const void*>(&sym_kernel<K, GUARD, 256, POT>);
}

template <bool POT>
const void* sym_select_pot(int k, bool guard, int threads) {
  if (threads > 256) return nullptr;
  if (guard) return k == 1 ? sym_fn<1, true, POT>(threads) : nullptr;
  switch (k) {
    case 1: return sym_fn<1, false, POT>(threads);
    case 2: return sym_fn<2, false, POT>(threads);
    case 4: return sym_fn<4, false, POT>(threads);
    case 8: return sym_fn<8, false, POT>(threads);
    default: return nullptr;
  }
}

const void* sym_select(int k, bool guard, int threads, bool pot) {
  return pot ? sym_select_pot<true>(k, guard, threads) : sym_select_pot<false>(k, guard, threads);
}

}  // namespace

size_t sym_smem_bytes(int threads, int k, int sub_tile, int stages, bool pot) {
  const size_t b = static_cast<size_t>(threads) * k;
  return 256 + static_cast<size_t>(stages) * sub_tile * 16 + (threads / 32) * b * (pot ? 4 : 3) * sizeof(float);
}

cudaError_t occupancy_sym(int k, bool guard, int threads, size_t smem, int* ctas, bool pot) {
  const void* f = sym_select(k, guard, threads, pot);
  if (!f) return cudaErrorInvalidValue;
  cudaError_t e = prepare_kernel(f, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, f, threads, smem);
}

cudaError_t launch_sym(const SymArgs& a, const SymMerge& m, int k, bool guard, int threads, int grid, size_t smem,
                       cudaStream_t s, bool pot) {
  const void* f = sym_select(k, guard, threads, pot);
  if (!f) return cudaErrorInvalidValue;
  cudaError_t e = prepare_kernel(f, smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<SymArgs*>(&a)};
  e = launch_pdl(f, dim3(grid), dim3(threads), args, smem, s);
  if (e != cudaSuccess) return e;
  const int mt = 256;
  const int64_t mb = (m.n + mt - 1) / mt;
  void* margs[] = {const_cast<SymMerge*>(&m)};
  const void* mf = pot ? reinterpret_cast<const void*>(&sym_merge_kernel<true>)
                       : reinterpret_cast<const void*>(&sym_merge_kernel<false>);
  return launch_pdl(mf, dim3(static_cast<unsigned>(mb)), dim3(mt), margs, 0, s);
}

}  // namespace cn
