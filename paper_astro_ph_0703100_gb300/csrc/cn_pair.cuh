// The pair kernel: softened direct summation (Eq. 1) for a set of i-tiles
// against their j-particles, with the j-tiles staged through a ring of
// shared-memory stages by bulk copies (the J-BAG / J-PACKING of Section
// 2.2), several i-particles held in registers per thread (the I-POT), and a
// two-level accumulation in which each j-tile's partial sum is folded into
// a running sum (the FORCE-LOOP of Section 2.2.2, Eq. 2).
//
// Work decomposition: the i set is cut into i-tiles of threads x K
// particles and the j set of each i-tile's system into j-tiles of j_tile
// records. One (i-tile, j-tile) pair is a "unit"; units are numbered
// tile-major, so consecutive units share an i-tile. Each CTA processes
// contiguous unit ranges ("chunks"): either one chunk per CTA of equal size
// (static schedule, every SM gets the same number of pair interactions) or
// fixed-size chunks popped from an atomic queue (dynamic schedule). An
// i-tile whose units fall in one chunk is written directly; an i-tile split
// over several chunks has each chunk write its FP32 (or double-single)
// partial to the workspace, and the chunk that finishes last sums the
// partials in chunk order in FP64 - a deterministic cross-CTA reduction.
#pragma once

#include "cn_device.cuh"
#include "cn_kernels.h"

namespace cn {

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ------------------------------------------------------------------ schedule
struct Sched {
  int64_t U;  // total units
  int64_t Q;  // number of chunks
  int64_t C;  // dynamic chunk size, 0 for the static schedule
  __device__ __forceinline__ int64_t begin(int64_t q) const { return C ? q * C : (q * U) / Q; }
  __device__ __forceinline__ int64_t end(int64_t q) const {
    return C ? ((q + 1) * C < U ? (q + 1) * C : U) : ((q + 1) * U) / Q;
  }
  // chunk holding unit u: the largest q with begin(q) <= u
  __device__ __forceinline__ int64_t chunk_of(int64_t u) const { return C ? u / C : ((u + 1) * Q - 1) / U; }
};

template <bool BATCHED>
__device__ __forceinline__ TileDesc tile_at(const PairArgs& a, int32_t t, int i_tile) {
  if constexpr (BATCHED) {
    return a.tiles[t];
  } else {
    TileDesc d;
    d.i0 = static_cast<int64_t>(t) * i_tile;
    const int64_t left = a.n_i - d.i0;
    d.ni = static_cast<int32_t>(left < i_tile ? left : i_tile);
    d.j0 = 0;
    d.nj = a.n_j;
    d.njt = a.njt;
    d.unit0 = static_cast<int64_t>(t) * a.njt;
    d.eps2 = a.eps2;
    d.pad = 0;
    return d;
  }
}

template <bool BATCHED>
__device__ __forceinline__ int32_t tile_of_unit(const PairArgs& a, int64_t u) {
  if constexpr (BATCHED) {
    int32_t lo = 0, hi = a.n_tiles - 1;
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (a.tiles[mid].unit0 <= u)
        lo = mid;
      else
        hi = mid - 1;
    }
    return lo;
  } else {
    return static_cast<int32_t>(u / a.njt);
  }
}

// ------------------------------------------------------------------ pair math
// One j record against K i-particles in FP32: 3 FADD + 3 FFMA for the
// softened squared distance, one MUFU rsqrt, 3 FMUL for m r^-3 and 3 FFMA
// into the partial. POT adds the pair potential m / r for every pair whose
// separation is not exactly zero; GUARD zeroes pairs with s == 0 (reachable
// only for eps2 == 0 and coincident points). EPSI: i-particle k's own
// softening e2i[k] (the i record's 4th slot) replaces eps2.
template <int K, bool POT, bool GUARD, bool EPSI = false>
__device__ __forceinline__ void pair_f32(const float4 pj, const float (&xi)[K][3], float eps2,
                                         const float (&e2i)[EPSI ? K : 1], float (&part)[K][POT ? 4 : 3]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float dx = pj.x - xi[k][0];
    const float dy = pj.y - xi[k][1];
    const float dz = pj.z - xi[k][2];
    const float e2 = EPSI ? e2i[EPSI ? k : 0] : eps2;
    float s, d2 = 0.f;
    if constexpr (POT) {
      d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      s = d2 + e2;
    } else {
      s = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, e2)));
    }
    float r = rsqrt_mufu(s);
    if constexpr (GUARD) r = (s > 0.f) ? r : 0.f;
    const float mr = pj.w * r;
    const float q = mr * (r * r);
    part[k][0] = fmaf(q, dx, part[k][0]);
    part[k][1] = fmaf(q, dy, part[k][1]);
    part[k][2] = fmaf(q, dz, part[k][2]);
    if constexpr (POT) part[k][3] += (d2 != 0.f) ? mr : 0.f;
  }
}

// ------------------------------------------------------------------ policies
// The kernel below is generic over the interaction, in the way the paper's
// generalised library kernel (Section 4.5 and the appendix's pipeline
// descriptions) is generic over the widths of the i record, the j record
// and the result. A policy supplies:
//   kJRec          float4 words per j record (1: (x, y, z, m); 2: a
//                  velocity or a weight record follows)
//   kSlotF4        float4 words per i-particle in a split tile's partial
//   kSums          FP64 sums per i-particle in the merge (the result width)
//   kSplitJ        lanes of a group share the thread's i-particles (reduce_lanes)
//   kMinBlocks     256-thread CTAs per SM its register budget is sized for
//   load_i         i-particle k's record(s) into registers
//   zero, tile     clear the running sums; fold one staged j-tile into them
//   store_final    a whole i-tile's results to the outputs
//   store_partial  a split tile's partial to its workspace slot
//   add_partial    one loaded partial into the FP64 merge sums
//   store_merged   the merged sums to the outputs
// Gravity with or without the potential and with a per-particle softening
// (F32Policy, packed F32x2Policy), its compensated form (DDPolicy), the
// gradient of L = sum_i w_i . a_i (AdjointPolicy, AdjointX2Policy) and the
// force-jerk-potential pipeline (JerkPolicy, JerkX2Policy) all run through
// the one staging, scheduling and merging loop of pair_kernel.
//
// Plain FP32: per-tile FP32 partial folded into an FP32 running sum.
// SPLITJ: groups of j_lanes consecutive lanes share one i-particle, lane
// `sub` of a group taking j records sub, sub + j_lanes, ... of each tile;
// the group's sums are combined by a fixed xor butterfly of warp shuffles
// at the end of each segment (small systems: many threads, no cross-CTA
// merge). EPSI: each i-particle's softening is its record's 4th slot.
template <int K, bool POT, bool GUARD, bool SPLITJ = false, bool EPSI = false>
struct F32Policy {
  static constexpr int NC = POT ? 4 : 3;
  static constexpr int kSlotF4 = 1;  // float4 per i-particle in a workspace slot
  static constexpr int kSums = 4;    // FP64 sums in the split-tile merge
  static constexpr int kJRec = 1;    // float4 per j record
  static constexpr bool kSplitJ = SPLITJ;
  static constexpr int kMinBlocks = K >= 8 ? 1 : 2;  // 256-thread CTAs per SM the register budget must allow
  float xi[K][3];
  float e2i[EPSI ? K : 1];
  float run[K][NC];

  __device__ __forceinline__ void load_i(const PairArgs& a, int64_t gi, bool valid, int k) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) v = __ldg(a.pos_i + gi);
    xi[k][0] = v.x;
    xi[k][1] = v.y;
    xi[k][2] = v.z;
    if constexpr (EPSI) e2i[k] = v.w;
  }

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c) run[k][c] = 0.f;
  }

  __device__ __forceinline__ void tile(const float4* js, int T, float eps2, int64_t /*self_off*/, bool /*diag*/,
                                       int /*row*/, int /*rows*/, int sub, int jl) {
    float part[K][NC];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c) part[k][c] = 0.f;
    if constexpr (SPLITJ) {
      // this lane's j records: sub, sub + jl, ... (j_tile is a multiple of 8 jl)
#pragma unroll 1
      for (int j = sub; j < T; j += 8 * jl) {
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) pair_f32<K, POT, GUARD, EPSI>(js[j + jj * jl], xi, eps2, e2i, part);
      }
    } else {
      // 16 j records per loop trip (j_tile is a multiple of 16): enough
      // independent pair terms in flight to cover the MUFU and FMA latencies.
#pragma unroll 1
      for (int j = 0; j < T; j += 16) {
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) pair_f32<K, POT, GUARD, EPSI>(js[j + jj], xi, eps2, e2i, part);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c) run[k][c] += part[k][c];
  }

  // sums the running sums of the j_lanes lanes of each group (xor butterfly)
  __device__ __forceinline__ void reduce_lanes(int jl) {
    for (int off = jl >> 1; off > 0; off >>= 1) {
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) run[k][c] += __shfl_xor_sync(0xffffffffu, run[k][c], off);
    }
  }

  __device__ __forceinline__ void store_final(const PairArgs& a, int64_t i, int k) const {
    float* acc = static_cast<float*>(a.acc_out) + 3 * i;
    acc[0] = run[k][0];
    acc[1] = run[k][1];
    acc[2] = run[k][2];
    if constexpr (POT) {
      if (a.pot_out) static_cast<float*>(a.pot_out)[i] = -run[k][3];
    }
  }

  __device__ __forceinline__ void store_partial(float4* slot, int il, int /*i_tile*/, int k) const {
    slot[il] = make_float4(run[k][0], run[k][1], run[k][2], POT ? run[k][3] : 0.f);
  }

  // adds one loaded partial (its kSlotF4 float4 words) to the FP64 sums
  __device__ static __forceinline__ void add_partial(const float4 (&v)[kSlotF4], double (&s)[kSums]) {
    s[0] += v[0].x;
    s[1] += v[0].y;
    s[2] += v[0].z;
    s[3] += v[0].w;
  }

  __device__ static __forceinline__ void store_merged(const PairArgs& a, int64_t i, const double (&s)[kSums]) {
    float* acc = static_cast<float*>(a.acc_out) + 3 * i;
    acc[0] = static_cast<float>(s[0]);
    acc[1] = static_cast<float>(s[1]);
    acc[2] = static_cast<float>(s[2]);
    if constexpr (POT) {
      if (a.pot_out) static_cast<float*>(a.pot_out)[i] = static_cast<float>(-s[3]);
    }
  }
};

// Packed FP32 form of the same pair term: two i-particles per 64-bit
// register pair, every FP32 operation issued as one f32x2 instruction
// (add / mul / fma .rn.f32x2) and the rsqrt as two MUFU operations. Each
// lane-level operation, and the order of operations, is the scalar
// pair_f32's, so the results are bitwise the same; the warp instructions
// per pair drop from 12 FP32 + 1 MUFU to 6 packed + 1 MUFU (the broadcast j
// record feeds the packed instructions without extra moves: 7.18 measured
// per pair, LDS included), which leaves the FP32 pipe (12 lane operations
// per pair) as the bound instead of the issue slot. The i coordinates are
// held negated so that x_j - x_i is one packed add.
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

template <int K, bool POT, bool GUARD, bool EPSI = false>
__device__ __forceinline__ void pair_f32x2(const float4 pj, const float2 (&nxi)[K / 2][3], float2 e2u,
                                           const float2 (&e2i)[EPSI ? K / 2 : 1], float2 (&part)[K / 2][POT ? 4 : 3]) {
  const float2 jx = dup2(pj.x), jy = dup2(pj.y), jz = dup2(pj.z), jm = dup2(pj.w);
#pragma unroll
  for (int p = 0; p < K / 2; ++p) {
    const float2 e2 = EPSI ? e2i[EPSI ? p : 0] : e2u;
    const float2 dx = __fadd2_rn(jx, nxi[p][0]);
    const float2 dy = __fadd2_rn(jy, nxi[p][1]);
    const float2 dz = __fadd2_rn(jz, nxi[p][2]);
    float2 s, d2 = dup2(0.f);
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
    const float2 mr = __fmul2_rn(jm, r);
    const float2 q = __fmul2_rn(mr, __fmul2_rn(r, r));
    part[p][0] = __ffma2_rn(q, dx, part[p][0]);
    part[p][1] = __ffma2_rn(q, dy, part[p][1]);
    part[p][2] = __ffma2_rn(q, dz, part[p][2]);
    if constexpr (POT)
      part[p][3] = __fadd2_rn(part[p][3], make_float2(d2.x != 0.f ? mr.x : 0.f, d2.y != 0.f ? mr.y : 0.f));
  }
}

// Plain FP32 with packed arithmetic (K even): the F32Policy's results,
// two i-particles per register pair. SPLITJ: as in F32Policy, groups of
// j_lanes lanes share the thread's i-particles, each lane taking every
// j_lanes-th j record, combined by an xor butterfly at segment ends.
template <int K, bool POT, bool GUARD, bool SPLITJ = false, bool EPSI = false>
struct F32x2Policy {
  static_assert(K % 2 == 0, "the packed form holds i-particles in pairs");
  static constexpr int NC = POT ? 4 : 3;
  static constexpr int kSlotF4 = 1;
  static constexpr int kSums = 4;
  static constexpr int kJRec = 1;
  static constexpr bool kSplitJ = SPLITJ;
  // K = 4 (and the split-j form with the potential) spill under a 128-register cap
  static constexpr int kMinBlocks = (K >= 4 || SPLITJ) ? 1 : 2;
  float2 nxi[K / 2][3];
  float2 e2i[EPSI ? K / 2 : 1];  // per-particle softening (EPSI)
  float2 run[K / 2][NC];

  __device__ __forceinline__ static float& half(float2& v, int k) { return (k & 1) ? v.y : v.x; }
  __device__ __forceinline__ static float half(const float2& v, int k) { return (k & 1) ? v.y : v.x; }

  __device__ __forceinline__ void load_i(const PairArgs& a, int64_t gi, bool valid, int k) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) v = __ldg(a.pos_i + gi);
    half(nxi[k >> 1][0], k) = -v.x;
    half(nxi[k >> 1][1], k) = -v.y;
    half(nxi[k >> 1][2], k) = -v.z;
    if constexpr (EPSI) half(e2i[k >> 1], k) = v.w;
  }

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int p = 0; p < K / 2; ++p)
#pragma unroll
      for (int c = 0; c < NC; ++c) run[p][c] = dup2(0.f);
  }

  __device__ __forceinline__ void tile(const float4* js, int T, float eps2, int64_t /*self_off*/, bool /*diag*/,
                                       int /*row*/, int /*rows*/, int sub, int jl) {
    float2 part[K / 2][NC];
#pragma unroll
    for (int p = 0; p < K / 2; ++p)
#pragma unroll
      for (int c = 0; c < NC; ++c) part[p][c] = dup2(0.f);
    const float2 e2 = dup2(eps2);
    if constexpr (SPLITJ) {
      // this lane's j records: sub, sub + jl, ... (j_tile is a multiple of 8
      // jl). Lane groups of 8 with K = 8 (the mid-size and list shapes) take
      // a loop with the stride as a constant: 1-2% faster there (N = 32768:
      // 0.805 -> 0.818 of the FP32 bound), same results; specialising more
      // widths in one kernel measured slower
      if (K == 8 && jl == 8) {
#pragma unroll 1
        for (int j = sub; j < T; j += 64) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) pair_f32x2<K, POT, GUARD, EPSI>(js[j + jj * 8], nxi, e2, e2i, part);
        }
      } else {
#pragma unroll 1
        for (int j = sub; j < T; j += 8 * jl) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) pair_f32x2<K, POT, GUARD, EPSI>(js[j + jj * jl], nxi, e2, e2i, part);
        }
      }
    } else {
#pragma unroll 1
      for (int j = 0; j < T; j += 16) {
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) pair_f32x2<K, POT, GUARD, EPSI>(js[j + jj], nxi, e2, e2i, part);
      }
    }
#pragma unroll
    for (int p = 0; p < K / 2; ++p)
#pragma unroll
      for (int c = 0; c < NC; ++c) run[p][c] = __fadd2_rn(run[p][c], part[p][c]);
  }

  // sums the running sums of the j_lanes lanes of each group (xor butterfly)
  __device__ __forceinline__ void reduce_lanes(int jl) {
    for (int off = jl >> 1; off > 0; off >>= 1) {
#pragma unroll
      for (int p = 0; p < K / 2; ++p)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          run[p][c].x += __shfl_xor_sync(0xffffffffu, run[p][c].x, off);
          run[p][c].y += __shfl_xor_sync(0xffffffffu, run[p][c].y, off);
        }
    }
  }

  __device__ __forceinline__ void store_final(const PairArgs& a, int64_t i, int k) const {
    float* acc = static_cast<float*>(a.acc_out) + 3 * i;
    acc[0] = half(run[k >> 1][0], k);
    acc[1] = half(run[k >> 1][1], k);
    acc[2] = half(run[k >> 1][2], k);
    if constexpr (POT) {
      if (a.pot_out) static_cast<float*>(a.pot_out)[i] = -half(run[k >> 1][3], k);
    }
  }

  __device__ __forceinline__ void store_partial(float4* slot, int il, int /*i_tile*/, int k) const {
    slot[il] = make_float4(half(run[k >> 1][0], k), half(run[k >> 1][1], k), half(run[k >> 1][2], k),
                           POT ? half(run[k >> 1][NC - 1], k) : 0.f);
  }

  __device__ static __forceinline__ void add_partial(const float4 (&v)[kSlotF4], double (&s)[kSums]) {
    F32Policy<K, POT, GUARD>::add_partial(v, s);
  }

  __device__ static __forceinline__ void store_merged(const PairArgs& a, int64_t i, const double (&s)[kSums]) {
    F32Policy<K, POT, GUARD>::store_merged(a, i, s);
  }
};

// Compensated ("split-precision") form. The pair term is evaluated in FP32
// with its roundings recovered, and summed without loss:
//   d = x_j - x_i           fast two-sum taking x_j as the larger operand:
//                           exact whenever |x_j| >= |x_i| (and by Sterbenz
//                           whenever the two are within a factor of two),
//                           otherwise the low word is approximate
//   s = |d|^2 + eps2        exact squares (FMUL + FMA residual), the three
//                           non-negative additions as fast two-sums ordered
//                           by FMNMX, plus the cross term 2 d_hi . d_lo
//   y = s^-1/2              MUFU estimate y0 corrected to first order by the
//                           residual rho = 1 - s y0^2 (formed by FMAs)
//   q = m y^3               m y0 y0^2 with both product residuals, plus the
//                           correction 3/2 rho (relative)
//   a += q d                the product residual and the d_lo and q_lo
//                           terms go to the low word; the high word is added
//                           to the running sum by Knuth's TwoSum, its error
//                           to the low word
// Each j-tile's (hi, lo) sums are folded into FP64 running sums and
// restarted, which keeps the FP32 low word from accumulating rounding over
// long j ranges. 82 FP32 lane operations + 6 FMNMX + 1 MUFU per pair (the
// potential adds 10 FP32 and 3 selects). Measured against the FP64 oracle: E_max ~1e-9 on
// Plummer spheres; a CPU emulation of these operations bounds the four
// parity workloads at 1.6e-8 (the inexact d low word for |x_i| > |x_j| sets
// it; with an ordered two-sum for d as well the error is ~1e-13, 8% slower).
// Partials of split tiles carry the FP64 sums as (hi, lo) FP32 pairs and
// are merged in FP64; outputs are FP64.
//
// One term, for one i-particle: scalar (K = 1, the guarded kernel) and
// packed (two i-particles per f32x2 register pair) share this sequence of
// lane-level operations, so both give bitwise the same results.
struct DSTerm {
  // Knuth's TwoSum: s = a + b, e = the rounding error of s (exact)
  __device__ static __forceinline__ void ts(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bp = __fadd_rn(s, -a);
    const float ap = __fadd_rn(s, -bp);
    e = __fadd_rn(__fadd_rn(a, -ap), __fadd_rn(b, -bp));
  }
  // fast two-sum with a taken as the larger operand: e = b + (a - s)
  __device__ static __forceinline__ void fts(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fadd_rn(b, __fadd_rn(a, -s));
  }
  // the same for non-negative operands, ordered by max / min (exact)
  __device__ static __forceinline__ void ofs_pos(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fadd_rn(fminf(a, b), __fadd_rn(fmaxf(a, b), -s));
  }
};

template <bool POT, bool GUARD>
__device__ __forceinline__ void pair_ds1(const float4 pj, const float (&nxi)[3], float eps2, float (&hi)[POT ? 4 : 3],
                                         float (&lo)[POT ? 4 : 3]) {
  const float xj[3] = {pj.x, pj.y, pj.z};
  float dh[3], dl[3], ph[3], pl[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    DSTerm::fts(xj[c], nxi[c], dh[c], dl[c]);
    ph[c] = __fmul_rn(dh[c], dh[c]);
    pl[c] = __fmaf_rn(dh[c], dh[c], -ph[c]);
  }
  float t1, e1, t2, e2, sh, e3;
  DSTerm::ofs_pos(ph[0], ph[1], t1, e1);
  DSTerm::ofs_pos(t1, ph[2], t2, e2);
  DSTerm::ofs_pos(t2, eps2, sh, e3);
  const float cross = __fmaf_rn(dh[0], dl[0], __fmaf_rn(dh[1], dl[1], __fmul_rn(dh[2], dl[2])));
  float sl = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, __fadd_rn(__fadd_rn(pl[0], pl[1]), pl[2])));
  sl = __fmaf_rn(2.0f, cross, sl);
  float y0 = rsqrt_mufu(sh);
  if constexpr (GUARD) y0 = (sh > 0.f) ? y0 : 0.f;
  const float y2 = __fmul_rn(y0, y0);
  const float y2l = __fmaf_rn(y0, y0, -y2);
  float rho = __fmaf_rn(-sh, y2, 1.0f);
  rho = __fmaf_rn(-sh, y2l, rho);
  rho = __fmaf_rn(-sl, y2, rho);
  const float mr = __fmul_rn(pj.w, y0);
  const float mrl = __fmaf_rn(pj.w, y0, -mr);
  const float q = __fmul_rn(mr, y2);
  float t = __fmaf_rn(mr, y2, -q);
  t = __fmaf_rn(mr, y2l, t);
  t = __fmaf_rn(mrl, y2, t);
  t = __fmaf_rn(q, __fmul_rn(1.5f, rho), t);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float fh = __fmul_rn(q, dh[c]);
    const float r = __fmaf_rn(q, dh[c], -fh);
    float s, e;
    DSTerm::ts(hi[c], fh, s, e);
    hi[c] = s;
    float l = __fadd_rn(lo[c], e);
    l = __fadd_rn(l, r);
    l = __fmaf_rn(q, dl[c], l);
    lo[c] = __fmaf_rn(t, dh[c], l);
  }
  if constexpr (POT) {
    // m y0 (1 + rho / 2), skipped when the separation is exactly zero
    const bool apart = t2 != 0.f;
    const float uh = apart ? mr : 0.f;
    const float ul = apart ? __fmaf_rn(mr, __fmul_rn(0.5f, rho), mrl) : 0.f;
    float s, e;
    DSTerm::ts(hi[3], uh, s, e);
    hi[3] = s;
    lo[3] = __fadd_rn(__fadd_rn(lo[3], e), ul);
  }
}

// Packed: the same operations on two i-particles (the .x and .y halves);
// selects and compares stay per half. a - b is formed as fma(-1, b, a),
// which rounds exactly as the subtraction does.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(dup2(-1.0f), b, a); }
// a b - c per half, as two scalar FMAs: the packed FMA takes no negated
// operand, while the scalar one negates c for free (the FP32 pipe does the
// same lane work either way)
__device__ __forceinline__ float2 fms2(float2 a, float2 b, float2 c) {
  return make_float2(__fmaf_rn(a.x, b.x, -c.x), __fmaf_rn(a.y, b.y, -c.y));
}
// TwoSum and the fast two-sum (a taken as the larger operand), per half
__device__ __forceinline__ void ts2(float2 a, float2 b, float2& s, float2& e) {
  s = __fadd2_rn(a, b);
  const float2 bp = sub2(s, a);
  const float2 ap = sub2(s, bp);
  e = __fadd2_rn(sub2(a, ap), sub2(b, bp));
}
__device__ __forceinline__ void fts2(float2 a, float2 b, float2& s, float2& e) {
  s = __fadd2_rn(a, b);
  e = __fadd2_rn(b, sub2(a, s));
}
__device__ __forceinline__ void ofs_pos2(float2 a, float2 b, float2& s, float2& e) {
  s = __fadd2_rn(a, b);
  e = __fadd2_rn(make_float2(fminf(a.x, b.x), fminf(a.y, b.y)), sub2(make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)), s));
}

template <bool POT, bool GUARD>
__device__ __forceinline__ void pair_ds2(const float4 pj, const float2 (&nxi)[3], float2 e2,
                                         float2 (&hi)[POT ? 4 : 3], float2 (&lo)[POT ? 4 : 3]) {
  const float xj[3] = {pj.x, pj.y, pj.z};
  float2 dh[3], dl[3], ph[3], pl[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    fts2(dup2(xj[c]), nxi[c], dh[c], dl[c]);
    ph[c] = __fmul2_rn(dh[c], dh[c]);
    pl[c] = fms2(dh[c], dh[c], ph[c]);
  }
  float2 t1, e1, t2, ee2, sh, e3;
  ofs_pos2(ph[0], ph[1], t1, e1);
  ofs_pos2(t1, ph[2], t2, ee2);
  ofs_pos2(t2, e2, sh, e3);
  const float2 cross = __ffma2_rn(dh[0], dl[0], __ffma2_rn(dh[1], dl[1], __fmul2_rn(dh[2], dl[2])));
  float2 sl = __fadd2_rn(__fadd2_rn(e1, ee2), __fadd2_rn(e3, __fadd2_rn(__fadd2_rn(pl[0], pl[1]), pl[2])));
  sl = __ffma2_rn(dup2(2.0f), cross, sl);
  float2 y0 = make_float2(rsqrt_mufu(sh.x), rsqrt_mufu(sh.y));
  if constexpr (GUARD) {
    y0.x = (sh.x > 0.f) ? y0.x : 0.f;
    y0.y = (sh.y > 0.f) ? y0.y : 0.f;
  }
  const float2 y2 = __fmul2_rn(y0, y0);
  const float2 y2l = fms2(y0, y0, y2);
  // nrho = -rho = s y0^2 - 1, formed with positive operands only (the same
  // roundings as the scalar form's rho, negated)
  float2 nrho = __ffma2_rn(sh, y2, dup2(-1.0f));
  nrho = __ffma2_rn(sh, y2l, nrho);
  nrho = __ffma2_rn(sl, y2, nrho);
  const float2 m = dup2(pj.w);
  const float2 mr = __fmul2_rn(m, y0);
  const float2 mrl = fms2(m, y0, mr);
  const float2 q = __fmul2_rn(mr, y2);
  float2 t = fms2(mr, y2, q);
  t = __ffma2_rn(mr, y2l, t);
  t = __ffma2_rn(mrl, y2, t);
  t = __ffma2_rn(q, __fmul2_rn(dup2(-1.5f), nrho), t);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 fh = __fmul2_rn(q, dh[c]);
    const float2 r = fms2(q, dh[c], fh);
    float2 s, e;
    ts2(hi[c], fh, s, e);
    hi[c] = s;
    float2 l = __fadd2_rn(lo[c], e);
    l = __fadd2_rn(l, r);
    l = __ffma2_rn(q, dl[c], l);
    lo[c] = __ffma2_rn(t, dh[c], l);
  }
  if constexpr (POT) {
    const bool ax = t2.x != 0.f, ay = t2.y != 0.f;
    const float2 ulr = __ffma2_rn(mr, __fmul2_rn(dup2(-0.5f), nrho), mrl);
    const float2 uh = make_float2(ax ? mr.x : 0.f, ay ? mr.y : 0.f);
    const float2 ul = make_float2(ax ? ulr.x : 0.f, ay ? ulr.y : 0.f);
    float2 s, e;
    ts2(hi[3], uh, s, e);
    hi[3] = s;
    lo[3] = __fadd2_rn(__fadd2_rn(lo[3], e), ul);
  }
}

// Scalar compensated policy (K i-particles per thread, one per register;
// the guarded kernels use K = 1).
template <int K, bool POT, bool GUARD>
struct DDPolicy {
  static constexpr int NC = POT ? 4 : 3;
  static constexpr int kSlotF4 = 2;  // FP64 sums as (hi, lo) FP32 pairs: hi float4 then lo float4
  static constexpr int kSums = 4;
  static constexpr int kJRec = 1;
  static constexpr bool kSplitJ = false;
  static constexpr int kMinBlocks = K >= 2 ? 1 : 2;
  __device__ __forceinline__ void reduce_lanes(int) {}
  float nxi[K][3];
  double run[K][NC];

  __device__ __forceinline__ void load_i(const PairArgs& a, int64_t gi, bool valid, int k) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) v = __ldg(a.pos_i + gi);
    nxi[k][0] = -v.x;
    nxi[k][1] = -v.y;
    nxi[k][2] = -v.z;
  }

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c) run[k][c] = 0.0;
  }

  __device__ __forceinline__ void tile(const float4* js, int T, float eps2, int64_t /*self_off*/, bool /*diag*/,
                                       int /*row*/, int /*rows*/, int /*sub*/, int /*jl*/) {
    float hi[K][NC], lo[K][NC];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c) hi[k][c] = lo[k][c] = 0.f;
#pragma unroll 1
    for (int j = 0; j < T; j += 4) {
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const float4 pj = js[j + jj];
#pragma unroll
        for (int k = 0; k < K; ++k) pair_ds1<POT, GUARD>(pj, nxi[k], eps2, hi[k], lo[k]);
      }
    }
    // fold the tile's (hi, lo) sums into the FP64 running sums
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c) run[k][c] += static_cast<double>(hi[k][c]) + static_cast<double>(lo[k][c]);
  }

  __device__ __forceinline__ void store_final(const PairArgs& a, int64_t i, int k) const {
    double* acc = static_cast<double*>(a.acc_out) + 3 * i;
    acc[0] = run[k][0];
    acc[1] = run[k][1];
    acc[2] = run[k][2];
    if constexpr (POT) {
      if (a.pot_out) static_cast<double*>(a.pot_out)[i] = -run[k][3];
    }
  }

  // an FP64 sum as an unevaluated (hi, lo) FP32 pair (exact to about 2^-48)
  __device__ static __forceinline__ float2 split64(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - static_cast<double>(h)));
  }

  __device__ static __forceinline__ void store_split(float4* slot, int il, int i_tile, const double (&r)[NC]) {
    float2 s[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) s[c] = c < NC ? split64(r[c < NC ? c : 0]) : make_float2(0.f, 0.f);
    slot[il] = make_float4(s[0].x, s[1].x, s[2].x, s[3].x);
    slot[i_tile + il] = make_float4(s[0].y, s[1].y, s[2].y, s[3].y);
  }

  __device__ __forceinline__ void store_partial(float4* slot, int il, int i_tile, int k) const {
    store_split(slot, il, i_tile, run[k]);
  }

  __device__ static __forceinline__ void add_partial(const float4 (&v)[kSlotF4], double (&s)[kSums]) {
    const float4 h = v[0];
    const float4 l = v[1];
    s[0] += static_cast<double>(h.x) + static_cast<double>(l.x);
    s[1] += static_cast<double>(h.y) + static_cast<double>(l.y);
    s[2] += static_cast<double>(h.z) + static_cast<double>(l.z);
    s[3] += static_cast<double>(h.w) + static_cast<double>(l.w);
  }

  __device__ static __forceinline__ void store_merged(const PairArgs& a, int64_t i, const double (&s)[kSums]) {
    double* acc = static_cast<double*>(a.acc_out) + 3 * i;
    acc[0] = s[0];
    acc[1] = s[1];
    acc[2] = s[2];
    if constexpr (POT) {
      if (a.pot_out) static_cast<double*>(a.pot_out)[i] = -s[3];
    }
  }
};

// Packed compensated policy (K even): two i-particles per f32x2 register
// pair, bitwise the results of DDPolicy.
template <int K, bool POT, bool GUARD>
struct DDx2Policy {
  static_assert(K % 2 == 0, "the packed form holds i-particles in pairs");
  static constexpr int NC = POT ? 4 : 3;
  static constexpr int kSlotF4 = 2;
  static constexpr int kSums = 4;
  static constexpr int kJRec = 1;
  static constexpr bool kSplitJ = false;
  // No 128-register cap: K = 2 spilled 24 bytes under it; with 150
  // registers (three 128-thread CTAs per SM) it runs 2-8% faster at
  // N = 12000 .. 18000 (16384: 0.722 -> 0.755 of its bound)
  static constexpr int kMinBlocks = 1;
  __device__ __forceinline__ void reduce_lanes(int) {}
  float2 nxi[K / 2][3];
  double run[K][NC];

  __device__ __forceinline__ static float& half(float2& v, int k) { return (k & 1) ? v.y : v.x; }

  __device__ __forceinline__ void load_i(const PairArgs& a, int64_t gi, bool valid, int k) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) v = __ldg(a.pos_i + gi);
    half(nxi[k >> 1][0], k) = -v.x;
    half(nxi[k >> 1][1], k) = -v.y;
    half(nxi[k >> 1][2], k) = -v.z;
  }

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < NC; ++c) run[k][c] = 0.0;
  }

  __device__ __forceinline__ void tile(const float4* js, int T, float eps2, int64_t /*self_off*/, bool /*diag*/,
                                       int /*row*/, int /*rows*/, int /*sub*/, int /*jl*/) {
    float2 hi[K / 2][NC], lo[K / 2][NC];
#pragma unroll
    for (int p = 0; p < K / 2; ++p)
#pragma unroll
      for (int c = 0; c < NC; ++c) hi[p][c] = lo[p][c] = dup2(0.f);
    const float2 e2 = dup2(eps2);
#pragma unroll 1
    for (int j = 0; j < T; j += 4) {
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const float4 pj = js[j + jj];
#pragma unroll
        for (int p = 0; p < K / 2; ++p) pair_ds2<POT, GUARD>(pj, nxi[p], e2, hi[p], lo[p]);
      }
    }
#pragma unroll
    for (int p = 0; p < K / 2; ++p)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        run[2 * p][c] += static_cast<double>(hi[p][c].x) + static_cast<double>(lo[p][c].x);
        run[2 * p + 1][c] += static_cast<double>(hi[p][c].y) + static_cast<double>(lo[p][c].y);
      }
  }

  __device__ __forceinline__ void store_final(const PairArgs& a, int64_t i, int k) const {
    double* acc = static_cast<double*>(a.acc_out) + 3 * i;
    acc[0] = run[k][0];
    acc[1] = run[k][1];
    acc[2] = run[k][2];
    if constexpr (POT) {
      if (a.pot_out) static_cast<double*>(a.pot_out)[i] = -run[k][3];
    }
  }

  __device__ __forceinline__ void store_partial(float4* slot, int il, int i_tile, int k) const {
    DDPolicy<1, POT, GUARD>::store_split(slot, il, i_tile, run[k]);
  }

  __device__ static __forceinline__ void add_partial(const float4 (&v)[kSlotF4], double (&s)[kSums]) {
    DDPolicy<1, POT, GUARD>::add_partial(v, s);
  }

  __device__ static __forceinline__ void store_merged(const PairArgs& a, int64_t i, const double (&s)[kSums]) {
    DDPolicy<1, POT, GUARD>::store_merged(a, i, s);
  }
};

// Adjoint of L = sum_i w_i . a_i (i set = j set). Per pair, with
// d = x_p - x_k, s = |d|^2 + eps2, g = s^-3/2, h = s^-5/2 and
// u = m_k w_p - m_p w_k, the thread owning k adds g u - 3 h (d . u) d to
// dL/dx_k and -g (w_p . d) to dL/dm_k: 3 FADD + 3 FFMA + MUFU + 4 FMUL for
// s, g and 3h; 6 for u; 3 for d . u; 1 for 3h (d . u); 6 into dL/dx; 3 for
// w_p . d; 1 into dL/dm. The self pair is skipped exactly: units whose
// j-range overlaps the i-tile compare indices (the `diag` path).
template <int K, bool GUARD, bool SELF>
__device__ __forceinline__ void pair_adjoint(const float4 pj, const float4 wp, const float (&xk)[K][3],
                                             const float (&mk)[K], const float (&wk)[K][3], float eps2, int j,
                                             const int (&self_j)[K], float (&part)[K][4]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float dx = pj.x - xk[k][0];
    const float dy = pj.y - xk[k][1];
    const float dz = pj.z - xk[k][2];
    const float s = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    float r = rsqrt_mufu(s);
    if constexpr (GUARD) r = (s > 0.f) ? r : 0.f;
    if constexpr (SELF) r = (j == self_j[k]) ? 0.f : r;
    const float r2 = r * r;
    const float g = r2 * r;
    const float h3 = g * (3.0f * r2);
    const float ux = fmaf(mk[k], wp.x, -(pj.w * wk[k][0]));
    const float uy = fmaf(mk[k], wp.y, -(pj.w * wk[k][1]));
    const float uz = fmaf(mk[k], wp.z, -(pj.w * wk[k][2]));
    const float c = h3 * fmaf(dx, ux, fmaf(dy, uy, dz * uz));
    part[k][0] = fmaf(-c, dx, fmaf(g, ux, part[k][0]));
    part[k][1] = fmaf(-c, dy, fmaf(g, uy, part[k][1]));
    part[k][2] = fmaf(-c, dz, fmaf(g, uz, part[k][2]));
    part[k][3] = fmaf(-g, fmaf(wp.x, dx, fmaf(wp.y, dy, wp.z * dz)), part[k][3]);
  }
}

template <int K, bool GUARD>
struct AdjointPolicy {
  static constexpr int NC = 4;
  static constexpr int kSlotF4 = 1;
  static constexpr int kSums = 4;
  static constexpr int kJRec = 2;  // (x, y, z, m) then (wx, wy, wz, 0)
  static constexpr bool kSplitJ = false;
  static constexpr int kMinBlocks = K >= 4 ? 1 : 2;
  static constexpr int kBlock = 64;  // j entries summed in FP32 before the compensated fold
  __device__ __forceinline__ void reduce_lanes(int) {}
  float xk[K][3];
  float mk[K];
  float wk[K][3];
  // Running sums as (hi, lo) pairs: the adjoint's sums cancel heavily (the
  // weights are signed), so each block of kBlock terms is added to the
  // running sum by TwoSum instead of a rounded FP32 addition.
  float run[K][4];
  float runl[K][4];

  __device__ __forceinline__ void load_i(const PairArgs& a, int64_t gi, bool valid, int k) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
      v = __ldg(a.pos_i + gi);
      w = __ldg(a.pos_i2 + gi);
    }
    xk[k][0] = v.x;
    xk[k][1] = v.y;
    xk[k][2] = v.z;
    mk[k] = v.w;
    wk[k][0] = w.x;
    wk[k][1] = w.y;
    wk[k][2] = w.z;
  }

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < 4; ++c) run[k][c] = runl[k][c] = 0.f;
  }

  // self_off = (first j index of the tile) - (first i index of the i-tile)
  __device__ __forceinline__ void tile(const float4* js, int T, float eps2, int64_t self_off, bool diag, int row,
                                       int rows, int /*sub*/, int /*jl*/) {
    const float4* jw = js + T;
    int self_j[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      // the j slot (0 .. T-1) holding this thread's own particle, or -1
      const int64_t sj = static_cast<int64_t>(k * rows + row) - self_off;
      self_j[k] = (sj >= 0 && sj < T) ? static_cast<int>(sj) : -1;
    }
#pragma unroll 1
    for (int jb = 0; jb < T; jb += kBlock) {
      const int je = jb + kBlock < T ? jb + kBlock : T;
      float part[K][4];
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int c = 0; c < 4; ++c) part[k][c] = 0.f;
      if (!diag) {
#pragma unroll 1
        for (int j = jb; j < je; j += 8) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
            pair_adjoint<K, GUARD, false>(js[j + jj], jw[j + jj], xk, mk, wk, eps2, j + jj, self_j, part);
        }
      } else {
#pragma unroll 1
        for (int j = jb; j < je; j += 8) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
            pair_adjoint<K, GUARD, true>(js[j + jj], jw[j + jj], xk, mk, wk, eps2, j + jj, self_j, part);
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float s, e;
          two_sum(run[k][c], part[k][c], s, e);
          run[k][c] = s;
          runl[k][c] = __fadd_rn(runl[k][c], e);
        }
    }
  }

  __device__ __forceinline__ float total(int k, int c) const { return __fadd_rn(run[k][c], runl[k][c]); }

  __device__ __forceinline__ void store_final(const PairArgs& a, int64_t i, int k) const {
    float* g = static_cast<float*>(a.acc_out) + 3 * i;
    g[0] = total(k, 0);
    g[1] = total(k, 1);
    g[2] = total(k, 2);
    static_cast<float*>(a.pot_out)[i] = total(k, 3);
  }

  __device__ __forceinline__ void store_partial(float4* slot, int il, int /*i_tile*/, int k) const {
    slot[il] = make_float4(total(k, 0), total(k, 1), total(k, 2), total(k, 3));
  }

  __device__ static __forceinline__ void add_partial(const float4 (&v)[kSlotF4], double (&s)[kSums]) {
    s[0] += v[0].x;
    s[1] += v[0].y;
    s[2] += v[0].z;
    s[3] += v[0].w;
  }

  __device__ static __forceinline__ void store_merged(const PairArgs& a, int64_t i, const double (&s)[kSums]) {
    float* g = static_cast<float*>(a.acc_out) + 3 * i;
    g[0] = static_cast<float>(s[0]);
    g[1] = static_cast<float>(s[1]);
    g[2] = static_cast<float>(s[2]);
    static_cast<float*>(a.pot_out)[i] = static_cast<float>(s[3]);
  }
};

// Force, jerk and potential (the force-jerk-potential pipeline description
// of the appendix) for particles moving with velocities v. Per pair, with
// d = x_j - x_i, w = v_j - v_i, s = |d|^2 + eps2, r = s^-1/2 and q = m r^3:
//   a += q d;   jerk += q (w - b d) with b = 3 (d . w) r^2;   pot += m r
// (d a / dt for straight-line motion): 3 + 3 FADD, 3 FFMA, MUFU, 3 FMUL for
// r^2, m r, q, 3 for d . w, 2 for b, 1 for q b, 3 into a, 6 into the jerk:
// 27 FP32 issue slots + 1 MUFU (the potential adds 3).
template <int K, bool POT, bool GUARD>
__device__ __forceinline__ void pair_jerk(const float4 pj, const float4 vj, const float (&xi)[K][3],
                                          const float (&vi)[K][3], float eps2, float (&part)[K][7]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float dx = pj.x - xi[k][0];
    const float dy = pj.y - xi[k][1];
    const float dz = pj.z - xi[k][2];
    const float wx = vj.x - vi[k][0];
    const float wy = vj.y - vi[k][1];
    const float wz = vj.z - vi[k][2];
    float s, d2 = 0.f;
    if constexpr (POT) {
      d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      s = d2 + eps2;
    } else {
      s = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    }
    float r = rsqrt_mufu(s);
    if constexpr (GUARD) r = (s > 0.f) ? r : 0.f;
    const float r2 = r * r;
    const float mr = pj.w * r;
    const float q = mr * r2;
    const float b = (3.0f * r2) * fmaf(dx, wx, fmaf(dy, wy, dz * wz));
    const float qb = q * b;
    part[k][0] = fmaf(q, dx, part[k][0]);
    part[k][1] = fmaf(q, dy, part[k][1]);
    part[k][2] = fmaf(q, dz, part[k][2]);
    part[k][3] = fmaf(-qb, dx, fmaf(q, wx, part[k][3]));
    part[k][4] = fmaf(-qb, dy, fmaf(q, wy, part[k][4]));
    part[k][5] = fmaf(-qb, dz, fmaf(q, wz, part[k][5]));
    if constexpr (POT) part[k][6] += (d2 != 0.f) ? mr : 0.f;
  }
}

template <int K, bool POT, bool GUARD>
struct JerkPolicy {
  static constexpr int kSlotF4 = 2;  // (ax, ay, az, jx) then (jy, jz, pot, 0)
  static constexpr int kSums = 7;
  static constexpr int kJRec = 2;    // (x, y, z, m) then (vx, vy, vz, -)
  static constexpr bool kSplitJ = false;
  static constexpr int kMinBlocks = 1;  // 20 registers of state per i-particle
  __device__ __forceinline__ void reduce_lanes(int) {}
  float xi[K][3];
  float vi[K][3];
  float run[K][7];

  __device__ __forceinline__ void load_i(const PairArgs& a, int64_t gi, bool valid, int k) {
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
      p = __ldg(a.pos_i + gi);
      v = __ldg(a.pos_i2 + gi);
    }
    xi[k][0] = p.x;
    xi[k][1] = p.y;
    xi[k][2] = p.z;
    vi[k][0] = v.x;
    vi[k][1] = v.y;
    vi[k][2] = v.z;
  }

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < 7; ++c) run[k][c] = 0.f;
  }

  __device__ __forceinline__ void tile(const float4* js, int T, float eps2, int64_t /*self_off*/, bool /*diag*/,
                                       int /*row*/, int /*rows*/, int /*sub*/, int /*jl*/) {
    const float4* jv = js + T;
    float part[K][7];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < 7; ++c) part[k][c] = 0.f;
#pragma unroll 1
    for (int j = 0; j < T; j += 4) {
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) pair_jerk<K, POT, GUARD>(js[j + jj], jv[j + jj], xi, vi, eps2, part);
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < 7; ++c) run[k][c] += part[k][c];
  }

  __device__ __forceinline__ void store_final(const PairArgs& a, int64_t i, int k) const {
    float* acc = static_cast<float*>(a.acc_out) + 3 * i;
    float* jk = static_cast<float*>(a.jerk_out) + 3 * i;
    acc[0] = run[k][0];
    acc[1] = run[k][1];
    acc[2] = run[k][2];
    jk[0] = run[k][3];
    jk[1] = run[k][4];
    jk[2] = run[k][5];
    if constexpr (POT) {
      if (a.pot_out) static_cast<float*>(a.pot_out)[i] = -run[k][6];
    }
  }

  __device__ __forceinline__ void store_partial(float4* slot, int il, int i_tile, int k) const {
    slot[il] = make_float4(run[k][0], run[k][1], run[k][2], run[k][3]);
    slot[i_tile + il] = make_float4(run[k][4], run[k][5], run[k][6], 0.f);
  }

  __device__ static __forceinline__ void add_partial(const float4 (&v)[kSlotF4], double (&s)[kSums]) {
    s[0] += v[0].x;
    s[1] += v[0].y;
    s[2] += v[0].z;
    s[3] += v[0].w;
    s[4] += v[1].x;
    s[5] += v[1].y;
    s[6] += v[1].z;
  }

  __device__ static __forceinline__ void store_merged(const PairArgs& a, int64_t i, const double (&s)[kSums]) {
    float* acc = static_cast<float*>(a.acc_out) + 3 * i;
    float* jk = static_cast<float*>(a.jerk_out) + 3 * i;
    acc[0] = static_cast<float>(s[0]);
    acc[1] = static_cast<float>(s[1]);
    acc[2] = static_cast<float>(s[2]);
    jk[0] = static_cast<float>(s[3]);
    jk[1] = static_cast<float>(s[4]);
    jk[2] = static_cast<float>(s[5]);
    if constexpr (POT) {
      if (a.pot_out) static_cast<float*>(a.pot_out)[i] = static_cast<float>(-s[6]);
    }
  }
};

// ------------------------------------------------------------------ packed adjoint and jerk
// The adjoint and force-jerk pair terms with two i-particles per register
// pair (f32x2 issue), K even. Lane-level operations and their order are the
// scalar forms'; negated terms are formed exactly by negated operands (the
// i records are held negated, -3 instead of 3), and the adjoint's mass sum,
// a sum of -g (w_p . d) terms, is accumulated with the opposite sign and
// negated when stored (round-to-nearest commutes with negation), so the
// results are bitwise those of the scalar policies.
template <int K, bool GUARD, bool SELF>
__device__ __forceinline__ void pair_adjoint_x2(const float4 pj, const float4 wp, const float2 (&nxk)[K / 2][3],
                                                const float2 (&mk)[K / 2], const float2 (&nwk)[K / 2][3], float2 e2,
                                                int j, const int (&self_j)[K], float2 (&part)[K / 2][4]) {
  const float2 jx = dup2(pj.x), jy = dup2(pj.y), jz = dup2(pj.z), jm = dup2(pj.w);
  const float2 wx = dup2(wp.x), wy = dup2(wp.y), wz = dup2(wp.z), m3 = dup2(-3.0f);
#pragma unroll
  for (int p = 0; p < K / 2; ++p) {
    const float2 dx = __fadd2_rn(jx, nxk[p][0]);
    const float2 dy = __fadd2_rn(jy, nxk[p][1]);
    const float2 dz = __fadd2_rn(jz, nxk[p][2]);
    const float2 s = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
    float2 r = make_float2(rsqrt_mufu(s.x), rsqrt_mufu(s.y));
    if constexpr (GUARD) {
      r.x = (s.x > 0.f) ? r.x : 0.f;
      r.y = (s.y > 0.f) ? r.y : 0.f;
    }
    if constexpr (SELF) {
      r.x = (j == self_j[2 * p]) ? 0.f : r.x;
      r.y = (j == self_j[2 * p + 1]) ? 0.f : r.y;
    }
    const float2 r2 = __fmul2_rn(r, r);
    const float2 g = __fmul2_rn(r2, r);
    const float2 nh3 = __fmul2_rn(g, __fmul2_rn(m3, r2));  // -3 g r^2
    const float2 ux = __ffma2_rn(mk[p], wx, __fmul2_rn(jm, nwk[p][0]));
    const float2 uy = __ffma2_rn(mk[p], wy, __fmul2_rn(jm, nwk[p][1]));
    const float2 uz = __ffma2_rn(mk[p], wz, __fmul2_rn(jm, nwk[p][2]));
    const float2 nc = __fmul2_rn(nh3, __ffma2_rn(dx, ux, __ffma2_rn(dy, uy, __fmul2_rn(dz, uz))));
    part[p][0] = __ffma2_rn(nc, dx, __ffma2_rn(g, ux, part[p][0]));
    part[p][1] = __ffma2_rn(nc, dy, __ffma2_rn(g, uy, part[p][1]));
    part[p][2] = __ffma2_rn(nc, dz, __ffma2_rn(g, uz, part[p][2]));
    part[p][3] = __ffma2_rn(g, __ffma2_rn(wx, dx, __ffma2_rn(wy, dy, __fmul2_rn(wz, dz))), part[p][3]);
  }
}

// SPLITJ (small systems): lane groups share the thread's i-particles, each
// lane taking every j_lanes-th j entry (the self test compares the entry's
// index in the tile, so it is unchanged), combined by an xor butterfly.
template <int K, bool GUARD, bool SPLITJ = false>
struct AdjointX2Policy {
  static_assert(K % 2 == 0, "the packed form holds i-particles in pairs");
  static constexpr int kSlotF4 = 1;
  static constexpr int kSums = 4;
  static constexpr int kJRec = 2;
  static constexpr bool kSplitJ = SPLITJ;
  // the (hi, lo) running sums spill under a 128-register cap even at K = 2
  static constexpr int kMinBlocks = 1;
  static constexpr int kBlock = AdjointPolicy<1, GUARD>::kBlock;  // entries per lane between compensated folds
  // the lanes of a group are combined in FP32 after their (hi, lo) sums
  // are collapsed (a butterfly of at most five additions)
  __device__ __forceinline__ void reduce_lanes(int jl) {
#pragma unroll
    for (int p = 0; p < K / 2; ++p)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        run[p][c] = __fadd2_rn(run[p][c], runl[p][c]);
        runl[p][c] = dup2(0.f);
      }
    for (int off = jl >> 1; off > 0; off >>= 1) {
#pragma unroll
      for (int p = 0; p < K / 2; ++p)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          run[p][c].x += __shfl_xor_sync(0xffffffffu, run[p][c].x, off);
          run[p][c].y += __shfl_xor_sync(0xffffffffu, run[p][c].y, off);
        }
    }
  }
  float2 nxk[K / 2][3];
  float2 mk[K / 2];
  float2 nwk[K / 2][3];
  float2 run[K / 2][4];   // component 3 holds -(dL/dm)
  float2 runl[K / 2][4];  // low words of the running sums

  __device__ __forceinline__ static float& half(float2& v, int k) { return (k & 1) ? v.y : v.x; }
  __device__ __forceinline__ static float half(const float2& v, int k) { return (k & 1) ? v.y : v.x; }

  __device__ __forceinline__ void load_i(const PairArgs& a, int64_t gi, bool valid, int k) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
      v = __ldg(a.pos_i + gi);
      w = __ldg(a.pos_i2 + gi);
    }
    half(nxk[k >> 1][0], k) = -v.x;
    half(nxk[k >> 1][1], k) = -v.y;
    half(nxk[k >> 1][2], k) = -v.z;
    half(mk[k >> 1], k) = v.w;
    half(nwk[k >> 1][0], k) = -w.x;
    half(nwk[k >> 1][1], k) = -w.y;
    half(nwk[k >> 1][2], k) = -w.z;
  }

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int p = 0; p < K / 2; ++p)
#pragma unroll
      for (int c = 0; c < 4; ++c) run[p][c] = runl[p][c] = dup2(0.f);
  }

  __device__ __forceinline__ void tile(const float4* js, int T, float eps2, int64_t self_off, bool diag, int row,
                                       int rows, int sub, int jl) {
    const float4* jw = js + T;
    const int j0 = SPLITJ ? sub : 0;   // this lane's first entry
    const int js1 = SPLITJ ? jl : 1;   // stride between its entries
    int self_j[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t sj = static_cast<int64_t>(k * rows + row) - self_off;
      self_j[k] = (sj >= 0 && sj < T) ? static_cast<int>(sj) : -1;
    }
    const float2 e2 = dup2(eps2);
#pragma unroll 1
    for (int jb = j0; jb < T; jb += kBlock * js1) {
      const int je = jb + kBlock * js1 < T ? jb + kBlock * js1 : T;
      float2 part[K / 2][4];
#pragma unroll
      for (int p = 0; p < K / 2; ++p)
#pragma unroll
        for (int c = 0; c < 4; ++c) part[p][c] = dup2(0.f);
      if (!diag) {
#pragma unroll 1
        for (int j = jb; j < je; j += 8 * js1) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int e = j + jj * js1;
            pair_adjoint_x2<K, GUARD, false>(js[e], jw[e], nxk, mk, nwk, e2, e, self_j, part);
          }
        }
      } else {
#pragma unroll 1
        for (int j = jb; j < je; j += 8 * js1) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int e = j + jj * js1;
            pair_adjoint_x2<K, GUARD, true>(js[e], jw[e], nxk, mk, nwk, e2, e, self_j, part);
          }
        }
      }
      // TwoSum of each block into the running (hi, lo) sums, per half
#pragma unroll
      for (int p = 0; p < K / 2; ++p)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float2 a = run[p][c], b = part[p][c];
          const float2 s = __fadd2_rn(a, b);
          const float2 bp = sub2(s, a);
          const float2 ap = sub2(s, bp);
          const float2 err = __fadd2_rn(sub2(a, ap), sub2(b, bp));
          run[p][c] = s;
          runl[p][c] = __fadd2_rn(runl[p][c], err);
        }
    }
  }

  __device__ __forceinline__ float total(int k, int c) const {
    return __fadd_rn(half(run[k >> 1][c], k), half(runl[k >> 1][c], k));
  }

  __device__ __forceinline__ void store_final(const PairArgs& a, int64_t i, int k) const {
    float* g = static_cast<float*>(a.acc_out) + 3 * i;
    g[0] = total(k, 0);
    g[1] = total(k, 1);
    g[2] = total(k, 2);
    static_cast<float*>(a.pot_out)[i] = -total(k, 3);
  }

  __device__ __forceinline__ void store_partial(float4* slot, int il, int /*i_tile*/, int k) const {
    slot[il] = make_float4(total(k, 0), total(k, 1), total(k, 2), -total(k, 3));
  }

  __device__ static __forceinline__ void add_partial(const float4 (&v)[kSlotF4], double (&s)[kSums]) {
    AdjointPolicy<K, GUARD>::add_partial(v, s);
  }

  __device__ static __forceinline__ void store_merged(const PairArgs& a, int64_t i, const double (&s)[kSums]) {
    AdjointPolicy<K, GUARD>::store_merged(a, i, s);
  }
};

template <int K, bool POT, bool GUARD>
__device__ __forceinline__ void pair_jerk_x2(const float4 pj, const float4 vj, const float2 (&nxi)[K / 2][3],
                                             const float2 (&nvi)[K / 2][3], float2 e2, float2 (&part)[K / 2][7]) {
  const float2 jx = dup2(pj.x), jy = dup2(pj.y), jz = dup2(pj.z), jm = dup2(pj.w);
  const float2 ux = dup2(vj.x), uy = dup2(vj.y), uz = dup2(vj.z), m3 = dup2(-3.0f);
#pragma unroll
  for (int p = 0; p < K / 2; ++p) {
    const float2 dx = __fadd2_rn(jx, nxi[p][0]);
    const float2 dy = __fadd2_rn(jy, nxi[p][1]);
    const float2 dz = __fadd2_rn(jz, nxi[p][2]);
    const float2 wx = __fadd2_rn(ux, nvi[p][0]);
    const float2 wy = __fadd2_rn(uy, nvi[p][1]);
    const float2 wz = __fadd2_rn(uz, nvi[p][2]);
    float2 s, d2 = dup2(0.f);
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
    const float2 r2 = __fmul2_rn(r, r);
    const float2 mr = __fmul2_rn(jm, r);
    const float2 q = __fmul2_rn(mr, r2);
    const float2 nb = __fmul2_rn(__fmul2_rn(m3, r2), __ffma2_rn(dx, wx, __ffma2_rn(dy, wy, __fmul2_rn(dz, wz))));
    const float2 nqb = __fmul2_rn(q, nb);  // -q b
    part[p][0] = __ffma2_rn(q, dx, part[p][0]);
    part[p][1] = __ffma2_rn(q, dy, part[p][1]);
    part[p][2] = __ffma2_rn(q, dz, part[p][2]);
    part[p][3] = __ffma2_rn(nqb, dx, __ffma2_rn(q, wx, part[p][3]));
    part[p][4] = __ffma2_rn(nqb, dy, __ffma2_rn(q, wy, part[p][4]));
    part[p][5] = __ffma2_rn(nqb, dz, __ffma2_rn(q, wz, part[p][5]));
    if constexpr (POT)
      part[p][6] = __fadd2_rn(part[p][6], make_float2(d2.x != 0.f ? mr.x : 0.f, d2.y != 0.f ? mr.y : 0.f));
  }
}

// SPLITJ (small systems): groups of j_lanes lanes share the thread's
// i-particles, each lane taking every j_lanes-th j entry, combined by an
// xor butterfly at segment ends, as in the plain packed form.
template <int K, bool POT, bool GUARD, bool SPLITJ = false>
struct JerkX2Policy {
  static_assert(K % 2 == 0, "the packed form holds i-particles in pairs");
  static constexpr int kSlotF4 = 2;
  static constexpr int kSums = 7;
  static constexpr int kJRec = 2;
  static constexpr bool kSplitJ = SPLITJ;
  static constexpr int kMinBlocks = 1;
  static constexpr int NC = POT ? 7 : 6;
  __device__ __forceinline__ void reduce_lanes(int jl) {
    for (int off = jl >> 1; off > 0; off >>= 1) {
#pragma unroll
      for (int p = 0; p < K / 2; ++p)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          run[p][c].x += __shfl_xor_sync(0xffffffffu, run[p][c].x, off);
          run[p][c].y += __shfl_xor_sync(0xffffffffu, run[p][c].y, off);
        }
    }
  }
  float2 nxi[K / 2][3];
  float2 nvi[K / 2][3];
  float2 run[K / 2][7];

  __device__ __forceinline__ static float& half(float2& v, int k) { return (k & 1) ? v.y : v.x; }
  __device__ __forceinline__ static float half(const float2& v, int k) { return (k & 1) ? v.y : v.x; }

  __device__ __forceinline__ void load_i(const PairArgs& a, int64_t gi, bool valid, int k) {
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
      p = __ldg(a.pos_i + gi);
      v = __ldg(a.pos_i2 + gi);
    }
    half(nxi[k >> 1][0], k) = -p.x;
    half(nxi[k >> 1][1], k) = -p.y;
    half(nxi[k >> 1][2], k) = -p.z;
    half(nvi[k >> 1][0], k) = -v.x;
    half(nvi[k >> 1][1], k) = -v.y;
    half(nvi[k >> 1][2], k) = -v.z;
  }

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int p = 0; p < K / 2; ++p)
#pragma unroll
      for (int c = 0; c < 7; ++c) run[p][c] = dup2(0.f);
  }

  __device__ __forceinline__ void tile(const float4* js, int T, float eps2, int64_t /*self_off*/, bool /*diag*/,
                                       int /*row*/, int /*rows*/, int sub, int jl) {
    const float4* jv = js + T;
    float2 part[K / 2][7];
#pragma unroll
    for (int p = 0; p < K / 2; ++p)
#pragma unroll
      for (int c = 0; c < 7; ++c) part[p][c] = dup2(0.f);
    const float2 e2 = dup2(eps2);
    if constexpr (SPLITJ) {
      // this lane's j entries: sub, sub + jl, ... (j_tile is a multiple of 8 jl)
#pragma unroll 1
      for (int j = sub; j < T; j += 4 * jl) {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          pair_jerk_x2<K, POT, GUARD>(js[j + jj * jl], jv[j + jj * jl], nxi, nvi, e2, part);
      }
    } else {
#pragma unroll 1
      for (int j = 0; j < T; j += 4) {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) pair_jerk_x2<K, POT, GUARD>(js[j + jj], jv[j + jj], nxi, nvi, e2, part);
      }
    }
#pragma unroll
    for (int p = 0; p < K / 2; ++p)
#pragma unroll
      for (int c = 0; c < NC; ++c) run[p][c] = __fadd2_rn(run[p][c], part[p][c]);
  }

  __device__ __forceinline__ void store_final(const PairArgs& a, int64_t i, int k) const {
    float* acc = static_cast<float*>(a.acc_out) + 3 * i;
    float* jk = static_cast<float*>(a.jerk_out) + 3 * i;
    acc[0] = half(run[k >> 1][0], k);
    acc[1] = half(run[k >> 1][1], k);
    acc[2] = half(run[k >> 1][2], k);
    jk[0] = half(run[k >> 1][3], k);
    jk[1] = half(run[k >> 1][4], k);
    jk[2] = half(run[k >> 1][5], k);
    if constexpr (POT) {
      if (a.pot_out) static_cast<float*>(a.pot_out)[i] = -half(run[k >> 1][6], k);
    }
  }

  __device__ __forceinline__ void store_partial(float4* slot, int il, int i_tile, int k) const {
    slot[il] = make_float4(half(run[k >> 1][0], k), half(run[k >> 1][1], k), half(run[k >> 1][2], k),
                           half(run[k >> 1][3], k));
    slot[i_tile + il] = make_float4(half(run[k >> 1][4], k), half(run[k >> 1][5], k), half(run[k >> 1][6], k), 0.f);
  }

  __device__ static __forceinline__ void add_partial(const float4 (&v)[kSlotF4], double (&s)[kSums]) {
    JerkPolicy<K, POT, GUARD>::add_partial(v, s);
  }

  __device__ static __forceinline__ void store_merged(const PairArgs& a, int64_t i, const double (&s)[kSums]) {
    JerkPolicy<K, POT, GUARD>::store_merged(a, i, s);
  }
};

// ------------------------------------------------------------------ debug checks
#ifdef CN_DEBUG_BOUNDS
// Debug build only (-DCN_DEBUG_BOUNDS): every tile the schedule reaches is
// checked against the unit numbering and the sizes the launch was planned
// with. A violation sets kStatusBadSchedule in the device status word,
// switches the CTA to the abort path (no more copies, waits or pair work)
// and empties the tile, so that nothing outside the buffers is touched.
__device__ __forceinline__ void bad_schedule(const PairArgs& a, volatile int* ctl) {
  set_status(a.status, kStatusBadSchedule);
  ctl[0] = 1;
}

// tile index tc as returned by the unit lookup: inside the table?
__device__ __forceinline__ int32_t checked_tile_index(const PairArgs& a, int32_t tc, volatile int* ctl) {
  if (tc >= 0 && tc < a.n_tiles) return tc;
  bad_schedule(a, ctl);
  return 0;
}

// descriptor td must hold unit u, fit the i-tile and lie inside the i and j
// arrays (j_extent: the j records, or the list entries of a gathering
// plan); j_tile records per j-tile
__device__ __forceinline__ void check_tile(const PairArgs& a, TileDesc& td, int64_t u, int IT, int T, int64_t j_extent,
                                           volatile int* ctl) {
  const bool ok = td.njt >= 1 && td.unit0 <= u && u < td.unit0 + td.njt && td.ni >= 0 && td.ni <= IT && td.i0 >= 0 &&
                  td.i0 + td.ni <= a.n_i && td.nj >= 1 && td.j0 >= 0 && td.j0 + td.nj <= j_extent &&
                  td.njt == (td.nj + T - 1) / T;
  if (ok) return;
  bad_schedule(a, ctl);
  td.ni = 0;
  td.unit0 = u;
  if (td.njt < 1) td.njt = 1;
}
#endif

// ------------------------------------------------------------------ kernel
// Register budget per policy: Policy::kMinBlocks 256-thread CTAs must fit
// on an SM (2: up to 128 registers per thread; 1: up to 255).
//
// GATHER (interaction-list plans with an index array): the records of a
// j-tile are pos_j[j_index[e]] for the tile's list entries e, not a
// contiguous range. Every thread then stages its share of each tile (the
// entries t = tid, tid + threads, ...): it copies those indices into shared
// memory (4-byte cp.async, fetched one load ahead so that it does not wait
// for them), copies their records with 16-byte cp.async and arrives on the
// stage's full barrier (initialised for one arrival per thread) once its
// copies have landed; lane 0 of each warp waits for the stage to be free.
// Measured on the 512 x 256 x 4096 lists: one 16-byte bulk copy per record
// issued by warp 0 took 2.8x the contiguous kernel's time (the copy engine
// takes small copies one at a time), cp.async by warp 0 alone 1.16x, spread
// over all warps 1.08-1.12x.
template <class Policy, int K, bool BATCHED, bool GATHER = false>
__global__ void __launch_bounds__(256, Policy::kMinBlocks) pair_kernel(const __grid_constant__ PairArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int NT = blockDim.x;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int T = a.j_tile;
  const int S = a.stages;
  // thread -> (i row, j lane): rows = threads / j_lanes i-particles per k
  constexpr bool SJ = Policy::kSplitJ;
  const int JL = SJ ? a.j_lanes : 1;
  const int sub = SJ ? tid % JL : 0;
  const int row = SJ ? tid / JL : tid;
  const int ROWS = SJ ? NT / JL : NT;
  const int IT = ROWS * K;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + S;
  volatile int* ctl = reinterpret_cast<volatile int*>(smem + 16 * S);  // [0] abort [1] last [2] chunk
  float4* ring = reinterpret_cast<float4*>(smem + 256);
  // gathering form: two buffers of T list indices behind the ring
  int32_t* gidx = reinterpret_cast<int32_t*>(ring + static_cast<size_t>(S) * T * Policy::kJRec);

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], GATHER ? NT : 1);  // gathering: one arrival per thread
      mbar_init(&empty[s], NT / 32);
    }
    ctl[0] = 0;
    ctl[1] = 0;
    mbar_init_fence();
  }
  __syncthreads();
  // Up to here only shared memory was touched; the previous kernel of the
  // stream may still be writing global memory until the wait returns.
  grid_dependency_wait();
  grid_launch_dependents();

  const Sched sc{a.total_units, a.n_chunks, a.chunk_units};
  const bool dynamic = a.chunk_units > 0;
  // prefetch distance in tiles: a stage is refilled once every warp has left
  // the tile two loads back (one tile of slack); a 2-stage ring refills the
  // stage of the previous tile, a 1-stage ring loads one tile at a time
  const uint32_t D = S > 2 ? static_cast<uint32_t>(S - 2) : static_cast<uint32_t>(S - 1);
  uint32_t issued = 0;    // loads issued (thread 0 only; every thread when gathering)
  uint32_t fetched = 0xffffffffu;  // gathering: the load whose indices were fetched ahead
  uint32_t consumed = 0;  // tiles consumed (identical in every thread)
  constexpr int JR = Policy::kJRec;
  Policy acc;

  int64_t q = dynamic ? -1 : static_cast<int64_t>(blockIdx.x);
  for (;;) {
    if (dynamic) {
      if (tid == 0) ctl[2] = atomicAdd(&a.queue[0], 1);
      __syncthreads();
      q = ctl[2];
      __syncthreads();
    }
    if (q >= sc.Q) break;
    const int64_t ub = sc.begin(q);
    const int64_t ue = sc.end(q);
    if (ub < ue) {
      int32_t tc = tile_of_unit<BATCHED>(a, ub);
#ifdef CN_DEBUG_BOUNDS
      tc = checked_tile_index(a, tc, ctl);
#endif
      TileDesc td = tile_at<BATCHED>(a, tc, IT);
#ifdef CN_DEBUG_BOUNDS
      check_tile(a, td, ub, IT, T, GATHER ? a.n_index : a.n_j, ctl);
#endif
      int64_t jt = ub - td.unit0;
      // producer cursor (meaningful in thread 0 only)
      int32_t tp = tc;
      TileDesc tdp = td;
      int64_t jtp = jt;
      const uint32_t last_load = consumed + static_cast<uint32_t>(ue - ub);
      int64_t seg_u0 = ub;
      bool seg_open = false;
      for (int64_t uc = ub; uc < ue; ++uc) {
        if constexpr (GATHER) {
          {
            for (;;) {
              // lane 0 decides for its warp (another warp may set ctl[0])
              int go = (!ctl[0] && issued < last_load && issued <= consumed + D) ? 1 : 0;
              go = __shfl_sync(0xffffffffu, go, 0);
              if (!go) break;
              const int slot = static_cast<int>(issued % S);
              int ok = 1;
              if (lane == 0 && issued >= static_cast<uint32_t>(S) &&
                  !mbar_wait(&empty[slot], ((issued / S) - 1) & 1u, a.wait_ns)) {
                set_status(a.status, kStatusTimeoutEmpty);
                ctl[0] = 1;
                ok = 0;
              }
              ok = __shfl_sync(0xffffffffu, ok, 0);
              if (!ok) break;
              __syncwarp();
              const int64_t jb = jtp * T;
              const int64_t left = tdp.nj - jb;
              const int cnt = static_cast<int>(left < T ? left : T);
#ifdef CN_DEBUG_BOUNDS
              if (tp >= a.n_tiles || cnt < 1 || tdp.j0 + jb < 0 || tdp.j0 + jb + cnt > a.n_index) {
                if (lane == 0) bad_schedule(a, ctl);
                break;
              }
#endif
              int32_t* ix = gidx + (issued & 1u) * T;
              if (fetched != issued) {  // the first load of a range: not fetched ahead
                for (int t = tid; t < cnt; t += NT) cp_async_4(ix + t, a.j_index + tdp.j0 + jb + t);
                cp_async_commit();
                cp_async_wait_all();
              } else {
                cp_async_wait_prior();  // the indices, committed before the latest records
              }
              float4* dst = ring + static_cast<size_t>(slot) * T;
              // the indices of the range's next load, fetched while the warp computes
              const uint32_t nxt = issued + 1;
              int64_t jtn = jtp + 1;
              int32_t tn = tp;
              TileDesc tdn = tdp;
              if (jtn == tdp.njt) {
                ++tn;
                jtn = 0;
                if (nxt < last_load) tdn = tile_at<BATCHED>(a, tn, IT);
              }
              if (nxt < last_load) {
                const int64_t jb2 = jtn * T;
                const int64_t left2 = tdn.nj - jb2;
                const int cnt2 = static_cast<int>(left2 < T ? left2 : T);
                int32_t* ix2 = gidx + (nxt & 1u) * T;
#ifdef CN_DEBUG_BOUNDS
                if (tn < a.n_tiles && tdn.j0 + jb2 >= 0 && tdn.j0 + jb2 + cnt2 <= a.n_index)
#endif
                  for (int t = tid; t < cnt2; t += NT) cp_async_4(ix2 + t, a.j_index + tdn.j0 + jb2 + t);
                fetched = nxt;
              }
              cp_async_commit();
              // the tile's records, and zeros (zero mass) past a short tile's end;
              // each thread's arrival on the full barrier lands with its copies
              for (int t = tid; t < T; t += NT) {
                if (t < cnt) {
                  int32_t e = ix[t];
#ifdef CN_DEBUG_BOUNDS
                  if (e < 0 || e >= a.n_j) {
                    bad_schedule(a, ctl);
                    e = 0;
                  }
#endif
                  cp_async_16(dst + t, a.pos_j + e);
                } else {
                  cp_async_zero_16(dst + t, a.pos_j);
                }
              }
              cp_async_arrive_noinc(&full[slot]);
              cp_async_commit();
              ++issued;
              jtp = jtn;
              tp = tn;
              tdp = tdn;
            }
          }
        } else if (tid == 0) {
          while (!ctl[0] && issued < last_load && issued <= consumed + D) {
            const int slot = static_cast<int>(issued % S);
            if (issued >= static_cast<uint32_t>(S) &&
                !mbar_wait(&empty[slot], ((issued / S) - 1) & 1u, a.wait_ns)) {
              set_status(a.status, kStatusTimeoutEmpty);
              ctl[0] = 1;
              break;
            }
            const int64_t jb = jtp * T;
            const int64_t left = tdp.nj - jb;
            const int cnt = static_cast<int>(left < T ? left : T);
#ifdef CN_DEBUG_BOUNDS
            if (tp >= a.n_tiles || cnt < 1 || tdp.j0 + jb < 0 || tdp.j0 + jb + cnt > a.n_j) {
              bad_schedule(a, ctl);
              break;
            }
#endif
            float4* dst = ring + static_cast<size_t>(slot) * T * JR;
            for (int z = cnt; z < T; ++z) {  // zero-mass (and zero-weight) padding of a short tile
              dst[z] = make_float4(0.f, 0.f, 0.f, 0.f);
              if constexpr (JR == 2) dst[T + z] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&full[slot], static_cast<uint32_t>(cnt) * 16u * JR);
            bulk_copy_g2s(dst, a.pos_j + tdp.j0 + jb, static_cast<uint32_t>(cnt) * 16u, &full[slot]);
            if constexpr (JR == 2)
              bulk_copy_g2s(dst + T, a.pos_j2 + tdp.j0 + jb, static_cast<uint32_t>(cnt) * 16u, &full[slot]);
            ++issued;
            if (++jtp == tdp.njt) {
              ++tp;
              jtp = 0;
              if (tp < a.n_tiles) tdp = tile_at<BATCHED>(a, tp, IT);
            }
          }
        }
        if (!seg_open) {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int il = k * ROWS + row;
            acc.load_i(a, td.i0 + il, il < td.ni, k);
          }
          acc.zero();
          seg_u0 = uc;
          seg_open = true;
        }
        const int slot = static_cast<int>(consumed % S);
        // After a timed-out wait anywhere in the CTA (ctl[0] set) every thread
        // keeps walking the same units and segment ends - so all of them meet
        // the same barriers - but waits, computes and releases nothing more.
        bool live = !ctl[0];
        if (live && !mbar_wait(&full[slot], (consumed / S) & 1u, a.wait_ns)) {
          set_status(a.status, kStatusTimeoutFull);
          ctl[0] = 1;
          live = false;
        }
        live = __all_sync(0xffffffffu, live);
        if (live) {
          // j-range of this unit relative to the i-tile (used by the adjoint's self-pair exclusion)
          const int64_t self_off = td.j0 + jt * T - td.i0;
          const bool diag = self_off < IT && self_off + T > 0;
          acc.tile(ring + static_cast<size_t>(slot) * T * JR, T, td.eps2, self_off, diag, row, ROWS, sub, JL);
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[slot]);
        }
        ++consumed;
        ++jt;
        if (jt == td.njt || uc + 1 == ue) {
          // ---- end of a segment: write the tile or its partial
          if constexpr (SJ) acc.reduce_lanes(JL);
          int64_t qf = sc.chunk_of(td.unit0);
          int64_t ql = sc.chunk_of(td.unit0 + td.njt - 1);
#ifdef CN_DEBUG_BOUNDS
          if (qf < 0 || ql >= sc.Q || qf > q || q > ql) {
            bad_schedule(a, ctl);
            qf = ql = q;  // the tile is then written by this chunk alone
          }
#endif
          if (qf == ql) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const int il = k * ROWS + row;
              if (il < td.ni && sub == 0) acc.store_final(a, td.i0 + il, k);
            }
          } else {
            const int which = (seg_u0 == ub) ? 0 : 1;
            float4* slotp = a.partials + static_cast<size_t>(q * 2 + which) * IT * Policy::kSlotF4;
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const int il = k * ROWS + row;
              if (sub == 0) acc.store_partial(slotp, il, IT, k);
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) {
              const unsigned before = atomicAdd(&a.counters[tc], 1u);
              ctl[1] = (before == static_cast<unsigned>(ql - qf)) ? 1 : 0;
            }
            __syncthreads();
            if (ctl[1]) {
              __threadfence();
              // every thread of the CTA takes particles of the tile in turn
              // (with split-j lanes only one lane in j_lanes held results,
              // and the FP64 adds are the merge's slow part on this GPU)
              for (int il = tid; il < td.ni; il += NT) {
                double s[Policy::kSums];
#pragma unroll
                for (int c = 0; c < Policy::kSums; ++c) s[c] = 0.0;
                // A batch of partials is loaded at once (independent L2 reads
                // in flight together), then added in chunk order.
                constexpr int kBatch = 8 / Policy::kSlotF4;
                for (int64_t p0 = qf; p0 <= ql; p0 += kBatch) {
                  float4 v[kBatch][Policy::kSlotF4];
#pragma unroll
                  for (int u = 0; u < kBatch; ++u) {
                    const int64_t p = p0 + u;
                    if (p <= ql) {
                      const int w = (sc.begin(p) >= td.unit0) ? 0 : 1;
                      const float4* slot = a.partials + static_cast<size_t>(p * 2 + w) * IT * Policy::kSlotF4;
#pragma unroll
                      for (int h = 0; h < Policy::kSlotF4; ++h) v[u][h] = __ldcg(slot + h * IT + il);
                    }
                  }
#pragma unroll
                  for (int u = 0; u < kBatch; ++u)
                    if (p0 + u <= ql) Policy::add_partial(v[u], s);
                }
                Policy::store_merged(a, td.i0 + il, s);
              }
              if (tid == 0) a.counters[tc] = 0u;
            }
          }
          seg_open = false;
          if (jt == td.njt) {
            ++tc;
            jt = 0;
            if (tc < a.n_tiles) td = tile_at<BATCHED>(a, tc, IT);
#ifdef CN_DEBUG_BOUNDS
            if (uc + 1 < ue) {
              tc = checked_tile_index(a, tc, ctl);
              td = tile_at<BATCHED>(a, tc, IT);
              check_tile(a, td, uc + 1, IT, T, GATHER ? a.n_index : a.n_j, ctl);
            }
#endif
          }
        }
      }
    }
    if (!dynamic) break;
  }

  if (dynamic && tid == 0) {
    __threadfence();
    const int done = atomicAdd(&a.queue[1], 1);
    if (done == static_cast<int>(gridDim.x) - 1) {
      a.queue[0] = 0;
      a.queue[1] = 0;
    }
  }
  // gathering: copies this thread issued (an aborted run may leave some)
  if constexpr (GATHER) cp_async_wait_all();
  // On an aborted run, wait (bounded) for copies that may still be in
  // flight - at most the latest one per stage, since a stage is refilled
  // only after every warp saw its previous copy land - before the shared
  // memory they target is released.
  // (The gathering form's copies are covered by each thread's own wait above.)
  if (!GATHER && tid == 0 && ctl[0]) {
    for (uint32_t c = issued > static_cast<uint32_t>(S) ? issued - S : 0u; c < issued; ++c) {
      if (!mbar_wait(&full[c % S], (c / S) & 1u, a.wait_ns)) {
        set_status(a.status, kStatusTimeoutDrain);
        break;
      }
    }
  }
}

}  // namespace cn
