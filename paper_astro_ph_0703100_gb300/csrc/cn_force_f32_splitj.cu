// Split-j FP32 pair-kernel instantiations with four or eight i-particles
// per lane group (packed f32x2), for single systems and for batched /
// interaction-list plans. Lanes of a group of j_lanes share the thread's
// i-particles and take every j_lanes-th j record of a tile; their sums are
// combined by the xor butterfly of F32x2Policy::reduce_lanes at segment
// ends. With K = 4 or 8 each j record feeds two or four independent packed
// pair terms, which hides the FP32 latency that limits K = 2 at mid-size N,
// while j_lanes keeps the i-tile (K x threads / j_lanes) small enough for
// those sizes and for small interaction-list groups. Unguarded kernels only
// (eps2 >= FLT_MIN); the guarded form keeps one i-particle per thread.
#include "cn_pair.cuh"

namespace cn {
namespace {

template <int K, bool POT, bool BATCHED>
const void* fn() {
  return reinterpret_cast<const void*>(&pair_kernel<F32x2Policy<K, POT, false, true, false>, K, BATCHED>);
}

template <bool POT, bool BATCHED>
const void* by_k(int k) {
  switch (k) {
    case 2: return BATCHED ? fn<2, POT, true>() : nullptr;  // single-system K = 2 lives with the other FP32 kernels
    case 4: return fn<4, POT, BATCHED>();
    case 8: return fn<8, POT, BATCHED>();
    default: return nullptr;
  }
}

}  // namespace

const void* select_f32_splitj_wide(int k, bool pot, bool batched) {
  if (batched) return pot ? by_k<true, true>(k) : by_k<false, true>(k);
  return pot ? by_k<true, false>(k) : by_k<false, false>(k);
}

}  // namespace cn
