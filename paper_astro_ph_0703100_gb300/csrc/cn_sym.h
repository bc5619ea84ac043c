// Symmetric (each unordered pair once) evaluation of an i set equal to the
// j set: launch arguments and entry points of cn_sym.cu.
#pragma once

#include "cn_kernels.h"

namespace cn {

// One launch covers the tile rows I in [row0, row0 + band) of the upper
// triangle of tile pairs (I <= J), i.e. units unit_base .. unit_base + units
// - 1 of the row-major numbering, split into equal contiguous ranges over
// the grid's CTAs. A CTA adds the i-side sums (tile I) of each of its units
// of one row, by TwoSum, into one (hi, lo) slot pair per (CTA, row) segment:
// slots_seg[(c + I - row0) * 2 tile + {0, tile} + p - I * tile] for CTA c (c +
// I - row0 is unique per segment, since along the unit sequence neither the
// CTA nor the row index decreases). Unit (I, J), I < J, writes its j-side
// sums (tile J, partner I) to slots_j[(I - row0) * n_pad + p].
struct SymArgs {
  const float4* pos;  // [n] (x, y, z, m)
  float4* slots_seg;  // [n_seg][2][tile] (hi, lo), n_seg >= grid + band rows
  int64_t n_seg;
  float4* slots_j;
  int* status;
  int64_t n;
  int64_t n_pad;      // n_tiles * tile
  int64_t unit_base;  // first unit of the launch (row-major over I <= J)
  int64_t units;      // units of the launch
  int32_t n_tiles;
  int32_t row0;       // first tile row of the launch
  int32_t sub_tile;   // j records per ring stage (divides the tile, multiple of 8)
  int32_t stages;
  float eps2;
  uint64_t wait_ns;
};

// Per-particle merge of one band: adds, in FP64, the band's j-side slots (x,
// y, z and the potential in w) in ascending partner order (partners I in
// [row0, row1), I < P) and, for particles of the band's own tiles, the
// i-side segments of their row in CTA order, to the running sums (acc64, or
// zero for the first band); the last band writes the FP32 accelerations,
// the others store the FP64 sums. The segments of row P are those of the
// CTAs whose unit ranges meet [row_start(P), row_start(P + 1)).
struct SymMerge {
  const float4* slots_seg;
  const float4* slots_j;
  double* acc64;     // [n][4] (acceleration, potential), NULL with a single band
  float* acc_out;    // [n][3]
  float* pot_out;    // [n] or NULL
  int64_t n;
  int64_t n_pad;
  int64_t unit_base;  // the band launch's schedule: first unit, units, CTAs
  int64_t units;
  int64_t grid;
  int32_t tile;
  int32_t n_tiles;
  int32_t row0;
  int32_t row1;
  int32_t first;
  int32_t last;
};

size_t sym_smem_bytes(int threads, int k, int sub_tile, int stages, bool pot);
cudaError_t occupancy_sym(int k, bool guard, int threads, size_t smem, int* ctas, bool pot);
cudaError_t launch_sym(const SymArgs& a, const SymMerge& m, int k, bool guard, int threads, int grid, size_t smem,
                       cudaStream_t s, bool pot);

}  // namespace cn
