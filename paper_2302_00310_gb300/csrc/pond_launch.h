// pond_launch.h -- the descriptor table read by the member step kernel, and
// the launch handles of its instantiations (not part of the C ABI).
//
// One kernel function serves both a single context (pond_step: a table with
// one member, one CTA per tile) and a batch (pond_batch_step: many members,
// a persistent grid), so a member's arithmetic is the same machine code
// either way and its state is bit for bit the same alone or in a batch.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <vector>

#include "pond_kernels.cuh"

namespace pond {

// The work unit of a launch is a strip: up to `strip` consecutive tiles of one
// row of a member's tiles, which one CTA steps from left to right, handing
// each tile's right-edge x-faces to the next tile as its left edge (a face's
// record depends only on its stencil, so the handed-over record is the one the
// next tile would compute).
template <typename R> struct InstDesc {
  StepConst K;
  State<R> S[2];
  Stats *stats;
  int tiles_x;     // tiles per row of the member's grid
  int tile_begin;  // first global strip index of the member
  int steps;       // launch k advances the member iff k < steps
  int parity;      // launch k reads buffer (parity + k) & 1 and writes the other
};

struct TableHdr {
  int n;            // members in the table
  int total_tiles;  // strips over all members
  int strip;        // tiles per strip (>= 1); a row's last strip may be shorter
  int pad[61];      // 256-byte header
};

// strips of a member with tiles_x x tiles_y tiles
inline int strips_of(int tiles_x, int tiles_y, int strip) { return (tiles_x + strip - 1) / strip * tiles_y; }

// Tiles per strip for a table of `tiles` tiles in rows of `tiles_x`, on
// `slots` resident CTAs: 2 where that keeps the launch's waves x strip length
// at its minimum (hands edges over without lengthening the launch's critical
// path), else 1.  Longer strips tie on that count in many grids but measured
// slower (a 1024^2 Riemann step, FP32: 1338 MLUPS in strips of 8 against 1504
// in strips of 1; strips of 1 and 2 within 1.5 % of each other).
constexpr int kMaxAutoStrip = 2;
inline int choose_strip(int tiles_x, int tiles_y, int slots) {
  int best = 1;
  long long best_cost = -1;
  for (int L = 1; L <= kMaxAutoStrip; L *= 2) {
    if (L > 1 && L > tiles_x) break;
    const long long units = strips_of(tiles_x, tiles_y, L);
    const long long cost = (units + slots - 1) / slots * L;
    if (best_cost < 0 || cost <= best_cost) { best = L; best_cost = cost; }
  }
  return best;
}

// device bytes reserved in a context's workspace for its one-member table
constexpr size_t kSoloTableBytes = 1024;
static_assert(sizeof(TableHdr) + sizeof(InstDesc<double>) <= kSoloTableBytes, "solo table");

// One instantiation of the member step kernel: its tile geometry, the
// shared-memory opt-in plus occupancy query, and the launch.
struct Shape {
  int code, bx, by;
  cudaError_t (*prepare)(int *ctas_per_sm);
  void (*launch)(const unsigned char *table, int k, int grid, cudaStream_t st);
};

}  // namespace pond

// Every tile code of dimension D (1D: code 1; 2D: codes 2-6, see
// pond_params.tile) and the iterated-face-frame shape, per precision; defined
// in pond_step_fp64.cu / pond_step_fp32.cu.
std::vector<pond::Shape> pond_shapes_fp64(int D);
std::vector<pond::Shape> pond_shapes_fp32(int D);
pond::Shape pond_iter_shape_fp64(int D);
pond::Shape pond_iter_shape_fp32(int D);
// the D2Q25 f-lattice (pond_step_fp64_q5.cu / pond_step_fp32_q5.cu)
std::vector<pond::Shape> pond_shapes_fp64_q5();
std::vector<pond::Shape> pond_shapes_fp32_q5();
pond::Shape pond_iter_shape_fp64_q5();
pond::Shape pond_iter_shape_fp32_q5();
// the multiscale f-lattice (pond_step_fp64_ms.cu / pond_step_fp32_ms.cu)
pond::Shape pond_ms_shape_fp64(int D);
pond::Shape pond_ms_shape_fp32(int D);
// g on the f-lattice (pond_step_fp64_g4.cu / pond_step_fp32_g4.cu)
pond::Shape pond_g4_shape_fp64(int D);
pond::Shape pond_g4_shape_fp32(int D);
