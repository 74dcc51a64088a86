// pond_step_impl.cuh -- the member step kernel and its launch handles.  Included
// only by pond_step_fp64.cu and pond_step_fp32.cu, so that each instantiation
// exists once.
#pragma once
#include "pond_launch.h"

namespace pond {

// Launch k of a chunk: the grid strides over the table's strips; member i owns
// strips [tile_begin_i, tile_begin_i + strips_i) and advances iff k < steps_i,
// from buffer (parity_i + k) & 1 into the other, with its own constants and
// status block.  A strip's tiles are stepped left to right, each handing its
// right-edge x-face records to the next (not with the iterated face frame,
// whose trace statistics count each face at one tile).  A one-member table
// with one CTA per strip is a plain step.
template <typename R, int DIM, int QF1, int BX, int BY, int NT, int MINB, bool ITER, bool MS = false,
          int QG1 = 3>
__global__ void __launch_bounds__(NT, MINB) member_step_kernel(const unsigned char *table, int k) {
  const TableHdr *H = reinterpret_cast<const TableHdr *>(table);
  const InstDesc<R> *desc = reinterpret_cast<const InstDesc<R> *>(table + sizeof(TableHdr));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ StepConst Ks;
  __shared__ int s_inst;
  const int n = H->n, total = H->total_tiles, L = H->strip > 0 ? H->strip : 1;
  int loaded = -1;
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    if (threadIdx.x == 0) {
      int lo = 0, hi = n - 1;  // the last member whose first strip is <= t
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (desc[mid].tile_begin <= t) lo = mid;
        else hi = mid - 1;
      }
      s_inst = lo;
    }
    __syncthreads();
    const int i = s_inst;
    const InstDesc<R> &d = desc[i];
    if (k < d.steps) {  // the same for every thread of the CTA
      if (i != loaded) {
        for (int w = threadIdx.x; w < (int)(sizeof(StepConst) / 4); w += NT)
          reinterpret_cast<int *>(&Ks)[w] = reinterpret_cast<const int *>(&d.K)[w];
        __syncthreads();
        loaded = i;
      }
      const int ls = t - d.tile_begin, p = (d.parity + k) & 1, tx = d.tiles_x;
      const int per_row = (tx + L - 1) / L, ty = ls / per_row, tx0 = (ls % per_row) * L;
      const int tx1 = tx0 + L < tx ? tx0 + L : tx;
      // values, not references into the table: the step's global stores could
      // alias the table as far as the compiler knows, forcing reloads
      const State<R> S = d.S[p], O = d.S[p ^ 1];
      Stats *const st = d.stats;
      for (int x = tx0; x < tx1; ++x) {
        const bool carry = !ITER && x > tx0;
        if (carry) {
          __syncthreads();  // the previous tile's phase C has read its face records
          hand_over_x_edge<R, DIM, QF1, BX, BY, NT, QG1>(smem_raw);
        }
        step_tile<R, DIM, QF1, BX, BY, NT, ITER, MS, QG1>(Ks, S, O, st, x * BX, DIM == 2 ? ty * BY : 0,
                                                          smem_raw, carry);
      }
    }
    __syncthreads();  // s_inst, Ks and the tile's shared memory are reused
  }
}

template <typename R, int DIM, int BX, int BY, int NT, int MINB, bool ITER, int QF1 = 4, bool MS = false,
          int QG1 = 3>
Shape make_shape(int code) {
  Shape s;
  s.code = code;
  s.bx = BX;
  s.by = BY;
  s.prepare = [](int *ctas) -> cudaError_t {
    constexpr size_t smem = Tile<DIM, BX, BY, QF1, QG1>::template smem_bytes<R, MS>();
    static_assert(smem + sizeof(StepConst) + 16 <= 227 * 1024, "tile too large for shared memory");
    cudaError_t e = cudaFuncSetAttribute(member_step_kernel<R, DIM, QF1, BX, BY, NT, MINB, ITER, MS, QG1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        ctas, member_step_kernel<R, DIM, QF1, BX, BY, NT, MINB, ITER, MS, QG1>, NT, smem);
  };
  s.launch = [](const unsigned char *table, int k, int grid, cudaStream_t st) {
    constexpr size_t smem = Tile<DIM, BX, BY, QF1, QG1>::template smem_bytes<R, MS>();
    member_step_kernel<R, DIM, QF1, BX, BY, NT, MINB, ITER, MS, QG1><<<grid, NT, smem, st>>>(table, k);
  };
  return s;
}

// tile codes: 1 = 1D, 252 cells; 2D (x by y): 2 = 8x8, 3 = 16x16, 4 = 16x8,
// 5 = 8x8 and 6 = 8x16 with registers capped for two CTAs per SM, 7 = 8x16
// and 8 = 8x8 with registers capped for three CTAs per SM, 9 = 8x16 with 192
// threads (no cap: one FP64 CTA per SM is all shared memory holds), 10 = 8x14
// with 128 threads and two CTAs per SM (an FP64 tile's shared memory fits
// twice, and 2 x 128 threads x 255 registers fit the register file), 11 (the
// mixed path only) = 8x14 with 128 threads and registers capped for three
// CTAs per SM
template <typename R> std::vector<Shape> all_shapes(int D) {
  if (D == 1) return {make_shape<R, 1, 252, 1, 256, 1, false>(1)};
  std::vector<Shape> s = {make_shape<R, 2, 8, 8, 160, 1, false>(2), make_shape<R, 2, 16, 16, 256, 1, false>(3),
                          make_shape<R, 2, 16, 8, 256, 1, false>(4), make_shape<R, 2, 8, 8, 160, 2, false>(5),
                          make_shape<R, 2, 8, 16, 160, 2, false>(6), make_shape<R, 2, 8, 16, 160, 3, false>(7),
                          make_shape<R, 2, 8, 8, 160, 3, false>(8), make_shape<R, 2, 8, 16, 192, 1, false>(9),
                          make_shape<R, 2, 8, 14, 128, 2, false>(10)};
  if constexpr (std::is_same<R, float>::value) s.push_back(make_shape<R, 2, 8, 14, 128, 3, false>(11));
  return s;
}

// the iterated face frame runs with one tile shape of its own: its trace loop
// spills, and the 8x8 one-CTA tile outran the 8x14 two-CTA one (23 against 27
// MLUPS on a 128^2 pulse in FP64)
template <typename R> Shape iter_shape(int D) {
  if (D == 1) return make_shape<R, 1, 252, 1, 256, 1, true>(1);
  return make_shape<R, 2, 8, 8, 160, 1, true>(2);
}

// the multiscale f-lattice: the default tile, 8x14 with 128 threads and two
// CTAs per SM, 252 cells in 1D
template <typename R> Shape ms_shape(int D) {
  if (D == 1) return make_shape<R, 1, 252, 1, 256, 1, false, 4, true>(1);
  return make_shape<R, 2, 8, 14, 128, 2, false, 4, true>(10);
}

// g on the f-lattice (D1Q4 / D2Q16): the default tile, 8x14 with 128
// threads and two CTAs per SM, 252 cells in 1D
template <typename R> Shape g4_shape(int D) {
  if (D == 1) return make_shape<R, 1, 252, 1, 256, 1, false, 4, false, 4>(1);
  return make_shape<R, 2, 8, 14, 128, 2, false, 4, false, 4>(10);
}

}  // namespace pond

namespace pond {
// the D2Q25 f-lattice (five nodes per axis), 8x8 tiles: 128 threads and two
// CTAs per SM (tile code 10, the default: 46.7 against 33.8 MLUPS in FP64 and
// 469 against 289 mixed on a 256^2 pulse) or 160 threads and one CTA (code 2,
// also the iterated face frame's)
template <typename R> std::vector<Shape> all_shapes_q5() {
  return {make_shape<R, 2, 8, 8, 160, 1, false, 5>(2), make_shape<R, 2, 8, 8, 128, 2, false, 5>(10)};
}
template <typename R> Shape iter_shape_q5() { return make_shape<R, 2, 8, 8, 160, 1, true, 5>(2); }
}  // namespace pond
