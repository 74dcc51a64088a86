// pond_internal.h -- the context object shared by the translation units of
// the library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "pond.h"
#include "pond_launch.h"

struct pond_ctx {
  pond_lattice lat;
  int D;
  int qf1;                // f-lattice nodes per axis: 4, or 5 (D2Q25)
  int qg1;                // g-lattice nodes per axis: 3, or 4 (g on the f-lattice)
  int64_t nx, ny, N;
  pond_params p;
  bool fp32;
  cudaStream_t stream;
  unsigned char *ws;
  size_t ws_bytes;
  bool own_ws;
  unsigned char *buf[2];  // state buffers (Hermite coefficients + frame)
  size_t buf_bytes;
  pond::Stats *stats;
  int cur;                // buffer holding the current state
  bool inited;
  double dt;
  int64_t steps;
  int tile;
  pond::StepConst K;
  cudaGraphExec_t graph[2];
  int graph_chunk;
  void *batch;            // the batch this context belongs to, if any
  unsigned char *table;   // its one-member descriptor table (device, in the workspace)
  pond::Shape shape;      // the step kernel instantiation it launches
  int tiles;              // tiles of its grid for that shape
};

namespace pond_detail {

inline int qf_of(int D, int qf1 = 4) { return D == 2 ? qf1 * qf1 : qf1; }
inline int qf1_of(pond_lattice lat) { return lat == POND_D2Q25 ? 5 : 4; }
inline int qg_of(int D, int qg1 = 3) { return D == 2 ? qg1 * qg1 : qg1; }
inline int qg1_of(const pond_params *p) { return p->g_same_as_f ? 4 : 3; }

// bytes of the arithmetic planes f, g, ux, uy, T of one state buffer, rounded
// up to 8; the mixed path's FP64 conserved moments M[4][N] follow them
inline size_t coef_bytes(int D, bool fp32, size_t N, int qf1 = 4, int qg1 = 3) {
  return ((size_t)(qf_of(D, qf1) + qg_of(D, qg1) + 3) * N * (fp32 ? 4 : 8) + 7) / 8 * 8;
}
inline size_t state_bytes(int D, bool fp32, size_t N, int qf1 = 4, int qg1 = 3) {
  return coef_bytes(D, fp32, N, qf1, qg1) + (fp32 ? 4 * N * sizeof(double) : 0);
}

template <typename R> pond::State<R> state_of(const pond_ctx *c, int b) {
  R *base = reinterpret_cast<R *>(c->buf[b]);
  pond::State<R> s;
  s.f = base;
  s.g = s.f + (size_t)qf_of(c->D, c->qf1) * c->N;
  s.ux = s.g + (size_t)qg_of(c->D, c->qg1) * c->N;
  s.uy = s.ux + c->N;
  s.T = s.uy + c->N;
  s.M = c->fp32 ? reinterpret_cast<double *>(c->buf[b] + coef_bytes(c->D, true, (size_t)c->N, c->qf1, c->qg1))
                 : nullptr;
  return s;
}

}  // namespace pond_detail

// the constants of one step for parameters p on a D-dimensional nx x ny grid
// with time step dt (pond_abi.cu; the context path and pond_step_noalloc)
void pond_fill_step_const(pond::StepConst &K, const pond_params &p, int D, int64_t nx, int64_t ny,
                          double dt);

// removes a context from its batch (pond_batch.cu); called by pond_destroy()
void pond_batch_detach(pond_ctx *c);

#define POND_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) {                              \
      (void)cudaGetLastError();                           \
      return POND_E_CUDA;                                 \
    }                                                     \
  } while (0)
