// pond_noalloc.cu -- pond_step_noalloc(): the FP64 time step for callers that
// cannot allocate device memory.
//
// pond_step() keeps a second state buffer and a status block in memory that a
// context allocates (or receives as a workspace).  Some callers may not call
// cudaMalloc at all.  For them this entry point advances a caller-owned
// device state in place and uses, as its only scratch, one file-scope
// __device__ array of POND_NOALLOC_SCRATCH_BYTES that every GPU loading this
// library holds until the process exits.  It calls no cudaMalloc, cudaFree or
// allocating library routine.
//
// The array is shared by every call on a device and keeps the last call's
// contents; the status block in it is cleared at the start of each call.
// Calls whose work overlaps on the GPU (other streams, other host threads)
// race on the array.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "pond.h"
#include "pond_internal.h"
#include "pond_kernels.cuh"

// the scratch: [status block (256 B)][one FP64 state buffer]
static __device__ __align__(256) unsigned char g_pond_noalloc_scratch[POND_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// Once per device, with that device current: the device address of the array
// (in host code its name is only a host-side stand-in) and the shared-memory
// opt-in of the step kernels this entry point launches.
pond_status scratch_for_current_device(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return POND_E_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pond_noalloc_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return POND_E_CUDA;
    }
    using T2 = pond::Tile<2, 8, 8>;
    using T1 = pond::Tile<1, 252, 1>;
    if (cudaFuncSetAttribute(pond::step_kernel<double, 2, 4, 8, 8, 160>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)T2::smem_bytes<double>()) != cudaSuccess ||
        cudaFuncSetAttribute(pond::step_kernel<double, 1, 4, 252, 1, 256>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)T1::smem_bytes<double>()) != cudaSuccess) {
      (void)cudaGetLastError();
      return POND_E_CUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_addr[dev];
  return POND_OK;
}

// In-place change of basis of the caller's FP64 planes: populations <-> their
// dimensional Hermite coefficients in the cell's frame (temperature T), the
// layout the step kernels keep the state in.  Each thread owns one cell and
// reads all of its values before writing.
template <int DIM, bool TO_COEF>
__global__ void noalloc_basis_kernel(double *f, double *g, const double *T, size_t N) {
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  using D = pond::Dims<DIM>;
  pond::Blk<double, 4, D::NYF> F;
  pond::Blk<double, 3, D::NYG> G;
  for (int q = 0; q < D::QF; ++q) F.v[q % 4][q / 4] = f[q * N + c];
  for (int q = 0; q < D::QG; ++q) G.v[q % 3][q / 3] = g[q * N + c];
  const double sT = sqrt(T[c]);
  if (TO_COEF) {
    pond::ana_x(F); pond::ana_y(F); pond::ana_x(G); pond::ana_y(G);
    pond::scale_orders(sT, F);
    pond::scale_orders(sT, G);
  } else {
    pond::scale_orders(1.0 / sT, F);
    pond::scale_orders(1.0 / sT, G);
    pond::syn_x(F); pond::syn_y(F); pond::syn_x(G); pond::syn_y(G);
  }
  for (int q = 0; q < D::QF; ++q) f[q * N + c] = F.v[q % 4][q / 4];
  for (int q = 0; q < D::QG; ++q) g[q * N + c] = G.v[q % 3][q / 3];
}

template <bool TO_COEF>
bool change_basis(int D, double *f, double *g, const double *T, size_t N, cudaStream_t st) {
  const unsigned nb = (unsigned)((N + 255) / 256);
  if (D == 2) noalloc_basis_kernel<2, TO_COEF><<<nb, 256, 0, st>>>(f, g, T, N);
  else noalloc_basis_kernel<1, TO_COEF><<<nb, 256, 0, st>>>(f, g, T, N);
  return cudaGetLastError() == cudaSuccess;
}

bool params_ok(const pond_params *p, int D) {
  if (!p || !(p->gamma > 1.0) || !(p->tau > 0.0) || !(p->prandtl > 0.0) || !(p->dx > 0.0) ||
      !(p->dt > 0.0))
    return false;
  for (int s = 0; s < 4; ++s) {
    if (p->bc[s] < POND_BC_PERIODIC || p->bc[s] > POND_BC_WALL) return false;
    // walls on the y sides in 2D (x sides periodic or zero-gradient), x sides in 1D
    if (p->bc[s] == POND_BC_WALL &&
        (D == 2 ? s < 2 || p->bc[0] == POND_BC_INFLOW || p->bc[1] == POND_BC_INFLOW : s > 1))
      return false;
  }
  if ((p->bc[0] == POND_BC_PERIODIC) != (p->bc[1] == POND_BC_PERIODIC)) return false;
  if (D == 2 && (p->bc[2] == POND_BC_PERIODIC) != (p->bc[3] == POND_BC_PERIODIC)) return false;
  return p->precision == POND_FP64 && (p->transform == POND_TENSOR || p->transform == POND_GRAD_K) &&
         (p->flux_form == POND_FLUX_MAIN || p->flux_form == POND_FLUX_APPC) &&
         (p->limiter == POND_VANLEER || p->limiter == POND_MINMOD) &&
         p->flux_frame == POND_FRAME_AVG && p->multiscale == 0 && p->g_same_as_f == 0;
}

}  // namespace

extern "C" pond_status pond_step_noalloc(pond_lattice lat, const int64_t dims[2],
                                         const pond_params *p, double *f, double *g, double *ux,
                                         double *uy, double *T, int64_t n, uint32_t *flags,
                                         void *stream) {
  if ((lat != POND_D1Q4 && lat != POND_D2Q16) || !dims || n < 0) return POND_E_INVAL;
  const int D = lat == POND_D2Q16 ? 2 : 1;
  const int64_t nx = dims[0], ny = D == 2 ? dims[1] : 1;
  if (nx < 2 || (D == 2 && ny < 2) || nx > (1 << 24) || ny > (1 << 24)) return POND_E_INVAL;
  for (int s = 0; s < 4; ++s)
    if (p && p->bc[s] == POND_BC_WALL && (D == 2 ? ny : nx) < 3) return POND_E_INVAL;
  if (!params_ok(p, D) || !f || !g || !ux || !T || (D == 2 && !uy)) return POND_E_INVAL;
  const size_t N = (size_t)(nx * ny), qf = D == 2 ? 16 : 4, qg = D == 2 ? 9 : 3;
  const size_t state_bytes = (qf + qg + 3) * N * sizeof(double);
  if (256 + state_bytes > (size_t)POND_NOALLOC_SCRATCH_BYTES) return POND_E_NOMEM;

  cudaStream_t st = (cudaStream_t)stream;
  if (flags) {
    // reading the flags synchronises the stream, which a stream capture
    // forbids (and would invalidate): flags must be NULL while capturing
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t qe = cudaStreamIsCapturing(st, &cs);
    if (qe != cudaSuccess) (void)cudaGetLastError();
    if (qe != cudaSuccess || cs != cudaStreamCaptureStatusNone) return POND_E_INVAL;
  }
  unsigned char *scratch = nullptr;
  pond_status s = scratch_for_current_device(&scratch);
  if (s != POND_OK) return s;
  pond::Stats *stats = reinterpret_cast<pond::Stats *>(scratch);
  double *buf = reinterpret_cast<double *>(scratch + 256);
  pond::State<double> caller{f, g, ux, D == 2 ? uy : buf + (qf + qg + 1) * N, T};
  pond::State<double> other{buf, buf + qf * N, buf + (qf + qg) * N, buf + (qf + qg + 1) * N,
                            buf + (qf + qg + 2) * N};
  if (cudaMemsetAsync(stats, 0, sizeof(pond::Stats), st) != cudaSuccess) {
    (void)cudaGetLastError();
    return POND_E_CUDA;
  }
  pond::StepConst K;
  pond_fill_step_const(K, *p, D, nx, ny, p->dt);
  if (n > 0 && !change_basis<true>(D, f, g, T, N, st)) return POND_E_CUDA;
  for (int64_t i = 0; i < n; ++i) {
    const pond::State<double> &in = (i & 1) ? other : caller;
    const pond::State<double> &out = (i & 1) ? caller : other;
    if (D == 2) {
      const dim3 grid((unsigned)((nx + 7) / 8), (unsigned)((ny + 7) / 8));
      pond::step_kernel<double, 2, 4, 8, 8, 160>
          <<<grid, 160, pond::Tile<2, 8, 8>::smem_bytes<double>(), st>>>(K, in, out, stats);
    } else {
      const dim3 grid((unsigned)((nx + 251) / 252), 1u);
      pond::step_kernel<double, 1, 4, 252, 1, 256>
          <<<grid, 256, pond::Tile<1, 252, 1>::smem_bytes<double>(), st>>>(K, in, out, stats);
    }
    if (cudaGetLastError() != cudaSuccess) return POND_E_CUDA;
  }
  if (n & 1) {
    // the state after an odd number of steps is in the scratch: copy it back
    const struct { double *dst; const double *src; size_t cnt; } cp[5] = {
        {f, other.f, qf * N}, {g, other.g, qg * N}, {ux, other.ux, N},
        {D == 2 ? uy : nullptr, other.uy, N}, {T, other.T, N}};
    for (const auto &c : cp) {
      if (!c.dst) continue;
      if (cudaMemcpyAsync(c.dst, c.src, c.cnt * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess) {
        (void)cudaGetLastError();
        return POND_E_CUDA;
      }
    }
  }
  if (n > 0 && !change_basis<false>(D, f, g, T, N, st)) return POND_E_CUDA;
  if (flags) {
    pond::Stats h;
    if (cudaMemcpyAsync(&h, stats, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      (void)cudaGetLastError();
      return POND_E_CUDA;
    }
    *flags = h.flags;
    if (h.flags & POND_FLAG_NONPHYSICAL) return POND_E_NONPHYSICAL;
  }
  return POND_OK;
}
