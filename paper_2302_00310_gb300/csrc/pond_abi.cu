// pond_abi.cu -- the C ABI of include/pond.h: contexts, device state, launches.
//
// Device state of a context (one workspace, 256-byte aligned sub-buffers):
//   [Stats block][one-member descriptor table][state buffer 0][state buffer 1]
// A state buffer holds, in the arithmetic type R of the context (double for
// POND_FP64, float for POND_FP32_MIXED), SoA arrays
//   f[Qf][N], g[Qg][N], ux[N], uy[N], T[N]          (N = nx*ny cells)
// where f and g are the dimensional Hermite coefficients of each cell's
// populations in its frame (ux, uy, T): B_ab = T^((a+b)/2) A_ab, with A_ab the
// Hermite coefficients sum_i phi_i He_a(c_ix) He_b(c_iy).  On the mixed path
// the FP64 conserved moments M[4][N] (rho, rho ux, rho uy, rho E) follow them
// (8-byte aligned).  The boundary exchanges populations: they are
// converted (in FP64) on the way in and out.  Steps ping-pong between the two
// buffers; between steps the idle buffer is used as staging at the boundary.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pond_internal.h"

using pond::State;
using pond::StepConst;
using pond::Stats;
using pond_detail::qf_of;
using pond_detail::qg_of;
using pond_detail::state_of;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// ---------------------------------------------------------------------------
// small kernels: initial equilibrium, moments, conversions, max |v|
// ---------------------------------------------------------------------------
// co-moving equilibria rho W (Eq. feqPond) and (C_v - D/2) T rho W
// (Eq. geqPond): their only nonzero Hermite coefficient is the zeroth
template <typename R, int DIM, int QF1, int QG1 = 3>
__global__ void init_kernel(const double *rho, const double *ux, const double *uy, const double *T,
                            State<R> S, size_t N, double gfac) {
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  const double r = rho[c], t = T[c], vx = ux[c], vy = DIM == 2 ? uy[c] : 0.0;
  for (int i = 0; i < (DIM == 2 ? QF1 * QF1 : QF1); ++i) S.f[i * N + c] = R(i == 0 ? r : 0.0);
  for (int i = 0; i < (DIM == 2 ? QG1 * QG1 : QG1); ++i) S.g[i * N + c] = R(i == 0 ? gfac * t * r : 0.0);
  S.ux[c] = R(vx);
  S.uy[c] = R(vy);
  S.T[c] = R(t);
  if (S.M) {  // C_v = gfac + D/2
    S.M[c] = r;
    S.M[N + c] = r * vx;
    S.M[2 * N + c] = r * vy;
    S.M[3 * N + c] = 0.5 * r * (vx * vx + vy * vy) + (gfac + 0.5 * DIM) * r * t;
  }
}

// rho, u, T of each cell (Eqs. eq::ConservationLaws, eq:E), in FP64: on the
// mixed path from its FP64 conserved moments, else from its dimensional
// Hermite coefficients: rho = B_00, rho (u - u_frame) = (B_10, B_01),
// sum |v - u_frame|^2 f = B_20 + B_02 + D T rho
template <typename R, int DIM, int QF1>
__global__ void moments_kernel(State<R> S, size_t N, double inv_cv, double *rho, double *ux,
                               double *uy, double *T) {
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  if (S.M) {
    const double r = S.M[c], vx = S.M[N + c] / r, vy = DIM == 2 ? S.M[2 * N + c] / r : 0.0;
    rho[c] = r;
    ux[c] = vx;
    if (uy) uy[c] = vy;
    T[c] = (S.M[3 * N + c] / r - 0.5 * (vx * vx + vy * vy)) * inv_cv;
    return;
  }
  const double fx = S.ux[c], fy = DIM == 2 ? (double)S.uy[c] : 0.0, fT = S.T[c];
  const double r = S.f[c], mx = (double)S.f[1 * N + c] / r;
  double my = 0.0, S2 = (double)S.f[2 * N + c] + DIM * fT * r;
  if constexpr (DIM == 2) { my = (double)S.f[QF1 * N + c] / r; S2 += (double)S.f[2 * QF1 * N + c]; }
  const double e = 0.5 * (S2 - r * (mx * mx + my * my)) + (double)S.g[c];
  rho[c] = r;
  ux[c] = fx + mx;
  if (uy) uy[c] = fy + my;
  T[c] = e / r * inv_cv;
}

// populations (FP64 planes p[i][ld], cells 0..n-1) <-> state coefficients
// (cells c0..c0+n-1) in the frame already stored for those cells; in place
// when the planes are the state's own (FP64)
template <typename R, int DIM, int QF1, int QG1 = 3>
__global__ void pops_to_coef_kernel(const double *pf, const double *pg, size_t ld, State<R> S,
                                    size_t N, size_t c0, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  using D = pond::Dims<DIM, QF1, QG1>;
  pond::Blk<double, QF1, D::NYF> F;
  pond::Blk<double, QG1, D::NYG> G;
  for (int q = 0; q < D::QF; ++q) F.v[q % QF1][q / QF1] = pf[q * ld + i];
  for (int q = 0; q < D::QG; ++q) G.v[q % QG1][q / QG1] = pg[q * ld + i];
  pond::ana_x(F); pond::ana_y(F); pond::ana_x(G); pond::ana_y(G);
  const double fT = S.T[c0 + i], sT = sqrt(fT);
  pond::scale_orders(sT, F);
  pond::scale_orders(sT, G);
  if (S.M) {  // mixed path: the conserved moments in FP64, v = u_frame + x
    const size_t c = c0 + i;
    const double fx = S.ux[c], fy = DIM == 2 ? (double)S.uy[c] : 0.0, r = F.v[0][0], bx = F.v[1][0];
    const double by = DIM == 2 ? F.v[0][1] : 0.0;
    double c2 = F.v[2][0] + DIM * fT * r;
    if constexpr (DIM == 2) c2 += F.v[0][2];
    S.M[c] = r;
    S.M[N + c] = fx * r + bx;
    S.M[2 * N + c] = fy * r + by;
    S.M[3 * N + c] = 0.5 * ((fx * fx + fy * fy) * r + 2.0 * (fx * bx + fy * by) + c2) + G.v[0][0];
  }
  for (int q = 0; q < D::QF; ++q) S.f[q * N + c0 + i] = R(F.v[q % QF1][q / QF1]);
  for (int q = 0; q < D::QG; ++q) S.g[q * N + c0 + i] = R(G.v[q % QG1][q / QG1]);
}
template <typename R, int DIM, int QF1, int QG1 = 3>
__global__ void coef_to_pops_kernel(State<R> S, size_t N, size_t c0, size_t n, double *pf,
                                    double *pg, size_t ld) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  using D = pond::Dims<DIM, QF1, QG1>;
  pond::Blk<double, QF1, D::NYF> F;
  pond::Blk<double, QG1, D::NYG> G;
  for (int q = 0; q < D::QF; ++q) F.v[q % QF1][q / QF1] = (double)S.f[q * N + c0 + i];
  for (int q = 0; q < D::QG; ++q) G.v[q % QG1][q / QG1] = (double)S.g[q * N + c0 + i];
  const double isT = 1.0 / sqrt((double)S.T[c0 + i]);
  pond::scale_orders(isT, F);
  pond::scale_orders(isT, G);
  pond::syn_x(F); pond::syn_y(F); pond::syn_x(G); pond::syn_y(G);
  for (int q = 0; q < D::QF; ++q) pf[q * ld + i] = F.v[q % QF1][q / QF1];
  for (int q = 0; q < D::QG; ++q) pg[q * ld + i] = G.v[q % QG1][q / QG1];
}

template <typename A, typename B>
__global__ void convert_kernel(const A *in, B *out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = B(in[i]);
}

// largest |v_i alpha| over cells for the CFL time step (Sec. V)
__global__ void vmax_kernel(const double *ux, const double *uy, const double *T, size_t N,
                            double cmax, unsigned long long *out) {
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (c < N) v = fmax(fabs(ux[c]), uy ? fabs(uy[c]) : 0.0) + sqrt(T[c]) * cmax;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

unsigned grid1(size_t n, unsigned b) { return (unsigned)((n + b - 1) / b); }

// ---------------------------------------------------------------------------
// step launches: the member step kernel with the context's one-member table,
// one CTA per tile (the same kernel function a batch runs)
// ---------------------------------------------------------------------------
// Picks the kernel instantiation, sets its shared-memory opt-in (outside any
// stream capture) and uploads the table.  Called whenever K changes.
pond_status prepare_step(pond_ctx *c) {
  if (c->K.ms) {
    c->shape = c->fp32 ? pond_ms_shape_fp32(c->D) : pond_ms_shape_fp64(c->D);
  } else if (c->qg1 == 4) {
    c->shape = c->fp32 ? pond_g4_shape_fp32(c->D) : pond_g4_shape_fp64(c->D);
  } else if (c->K.iterative) {
    if (c->qf1 == 5) c->shape = c->fp32 ? pond_iter_shape_fp32_q5() : pond_iter_shape_fp64_q5();
    else c->shape = c->fp32 ? pond_iter_shape_fp32(c->D) : pond_iter_shape_fp64(c->D);
  } else {
    const std::vector<pond::Shape> all =
        c->qf1 == 5 ? (c->fp32 ? pond_shapes_fp32_q5() : pond_shapes_fp64_q5())
                    : (c->fp32 ? pond_shapes_fp32(c->D) : pond_shapes_fp64(c->D));
    bool found = false;
    for (const pond::Shape &sh : all)
      if (sh.code == c->tile) { c->shape = sh; found = true; }
    if (!found) return POND_E_INVAL;
  }
  int occ = 0, dev = 0, sms = 0;
  POND_CUDA(c->shape.prepare(&occ));
  POND_CUDA(cudaGetDevice(&dev));
  POND_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int tx = (int)((c->nx + c->shape.bx - 1) / c->shape.bx);
  const int ty = c->D == 2 ? (int)((c->ny + c->shape.by - 1) / c->shape.by) : 1;
  // one CTA per strip of tiles (the iterated face frame hands no edges over)
  const int strip = c->K.iterative ? 1
                   : c->p.strip > 0 ? (c->p.strip < tx ? c->p.strip : tx)
                                    : pond::choose_strip(tx, ty, sms * (occ > 0 ? occ : 1));
  c->tiles = pond::strips_of(tx, ty, strip);
  unsigned char host[pond::kSoloTableBytes];
  memset(host, 0, sizeof(host));
  pond::TableHdr hdr;
  memset(&hdr, 0, sizeof(hdr));
  hdr.n = 1;
  hdr.total_tiles = c->tiles;
  hdr.strip = strip;
  memcpy(host, &hdr, sizeof(hdr));
  auto fill = [&](auto tag) {
    using R = decltype(tag);
    pond::InstDesc<R> d;
    memset(&d, 0, sizeof(d));
    d.K = c->K;
    d.S[0] = state_of<R>(c, 0);
    d.S[1] = state_of<R>(c, 1);
    d.stats = c->stats;
    d.tiles_x = tx;
    d.tile_begin = 0;
    d.steps = 0x7fffffff;
    d.parity = 0;  // launch k = c->cur reads buffer cur
    memcpy(host + sizeof(hdr), &d, sizeof(d));
  };
  if (c->fp32) fill(0.0f);
  else fill(0.0);
  POND_CUDA(cudaMemcpyAsync(c->table, host, sizeof(host), cudaMemcpyHostToDevice, c->stream));
  POND_CUDA(cudaStreamSynchronize(c->stream));  // the host copy goes out of scope
  return POND_OK;
}

pond_status step_once(pond_ctx *c) {
  c->shape.launch(c->table, c->cur, c->tiles, c->stream);
  POND_CUDA(cudaGetLastError());
  c->cur ^= 1;
  return POND_OK;
}

// Fastest in tile sweeps on GB300 (256^2 pulse and 1024^2 Riemann grids):
// 8x14 tiles with 128 threads and two CTAs per SM in both precisions (FP64:
// shared memory and the register file each hold exactly two; mixed: 1,421
// and 1,518 MLUPS against 1,247 and 1,476 for 8x16 tiles with 160 threads).
// On the mixed path a grid of at least four waves of three CTAs per SM takes
// the same tile with registers capped for three CTAs (code 11: 1,987 against
// 1,750 MLUPS on the 1024^2 Riemann problem; on the 256^2 pulse, 1.3 waves,
// 1,451 against 1,563).  (D2Q25: 8x8 tiles with 128 threads, two CTAs per SM.)
// The multiscale and g-on-f kernels have the one shape code 10.
int auto_tile(const pond_ctx *c) {
  if (c->D == 1) return 1;
  if (!c->fp32 || c->qf1 == 5 || c->p.multiscale || c->qg1 == 4) return 10;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return 10;
  }
  const long long tiles = (long long)((c->nx + 7) / 8) * (long long)((c->ny + 13) / 14);
  return tiles >= 4LL * 3 * sms ? 11 : 10;
}

bool valid_params(const pond_params *p) {
  if (!p) return false;
  if (!(p->gamma > 1.0) || !(p->tau > 0.0) || !(p->prandtl > 0.0) || !(p->dx > 0.0)) return false;
  if (!(p->dt > 0.0) && !(p->cfl > 0.0)) return false;
  for (int s = 0; s < 4; ++s)
    if (p->bc[s] < POND_BC_PERIODIC || p->bc[s] > POND_BC_WALL) return false;
  if ((p->bc[0] == POND_BC_PERIODIC) != (p->bc[1] == POND_BC_PERIODIC)) return false;
  if ((p->bc[2] == POND_BC_PERIODIC) != (p->bc[3] == POND_BC_PERIODIC)) return false;
  if (p->precision != POND_FP64 && p->precision != POND_FP32_MIXED) return false;
  if (p->transform != POND_TENSOR && p->transform != POND_GRAD_K) return false;
  if (p->flux_form != POND_FLUX_MAIN && p->flux_form != POND_FLUX_APPC) return false;
  if (p->limiter != POND_VANLEER && p->limiter != POND_MINMOD) return false;
  if (p->flux_frame != POND_FRAME_AVG && p->flux_frame != POND_FRAME_ITER) return false;
  if (p->flux_frame == POND_FRAME_ITER && (!(p->iter_tol > 0.0) || p->iter_max < 1)) return false;
  if (!(p->xi_fp64_threshold > 0.0)) return false;
  if (p->tile < 0 || p->tile > 11) return false;
  if (p->tile == 11 && p->precision != POND_FP32_MIXED) return false;  // a mixed-path shape
  if (p->strip < 0 || p->strip > 8) return false;
  if (p->multiscale != 0 && p->multiscale != 1) return false;
  if (p->g_same_as_f != 0 && p->g_same_as_f != 1) return false;
  if (p->multiscale) {  // D1Q3/D1Q4 and D2Q9/D2Q16, averaged frame
    if (p->flux_frame != POND_FRAME_AVG) return false;
    if (std::isnan(p->ms_theta_u) || std::isnan(p->ms_theta_T)) return false;
  }
  return true;
}

// walls: on the y sides in 2D (the x sides then periodic or zero-gradient),
// on the x sides in 1D, with at least three cells across
bool walls_ok(const pond_params *p, int D, int64_t nx, int64_t ny) {
  for (int s = 0; s < 4; ++s) {
    if (p->bc[s] != POND_BC_WALL) continue;
    if (D == 2 && (s < 2 || ny < 3 || p->bc[0] == POND_BC_INFLOW || p->bc[1] == POND_BC_INFLOW))
      return false;
    if (D == 1 && (s > 1 || nx < 3)) return false;
  }
  return true;
}

void set_step_const(pond_ctx *c) { pond_fill_step_const(c->K, c->p, c->D, c->nx, c->ny, c->dt); }

void drop_graphs(pond_ctx *c) {
  for (int i = 0; i < 2; ++i)
    if (c->graph[i]) { cudaGraphExecDestroy(c->graph[i]); c->graph[i] = nullptr; }
}

// captures `chunk` consecutive steps starting from buffer `from`
pond_status build_graph(pond_ctx *c, int from, int chunk) {
  cudaGraph_t g = nullptr;
  const int save = c->cur;
  c->cur = from;
  POND_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  pond_status s = POND_OK;
  for (int i = 0; i < chunk && s == POND_OK; ++i) s = step_once(c);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  c->cur = save;
  if (s != POND_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    (void)cudaGetLastError();
    return s != POND_OK ? s : POND_E_CUDA;
  }
  e = cudaGraphInstantiate(&c->graph[from], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { (void)cudaGetLastError(); return POND_E_CUDA; }
  return POND_OK;
}

template <typename T>
pond_status to_device(pond_ctx *c, const T *src, T *dst, size_t n, int on_device) {
  POND_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(T), on_device ? cudaMemcpyDeviceToDevice
                                                                 : cudaMemcpyHostToDevice,
                            c->stream));
  return POND_OK;
}

// converts cells [c0, c0 + n) between populations p[i][ld] and the state
template <typename R>
pond_status convert_pops(pond_ctx *c, double *pf, double *pg, size_t ld, size_t c0, size_t n,
                                bool to_state) {
  const size_t N = (size_t)c->N;
  const unsigned nb = grid1(n, 256);
  const State<R> S = state_of<R>(c, c->cur);
  if (to_state) {
    if (c->qg1 == 4 && c->D == 2) pops_to_coef_kernel<R, 2, 4, 4><<<nb, 256, 0, c->stream>>>(pf, pg, ld, S, N, c0, n);
    else if (c->qg1 == 4) pops_to_coef_kernel<R, 1, 4, 4><<<nb, 256, 0, c->stream>>>(pf, pg, ld, S, N, c0, n);
    else if (c->qf1 == 5) pops_to_coef_kernel<R, 2, 5><<<nb, 256, 0, c->stream>>>(pf, pg, ld, S, N, c0, n);
    else if (c->D == 2) pops_to_coef_kernel<R, 2, 4><<<nb, 256, 0, c->stream>>>(pf, pg, ld, S, N, c0, n);
    else pops_to_coef_kernel<R, 1, 4><<<nb, 256, 0, c->stream>>>(pf, pg, ld, S, N, c0, n);
  } else {
    if (c->qg1 == 4 && c->D == 2) coef_to_pops_kernel<R, 2, 4, 4><<<nb, 256, 0, c->stream>>>(S, N, c0, n, pf, pg, ld);
    else if (c->qg1 == 4) coef_to_pops_kernel<R, 1, 4, 4><<<nb, 256, 0, c->stream>>>(S, N, c0, n, pf, pg, ld);
    else if (c->qf1 == 5) coef_to_pops_kernel<R, 2, 5><<<nb, 256, 0, c->stream>>>(S, N, c0, n, pf, pg, ld);
    else if (c->D == 2) coef_to_pops_kernel<R, 2, 4><<<nb, 256, 0, c->stream>>>(S, N, c0, n, pf, pg, ld);
    else coef_to_pops_kernel<R, 1, 4><<<nb, 256, 0, c->stream>>>(S, N, c0, n, pf, pg, ld);
  }
  POND_CUDA(cudaGetLastError());
  return POND_OK;
}

}  // namespace

// ===========================================================================
// exported ABI
// ===========================================================================
extern "C" {

int pond_abi_version(void) { return POND_ABI_VERSION; }

void pond_params_default(pond_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->gamma = 1.4;
  p->tau = 1e-4;
  p->prandtl = 1.0;
  p->dx = 1.0;
  p->dt = 0.0;
  p->cfl = 0.2;
  for (int s = 0; s < 4; ++s) p->bc[s] = POND_BC_PERIODIC;
  p->precision = POND_FP64;
  p->transform = POND_TENSOR;
  p->flux_form = POND_FLUX_MAIN;
  p->limiter = POND_VANLEER;
  p->flux_frame = POND_FRAME_AVG;
  p->iter_tol = 1e-12;
  p->iter_max = 10;
  p->xi_fp64_threshold = 8.0;
  p->tile = 0;
}

const char *pond_strerror(pond_status s) {
  switch (s) {
    case POND_OK: return "ok";
    case POND_E_INVAL: return "invalid argument";
    case POND_E_NOMEM: return "out of device memory or workspace too small";
    case POND_E_CUDA: return "CUDA runtime error";
    case POND_E_NONPHYSICAL: return "nonphysical state (rho <= 0, T <= 0 or NaN)";
    case POND_E_NOCONV: return "iterated face frame did not converge";
    case POND_E_CFL: return "CFL number above 1";
    case POND_E_STATE: return "call out of order";
  }
  return "unknown status";
}

pond_status pond_workspace_size(pond_lattice lat, const int64_t dims[2], const pond_params *p,
                                size_t *bytes) {
  if (!dims || !bytes || !p || (lat != POND_D1Q4 && lat != POND_D2Q16 && lat != POND_D2Q25))
    return POND_E_INVAL;
  const int D = lat == POND_D1Q4 ? 1 : 2;
  const int64_t nx = dims[0], ny = D == 2 ? dims[1] : 1;
  if (nx < 2 || (D == 2 && ny < 2) || nx > (1 << 24) || ny > (1 << 24)) return POND_E_INVAL;
  const bool fp32 = p->precision == POND_FP32_MIXED;
  *bytes = align_up(sizeof(Stats)) + pond::kSoloTableBytes +
           2 * align_up(pond_detail::state_bytes(D, fp32, (size_t)(nx * ny), pond_detail::qf1_of(lat),
                                                 pond_detail::qg1_of(p)));
  return POND_OK;
}

pond_status pond_create(pond_ctx **out, pond_lattice lat, const int64_t dims[2],
                        const pond_params *p, void *workspace, size_t workspace_bytes,
                        void *stream) {
  if (!out) return POND_E_INVAL;
  *out = nullptr;
  size_t need = 0;
  pond_status s = pond_workspace_size(lat, dims, p, &need);
  if (s != POND_OK) return s;
  if (!valid_params(p)) return POND_E_INVAL;
  const int D = lat == POND_D1Q4 ? 1 : 2;
  if (!walls_ok(p, D, dims[0], D == 2 ? dims[1] : 1)) return POND_E_INVAL;
  if (D == 1 && p->tile > 1) return POND_E_INVAL;
  if (D == 2 && p->tile == 1) return POND_E_INVAL;
  if (lat == POND_D2Q25 && p->tile != 0 && p->tile != 2 && p->tile != 10) return POND_E_INVAL;
  if (p->multiscale && (lat == POND_D2Q25 || (p->tile != 0 && p->tile != (D == 1 ? 1 : 10))))
    return POND_E_INVAL;
  if (p->g_same_as_f && (lat == POND_D2Q25 || p->multiscale || p->flux_frame != POND_FRAME_AVG ||
                         (p->tile != 0 && p->tile != (D == 1 ? 1 : 10))))
    return POND_E_INVAL;
  if (workspace && (workspace_bytes < need || ((uintptr_t)workspace % kAlign) != 0))
    return POND_E_NOMEM;
  pond_ctx *c = new (std::nothrow) pond_ctx();
  if (!c) return POND_E_NOMEM;
  c->lat = lat;
  c->D = D;
  c->qf1 = pond_detail::qf1_of(lat);
  c->qg1 = pond_detail::qg1_of(p);
  c->nx = dims[0];
  c->ny = D == 2 ? dims[1] : 1;
  c->N = c->nx * c->ny;
  c->p = *p;
  c->fp32 = p->precision == POND_FP32_MIXED;
  c->stream = (cudaStream_t)stream;
  if (workspace) {
    c->ws = (unsigned char *)workspace;
    c->own_ws = false;
  } else {
    if (cudaMalloc((void **)&c->ws, need) != cudaSuccess) {
      (void)cudaGetLastError();
      delete c;
      return POND_E_NOMEM;
    }
    c->own_ws = true;
  }
  c->ws_bytes = need;
  c->stats = reinterpret_cast<Stats *>(c->ws);
  c->table = c->ws + align_up(sizeof(Stats));
  c->buf_bytes = (need - align_up(sizeof(Stats)) - pond::kSoloTableBytes) / 2;
  c->buf[0] = c->table + pond::kSoloTableBytes;
  c->buf[1] = c->buf[0] + c->buf_bytes;
  c->cur = 0;
  c->tile = p->flux_frame == POND_FRAME_ITER ? (D == 1 ? 1 : 2) : (p->tile ? p->tile : auto_tile(c));
  c->graph_chunk = 8;
  if (cudaMemsetAsync(c->stats, 0, sizeof(Stats), c->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    pond_destroy(c);
    return POND_E_CUDA;
  }
  *out = c;
  return POND_OK;
}

void pond_destroy(pond_ctx *c) {
  if (!c) return;
  pond_batch_detach(c);
  cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  if (c->own_ws && c->ws) cudaFree(c->ws);
  (void)cudaGetLastError();
  delete c;
}

pond_status pond_init(pond_ctx *c, const double *rho, const double *ux, const double *uy,
                      const double *T, int on_device) {
  if (!c || !rho || !ux || !T || (c->D == 2 && !uy)) return POND_E_INVAL;
  const size_t N = (size_t)c->N;
  // stage the primitive fields (FP64) in the idle buffer
  double *st = reinterpret_cast<double *>(c->buf[1 - c->cur]);
  double *srho = st, *sux = st + N, *suy = st + 2 * N, *sT = st + 3 * N;
  pond_status s;
  if ((s = to_device(c, rho, srho, N, on_device)) != POND_OK) return s;
  if ((s = to_device(c, ux, sux, N, on_device)) != POND_OK) return s;
  if (c->D == 2 && (s = to_device(c, uy, suy, N, on_device)) != POND_OK) return s;
  if ((s = to_device(c, T, sT, N, on_device)) != POND_OK) return s;
  POND_CUDA(cudaMemsetAsync(c->stats, 0, sizeof(Stats), c->stream));
  const double gfac = 1.0 / (c->p.gamma - 1.0) - 0.5 * c->D;
  const unsigned nb = grid1(N, 256);
  if (c->qg1 == 4) {
    const double *uy2 = c->D == 2 ? suy : nullptr;
    if (c->D == 2 && c->fp32) init_kernel<float, 2, 4, 4><<<nb, 256, 0, c->stream>>>(srho, sux, uy2, sT, state_of<float>(c, c->cur), N, gfac);
    else if (c->D == 2) init_kernel<double, 2, 4, 4><<<nb, 256, 0, c->stream>>>(srho, sux, uy2, sT, state_of<double>(c, c->cur), N, gfac);
    else if (c->fp32) init_kernel<float, 1, 4, 4><<<nb, 256, 0, c->stream>>>(srho, sux, uy2, sT, state_of<float>(c, c->cur), N, gfac);
    else init_kernel<double, 1, 4, 4><<<nb, 256, 0, c->stream>>>(srho, sux, uy2, sT, state_of<double>(c, c->cur), N, gfac);
  } else if (c->D == 2) {
    if (c->qf1 == 5) {
      if (c->fp32) init_kernel<float, 2, 5><<<nb, 256, 0, c->stream>>>(srho, sux, suy, sT, state_of<float>(c, c->cur), N, gfac);
      else init_kernel<double, 2, 5><<<nb, 256, 0, c->stream>>>(srho, sux, suy, sT, state_of<double>(c, c->cur), N, gfac);
    } else if (c->fp32) init_kernel<float, 2, 4><<<nb, 256, 0, c->stream>>>(srho, sux, suy, sT, state_of<float>(c, c->cur), N, gfac);
    else init_kernel<double, 2, 4><<<nb, 256, 0, c->stream>>>(srho, sux, suy, sT, state_of<double>(c, c->cur), N, gfac);
  } else {
    if (c->fp32) init_kernel<float, 1, 4><<<nb, 256, 0, c->stream>>>(srho, sux, nullptr, sT, state_of<float>(c, c->cur), N, gfac);
    else init_kernel<double, 1, 4><<<nb, 256, 0, c->stream>>>(srho, sux, nullptr, sT, state_of<double>(c, c->cur), N, gfac);
  }
  POND_CUDA(cudaGetLastError());
  c->dt = c->p.dt;
  if (!(c->dt > 0.0)) {
    unsigned long long *slot = &c->stats->noconv;  // borrowed before the counters are reset
    POND_CUDA(cudaMemsetAsync(slot, 0, sizeof(*slot), c->stream));
    vmax_kernel<<<nb, 256, 0, c->stream>>>(sux, c->D == 2 ? suy : nullptr, sT, N,
                                           c->qf1 == 5 ? pond::Nodes<5>::cmax : pond::Nodes<4>::cmax, slot);
    POND_CUDA(cudaGetLastError());
    unsigned long long bits = 0;
    POND_CUDA(cudaMemcpyAsync(&bits, slot, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
    POND_CUDA(cudaStreamSynchronize(c->stream));
    double vmax;
    memcpy(&vmax, &bits, sizeof(vmax));
    if (!(vmax > 0.0) || !std::isfinite(vmax)) return POND_E_INVAL;
    c->dt = c->p.cfl * c->p.dx / vmax;
    POND_CUDA(cudaMemsetAsync(slot, 0, sizeof(*slot), c->stream));
  }
  set_step_const(c);
  drop_graphs(c);
  if ((s = prepare_step(c)) != POND_OK) return s;
  c->steps = 0;
  c->inited = true;
  POND_CUDA(cudaStreamSynchronize(c->stream));
  return POND_OK;
}

pond_status pond_step(pond_ctx *c, int64_t n) {
  if (!c || n < 0) return POND_E_INVAL;
  if (!c->inited) return POND_E_STATE;
  // stream capture is not possible on the legacy default stream: launch directly there
  const int chunk = c->stream ? c->graph_chunk : 0;
  int64_t done = 0;
  while (chunk > 0 && n - done >= chunk) {
    if (!c->graph[c->cur]) {
      pond_status s = build_graph(c, c->cur, chunk);
      if (s != POND_OK) return s;
    }
    POND_CUDA(cudaGraphLaunch(c->graph[c->cur], c->stream));
    if (chunk & 1) c->cur ^= 1;
    done += chunk;
  }
  for (; done < n; ++done) {
    pond_status s = step_once(c);
    if (s != POND_OK) return s;
  }
  c->steps += n;
  return POND_OK;
}

pond_status pond_moments(pond_ctx *c, double *rho, double *ux, double *uy, double *T,
                         int on_device) {
  if (!c || !rho || !ux || !T) return POND_E_INVAL;
  if (!c->inited) return POND_E_STATE;
  const size_t N = (size_t)c->N;
  double *out[4];
  double *st = reinterpret_cast<double *>(c->buf[1 - c->cur]);
  if (on_device) {
    out[0] = rho; out[1] = ux; out[2] = uy; out[3] = T;
  } else {
    out[0] = st; out[1] = st + N; out[2] = st + 2 * N; out[3] = st + 3 * N;
  }
  if (c->D == 1) out[2] = nullptr;
  const double inv_cv = c->p.gamma - 1.0;
  const unsigned nb = grid1(N, 256);
  if (c->D == 2) {
    if (c->qf1 == 5) {
      if (c->fp32) moments_kernel<float, 2, 5><<<nb, 256, 0, c->stream>>>(state_of<float>(c, c->cur), N, inv_cv, out[0], out[1], out[2], out[3]);
      else moments_kernel<double, 2, 5><<<nb, 256, 0, c->stream>>>(state_of<double>(c, c->cur), N, inv_cv, out[0], out[1], out[2], out[3]);
    } else if (c->fp32) moments_kernel<float, 2, 4><<<nb, 256, 0, c->stream>>>(state_of<float>(c, c->cur), N, inv_cv, out[0], out[1], out[2], out[3]);
    else moments_kernel<double, 2, 4><<<nb, 256, 0, c->stream>>>(state_of<double>(c, c->cur), N, inv_cv, out[0], out[1], out[2], out[3]);
  } else {
    if (c->fp32) moments_kernel<float, 1, 4><<<nb, 256, 0, c->stream>>>(state_of<float>(c, c->cur), N, inv_cv, out[0], out[1], out[2], out[3]);
    else moments_kernel<double, 1, 4><<<nb, 256, 0, c->stream>>>(state_of<double>(c, c->cur), N, inv_cv, out[0], out[1], out[2], out[3]);
  }
  POND_CUDA(cudaGetLastError());
  if (!on_device) {
    POND_CUDA(cudaMemcpyAsync(rho, out[0], N * 8, cudaMemcpyDeviceToHost, c->stream));
    POND_CUDA(cudaMemcpyAsync(ux, out[1], N * 8, cudaMemcpyDeviceToHost, c->stream));
    if (c->D == 2 && uy) POND_CUDA(cudaMemcpyAsync(uy, out[2], N * 8, cudaMemcpyDeviceToHost, c->stream));
    POND_CUDA(cudaMemcpyAsync(T, out[3], N * 8, cudaMemcpyDeviceToHost, c->stream));
  }
  POND_CUDA(cudaStreamSynchronize(c->stream));
  return POND_OK;
}

// copies one FP64 boundary array to/from state component `comp` (n values)
static pond_status xfer(pond_ctx *c, double *ext, size_t comp_off, size_t n, bool to_state,
                        int on_device) {
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (!c->fp32) {
    double *dst = reinterpret_cast<double *>(c->buf[c->cur]) + comp_off;
    if (to_state) POND_CUDA(cudaMemcpyAsync(dst, ext, n * 8, kin, c->stream));
    else POND_CUDA(cudaMemcpyAsync(ext, dst, n * 8, kout, c->stream));
    return POND_OK;
  }
  float *st = reinterpret_cast<float *>(c->buf[c->cur]) + comp_off;
  double *stage = reinterpret_cast<double *>(c->buf[1 - c->cur]);
  const unsigned nb = grid1(n, 256);
  if (to_state) {
    POND_CUDA(cudaMemcpyAsync(stage, ext, n * 8, kin, c->stream));
    convert_kernel<double, float><<<nb, 256, 0, c->stream>>>(stage, st, n);
    POND_CUDA(cudaGetLastError());
  } else {
    convert_kernel<float, double><<<nb, 256, 0, c->stream>>>(st, stage, n);
    POND_CUDA(cudaGetLastError());
    POND_CUDA(cudaMemcpyAsync(ext, stage, n * 8, kout, c->stream));
  }
  // the staging buffer is reused by the next component
  POND_CUDA(cudaStreamSynchronize(c->stream));
  return POND_OK;
}

// populations in or out: device arrays are converted directly; host arrays go
// through the idle state buffer in chunks of cells
static pond_status pops_io(pond_ctx *c, double *f, double *g, bool to_state, int on_device) {
  const size_t N = (size_t)c->N, qf = qf_of(c->D, c->qf1), qg = qg_of(c->D, c->qg1);
  auto conv = [&](double *pf, double *pg, size_t ld, size_t c0, size_t n) {
    return c->fp32 ? convert_pops<float>(c, pf, pg, ld, c0, n, to_state)
                   : convert_pops<double>(c, pf, pg, ld, c0, n, to_state);
  };
  if (on_device) return conv(f, g, N, 0, N);
  double *stage = reinterpret_cast<double *>(c->buf[1 - c->cur]);
  size_t chunk = c->buf_bytes / ((qf + qg) * sizeof(double));
  if (chunk > N) chunk = N;
  pond_status s;
  for (size_t c0 = 0; c0 < N; c0 += chunk) {
    const size_t n = chunk < N - c0 ? chunk : N - c0;
    double *sf = stage, *sg = stage + qf * n;
    if (to_state) {
      for (size_t q = 0; q < qf; ++q)
        POND_CUDA(cudaMemcpyAsync(sf + q * n, f + q * N + c0, n * 8, cudaMemcpyHostToDevice, c->stream));
      for (size_t q = 0; q < qg; ++q)
        POND_CUDA(cudaMemcpyAsync(sg + q * n, g + q * N + c0, n * 8, cudaMemcpyHostToDevice, c->stream));
      if ((s = conv(sf, sg, n, c0, n)) != POND_OK) return s;
    } else {
      if ((s = conv(sf, sg, n, c0, n)) != POND_OK) return s;
      for (size_t q = 0; q < qf; ++q)
        POND_CUDA(cudaMemcpyAsync(f + q * N + c0, sf + q * n, n * 8, cudaMemcpyDeviceToHost, c->stream));
      for (size_t q = 0; q < qg; ++q)
        POND_CUDA(cudaMemcpyAsync(g + q * N + c0, sg + q * n, n * 8, cudaMemcpyDeviceToHost, c->stream));
    }
  }
  return POND_OK;
}

static pond_status state_io(pond_ctx *c, double *f, double *g, double *ux, double *uy, double *T,
                            bool to_state, int on_device) {
  if (!c || !f || !g || !ux || !T || (c->D == 2 && !uy)) return POND_E_INVAL;
  const size_t N = (size_t)c->N, qf = qf_of(c->D, c->qf1), qg = qg_of(c->D, c->qg1);
  pond_status s;
  // the frame goes in before the populations, whose coefficients are taken in it
  if (!to_state && (s = pops_io(c, f, g, to_state, on_device)) != POND_OK) return s;
  // the staging buffer is shared by the populations and the frame planes
  POND_CUDA(cudaStreamSynchronize(c->stream));
  if ((s = xfer(c, ux, (qf + qg) * N, N, to_state, on_device)) != POND_OK) return s;
  if (c->D == 2 && (s = xfer(c, uy, (qf + qg + 1) * N, N, to_state, on_device)) != POND_OK) return s;
  if ((s = xfer(c, T, (qf + qg + 2) * N, N, to_state, on_device)) != POND_OK) return s;
  if (to_state && (s = pops_io(c, f, g, to_state, on_device)) != POND_OK) return s;
  POND_CUDA(cudaStreamSynchronize(c->stream));
  return POND_OK;
}

pond_status pond_get_state(pond_ctx *c, double *f, double *g, double *ux, double *uy, double *T,
                           int on_device) {
  if (!c) return POND_E_INVAL;
  if (!c->inited) return POND_E_STATE;
  return state_io(c, f, g, ux, uy, T, false, on_device);
}

pond_status pond_set_state(pond_ctx *c, const double *f, const double *g, const double *ux,
                           const double *uy, const double *T, int on_device) {
  if (!c) return POND_E_INVAL;
  if (!c->inited) {
    // a state given directly still needs a time step
    if (!(c->p.dt > 0.0)) return POND_E_STATE;
    c->dt = c->p.dt;
    set_step_const(c);
    pond_status s0 = prepare_step(c);
    if (s0 != POND_OK) return s0;
  }
  if (c->D == 1) {
    // keep the unused uy plane defined
    if (c->fp32) POND_CUDA(cudaMemsetAsync(state_of<float>(c, c->cur).uy, 0, c->N * 4, c->stream));
    else POND_CUDA(cudaMemsetAsync(state_of<double>(c, c->cur).uy, 0, c->N * 8, c->stream));
  }
  pond_status s = state_io(c, const_cast<double *>(f), const_cast<double *>(g),
                           const_cast<double *>(ux), const_cast<double *>(uy),
                           const_cast<double *>(T), true, on_device);
  if (s != POND_OK) return s;
  drop_graphs(c);
  c->steps = 0;
  c->inited = true;
  return POND_OK;
}

pond_status pond_status_flags(pond_ctx *c, uint32_t *flags, double *max_cfl, int64_t *noconv) {
  if (!c) return POND_E_INVAL;
  Stats h;
  POND_CUDA(cudaMemcpyAsync(&h, c->stats, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  POND_CUDA(cudaStreamSynchronize(c->stream));
  if (flags) *flags = h.flags;
  if (max_cfl) memcpy(max_cfl, &h.max_cfl_bits, sizeof(double));
  if (noconv) *noconv = (int64_t)h.noconv;
  return (h.flags & POND_FLAG_NONPHYSICAL) ? POND_E_NONPHYSICAL : POND_OK;
}

pond_status pond_iter_stats(pond_ctx *c, int64_t *face_evals, int64_t *traces, int32_t *max_traces) {
  if (!c) return POND_E_INVAL;
  Stats h;
  POND_CUDA(cudaMemcpyAsync(&h, c->stats, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  POND_CUDA(cudaStreamSynchronize(c->stream));
  if (face_evals) *face_evals = (int64_t)h.face_evals;
  if (traces) *traces = (int64_t)h.traces;
  if (max_traces) *max_traces = (int32_t)h.max_traces;
  return POND_OK;
}

pond_status pond_ms_stats(pond_ctx *c, int64_t *high_cell_updates) {
  if (!c) return POND_E_INVAL;
  Stats h;
  POND_CUDA(cudaMemcpyAsync(&h, c->stats, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  POND_CUDA(cudaStreamSynchronize(c->stream));
  if (high_cell_updates) *high_cell_updates = (int64_t)h.ms_high;
  return POND_OK;
}

pond_status pond_reset_flags(pond_ctx *c) {
  if (!c) return POND_E_INVAL;
  POND_CUDA(cudaMemsetAsync(c->stats, 0, sizeof(Stats), c->stream));
  return POND_OK;
}

pond_status pond_sync(pond_ctx *c) {
  if (!c) return POND_E_INVAL;
  POND_CUDA(cudaStreamSynchronize(c->stream));
  return POND_OK;
}

pond_status pond_info(pond_ctx *c, double *dt, int64_t *steps, int32_t *tile) {
  if (!c) return POND_E_INVAL;
  if (dt) *dt = c->dt;
  if (steps) *steps = c->steps;
  if (tile) *tile = c->tile;
  return POND_OK;
}

// ---- checkpoint / restore: the raw state (coefficients and frame in the
// context's arithmetic), the step counter, the time step and the status block
namespace {
struct CkptHdr {
  char magic[8];
  int32_t abi, D, fp32, pad;
  int64_t nx, ny, steps;
  double dt;
  Stats stats;
  uint64_t state_bytes;
};
size_t state_bytes_of(const pond_ctx *c) {
  return pond_detail::state_bytes(c->D, c->fp32, (size_t)c->N, c->qf1, c->qg1);
}
const char kCkptMagic[8] = {'P', 'O', 'N', 'D', 'C', 'K', 'P', '1'};
}  // namespace

pond_status pond_checkpoint_size(pond_ctx *c, size_t *bytes) {
  if (!c || !bytes) return POND_E_INVAL;
  *bytes = sizeof(CkptHdr) + state_bytes_of(c);
  return POND_OK;
}

pond_status pond_checkpoint(pond_ctx *c, void *host, size_t bytes) {
  if (!c || !host) return POND_E_INVAL;
  if (!c->inited) return POND_E_STATE;
  const size_t sb = state_bytes_of(c);
  if (bytes < sizeof(CkptHdr) + sb) return POND_E_INVAL;
  CkptHdr h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kCkptMagic, 8);
  h.abi = POND_ABI_VERSION;
  h.D = c->D;
  h.fp32 = c->fp32 ? 1 : 0;
  h.nx = c->nx;
  h.ny = c->ny;
  h.steps = c->steps;
  h.dt = c->dt;
  h.state_bytes = sb;
  unsigned char *dst = static_cast<unsigned char *>(host);
  POND_CUDA(cudaMemcpyAsync(&h.stats, c->stats, sizeof(Stats), cudaMemcpyDeviceToHost, c->stream));
  POND_CUDA(cudaMemcpyAsync(dst + sizeof(CkptHdr), c->buf[c->cur], sb, cudaMemcpyDeviceToHost, c->stream));
  POND_CUDA(cudaStreamSynchronize(c->stream));
  memcpy(dst, &h, sizeof(h));
  return POND_OK;
}

pond_status pond_restore(pond_ctx *c, const void *host, size_t bytes) {
  if (!c || !host || bytes < sizeof(CkptHdr)) return POND_E_INVAL;
  CkptHdr h;
  memcpy(&h, host, sizeof(h));
  const size_t sb = state_bytes_of(c);
  if (memcmp(h.magic, kCkptMagic, 8) != 0 || h.abi != POND_ABI_VERSION || h.D != c->D ||
      h.fp32 != (c->fp32 ? 1 : 0) || h.nx != c->nx || h.ny != c->ny || h.state_bytes != sb ||
      bytes < sizeof(CkptHdr) + sb || !(h.dt > 0.0))
    return POND_E_INVAL;
  POND_CUDA(cudaStreamSynchronize(c->stream));
  c->cur = 0;
  POND_CUDA(cudaMemcpyAsync(c->buf[0], static_cast<const unsigned char *>(host) + sizeof(CkptHdr), sb,
                            cudaMemcpyHostToDevice, c->stream));
  POND_CUDA(cudaMemcpyAsync(c->stats, &h.stats, sizeof(Stats), cudaMemcpyHostToDevice, c->stream));
  c->dt = h.dt;
  set_step_const(c);
  drop_graphs(c);
  pond_status s = prepare_step(c);  // synchronises the stream
  if (s != POND_OK) return s;
  c->steps = h.steps;
  c->inited = true;
  return POND_OK;
}

}  // extern "C"

// The constants of one step (both entry points that launch the step kernels).
void pond_fill_step_const(pond::StepConst &K, const pond_params &p, int D, int64_t nx, int64_t ny,
                          double dt) {
  memset(&K, 0, sizeof(K));
  K.nx = (int)nx;
  K.ny = (int)ny;
  for (int s = 0; s < 4; ++s) {
    K.bc[s] = p.bc[s];
    for (int m = 0; m < 4; ++m) K.inflow[s][m] = p.inflow[s][m];
  }
  const double tau = p.tau, h = 0.5 * dt;
  K.lam = dt / p.dx;
  // face phi = kappa1 phi_bar + kappa2 phi^eq (inverse of Eq. eq:FluxTransf)
  K.kappa1 = 2.0 * tau / (2.0 * tau + h);
  K.kr = (h / (2.0 * tau + h)) / K.kappa1;
  // phi_bar^+ = (2 tau - h)/(2 tau + dt) phi~ + 3h/(2 tau + dt) phi^eq  (Eqs. eq:variableTransform, eq:Fbarplus)
  K.kp_a = K.kappa1 * (2.0 * tau - h) / (2.0 * tau + dt);
  K.kp_b = K.kappa1 * 3.0 * h / (2.0 * tau + dt);
  K.a1 = (2.0 * tau - dt) / (2.0 * tau + dt);
  K.a2 = 2.0 * dt / (2.0 * tau + dt);
  const double tau2 = tau / p.prandtl;
  K.qe = p.prandtl == 1.0 ? 1.0 : 1.0 + 0.5 * dt * (1.0 / tau - 1.0 / tau2);
  const double cv = 1.0 / (p.gamma - 1.0);
  K.inv_cv = 1.0 / cv;
  K.gfac = cv - 0.5 * D;
  K.iter_tol = p.iter_tol;
  K.iter_max = p.iter_max;
  K.tau1 = tau;
  K.tau2 = tau2;
  K.cfac = 1.0 + dt / (2.0 * tau);
  K.inv2dx = 1.0 / (2.0 * p.dx);
  K.grad_k = p.transform == POND_GRAD_K;
  K.appc = p.flux_form == POND_FLUX_APPC;
  K.limiter = p.limiter;
  K.iterative = p.flux_frame == POND_FRAME_ITER;
  K.xi_thr = (float)p.xi_fp64_threshold;
  K.ms = p.multiscale;
  K.ms_theta_u = p.ms_theta_u;
  K.ms_theta_T = p.ms_theta_T;
  K.cf.lam = (float)K.lam;
  K.cf.kappa1 = (float)K.kappa1;
  K.cf.kr = (float)K.kr;
  K.cf.kp_a = (float)K.kp_a;
  K.cf.kp_b = (float)K.kp_b;
  K.cf.a1 = (float)K.a1;
  K.cf.a2 = (float)K.a2;
  K.cf.qe = (float)K.qe;
  K.cf.inv_cv = (float)K.inv_cv;
  K.cf.gfac = (float)K.gfac;
}
