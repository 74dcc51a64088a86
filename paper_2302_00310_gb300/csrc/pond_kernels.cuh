// pond_kernels.cuh -- the fused PonD step kernel and its helpers (sm_103a).
//
// One launch advances every cell by one time step of Sec. IV.A.3 of
// arXiv:2302.00310 (with the Strang-split quasi-equilibrium step of Sec. IV.B).
// A CTA owns a BX x BY tile of cells and runs three phases separated by block
// barriers:
//   A. every cell of the halo-2 tile: load phi~ (SoA, coalesced), first QE
//      half step, phi_bar^+ of Eq. eq:Fbarplus -> shared memory;
//   B. every face touching the tile: averaged face frame (Eq. eq::AvgFrame),
//      the 8 (2D) / 4 (1D) stencil cells moved into it by the Hermite shift
//      (Sec. II.B), limited MUSCL half-step trace (Eq. eq:InterfacePop),
//      interface moments, non-co-moving equilibrium (Eq. NonComovingEq) in
//      closed form, face phi (inverse of Eq. eq:FluxTransf) -> shared memory;
//   C. every cell of the tile: face phi moved into the cell frame and
//      multiplied by v.n (Eq. fluxEq), DUGKS update (Eq. eq:FinalUpdateDUGKS),
//      new co-moving frame, second QE half step, store.
// All linear algebra is done on dimensional Hermite coefficients
// (pond_hermite.cuh), and the state itself is stored as each cell's
// B_ab = sum_i phi_i H_a(v_ix - u_x; T) H_b(v_iy - u_y; T) in its frame {u, T}
// (an invertible change of basis on the lattice, Eq. GradsProjection): a step
// needs no synthesis or analysis of its own cells, the conserved moments are
// stored values (rho = B_00, rho (u - u_frame) = B_10), and a frame change is
// a unit-triangular map with no square root.  Populations (divided by the
// lattice weights) are synthesised only where the limiter needs them (the
// stencil in the face frame) and at the library boundary.
#pragma once
#include <cstdint>
#include <type_traits>

#include "pond_hermite.cuh"
#include "pond_packed.cuh"

namespace pond {

enum { BC_PERIODIC = 0, BC_ZERO_GRADIENT = 1, BC_INFLOW = 2, BC_WALL = 3 };

// A tile's halo stride and face count as a type: the stencil and face
// functions take either this (the step kernels: the shared-memory offsets
// become immediates, also inside the mixed path's out-of-line calls, which
// are then instantiated per tile shape) or a plain int.
template <int V> struct CInt {
  __device__ constexpr operator int() const { return V; }
};
enum { LIM_VANLEER = 0, LIM_MINMOD = 1 };
enum { FLAG_NONPHYSICAL = 1u, FLAG_CFL = 2u, FLAG_NOCONV = 4u };

// Per-run constants, passed by value (kernel parameter space).
struct StepConst {
  int nx, ny;
  int bc[4];
  double inflow[4][4];  // rho, ux, uy, T (a wall: unused, its ux, uy, T)
  double lam;           // dt/dx
  double kappa1;        // 2 tau/(2 tau + h), h = dt/2: weight of phi_bar in the face phi
  double kr;            // (h/(2 tau + h))/kappa1: weight of phi^eq relative to kappa1
  double kp_a;          // kappa1 (2 tau - h)/(2 tau + dt): phi_bar^+ weight of phi~ (times kappa1)
  double kp_b;          // kappa1 3h/(2 tau + dt): phi_bar^+ weight of phi^eq (times kappa1)
  double a1, a2;        // DUGKS update: (2 tau - dt)/(2 tau + dt), 2 dt/(2 tau + dt)
  double qe;            // 1 + dt/2 (1/tau1 - 1/tau2): QE half step on 3rd-order (f) / 1st-order (g) content
  double inv_cv;        // 1/C_v
  double gfac;          // C_v - D/2
  double iter_tol;
  double tau1, tau2;    // relaxation times (tau2 = tau1 / Pr)
  double cfac;          // 1 + dt/(2 tau1): phi~ - phi^eq over phi - phi^eq
  double inv2dx;        // 1/(2 dx): centred differences at wall ghosts
  double ms_theta_u, ms_theta_T;  // multiscale switching thresholds
  int iter_max;
  int grad_k, appc, limiter, iterative;
  int ms;               // multiscale f-lattice (D1Q3 / D2Q9 where smooth)
  float xi_thr;         // mixed path: FP64 frame transformation when max_j |a c_j + b| exceeds this
  // FP32 copies of the coefficients above for the mixed path (no conversion in the kernel)
  struct {
    float lam, kappa1, kr, kp_a, kp_b, a1, a2, qe, inv_cv, gfac;
  } cf;
};

// A coefficient of the run in the arithmetic type R.
template <typename R> __device__ __forceinline__ R kc(double d, float f);
template <> __device__ __forceinline__ double kc<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float kc<float>(double, float f) { return f; }

// State planes (SoA, x fastest): f[a + 4b][N] and g[a + 3b][N] are the
// dimensional Hermite coefficients B_ab of phi~ in the cell's frame (ux, uy, T).
// Mixed path: M[4][N] are each cell's conserved moments rho, rho ux, rho uy,
// rho E (Eqs. eq::ConservationLaws, eq:E) in FP64, the sums a step adds the
// face fluxes to (the coefficients hold them rounded to FP32); null in FP64.
template <typename R> struct State {
  R *f, *g, *ux, *uy, *T;
  double *M;
};

struct Stats {
  unsigned int flags;
  unsigned int max_traces;          // iterated face frame: most traces made at one face
  unsigned long long max_cfl_bits;  // bit pattern of a non-negative double
  unsigned long long noconv;
  unsigned long long traces;        // iterated face frame: traces made, over all face evaluations
  unsigned long long face_evals;    // iterated face frame: face evaluations counted
  unsigned long long ms_high;       // multiscale: cell updates on the high-order lattice
};

// QF1: f-lattice nodes per axis (4: D1Q4 / D2Q16, 5: D2Q25); QG1: g-lattice
// nodes per axis (3: D1Q3 / D2Q9, as in the paper's runs; 4: g on f's D1Q4 /
// D2Q16 lattice)
template <int DIM, int QF1 = 4, int QG1 = 3> struct Dims {
  static constexpr int QF = DIM == 2 ? QF1 * QF1 : QF1;
  static constexpr int QG = DIM == 2 ? QG1 * QG1 : QG1;
  static constexpr int NYF = DIM == 2 ? QF1 : 1;
  static constexpr int NYG = DIM == 2 ? QG1 : 1;
  // shared-memory record of a halo cell: f coeffs, g coeffs, ux, uy, T, and
  // (mixed path) sqrt T
  static constexpr int IUX = QF + QG, IUY = IUX + 1, IT = IUX + 2, IST = IUX + 3;
  static constexpr int NPREP = QF + QG + 4;
  // shared-memory record of a face: f coeffs, g coeffs, uFx, uFy, TF, and
  // (mixed path) sqrt TF and the conserved fluxes: mass, x-, y-momentum, energy
  static constexpr int FUX = QF + QG, FUY = FUX + 1, FT = FUX + 2, FST = FUX + 3;
  static constexpr int FJ = FUX + 4;
  template <typename R> static constexpr int nface() {
    return std::is_same<R, float>::value ? QF + QG + 8 : QF + QG + 3;
  }
};

template <int DIM, int BX, int BY, int QF1 = 4, int QG1 = 3> struct Tile {
  static constexpr int HX = BX + 4, HY = DIM == 2 ? BY + 4 : 1, OY = DIM == 2 ? 2 : 0;
  static constexpr int NH = HX * HY;
  static constexpr int NFX = (BX + 1) * (DIM == 2 ? BY : 1);
  static constexpr int NFY = DIM == 2 ? BX * (BY + 1) : 0;
  static constexpr int NFACES = NFX + NFY;
  static constexpr int NCELL = BX * (DIM == 2 ? BY : 1);
  // MS: a byte per halo cell after the face records, its multiscale lattice
  template <typename R, bool MS = false> static constexpr size_t smem_bytes() {
    return sizeof(R) * ((size_t)NH * Dims<DIM, QF1, QG1>::NPREP +
                        (size_t)NFACES * Dims<DIM, QF1, QG1>::template nface<R>()) +
           (MS ? ((size_t)NH + 15) / 16 * 16 : 0);
  }
};

// ---- boundary ghosts (Sec. IV.D): x rule first, then y rule ----------------
template <int DIM>
__device__ __forceinline__ int map_cell(const StepConst &K, int j, int k, int &sj, int &sk) {
  if (j < 0 || j >= K.nx) {
    const int side = j < 0 ? 0 : 1, b = K.bc[side];
    if (b == BC_INFLOW) return side;
    if (b == BC_PERIODIC) { j %= K.nx; if (j < 0) j += K.nx; }
    else j = j < 0 ? 0 : K.nx - 1;
  }
  if (DIM == 2 && (k < 0 || k >= K.ny)) {
    const int side = k < 0 ? 2 : 3, b = K.bc[side];
    if (b == BC_INFLOW) return side;
    if (b == BC_PERIODIC) { k %= K.ny; if (k < 0) k += K.ny; }
    else k = k < 0 ? 0 : K.ny - 1;
  }
  sj = j; sk = (DIM == 2) ? k : 0;
  return -1;
}

// QE half step (Sec. IV.B) in the co-moving frame: f* - f^eq is the total
// order-3 Hermite content of f and g* - g^eq the order-1 content of g
// (Eq. eq::quasi_f), so the relaxation scales those coefficients by qe.
template <typename R, int QF1, int NYF, int QG1, int NYG>
__device__ __forceinline__ void qe_scale(Blk<R, QF1, NYF> &F, Blk<R, QG1, NYG> &G, R qe) {
#pragma unroll
  for (int a = 0; a < QF1; ++a)
#pragma unroll
    for (int b = 0; b < NYF; ++b)
      if (a + b == 3) F.v[a][b] *= qe;
#pragma unroll
  for (int a = 0; a < QG1; ++a)
#pragma unroll
    for (int b = 0; b < NYG; ++b)
      if (a + b == 1) G.v[a][b] *= qe;
}

template <typename R> __device__ __forceinline__ R qnan();
template <> __device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000LL); }
template <> __device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }

__device__ __forceinline__ float div_nr(float x, float y) { return __fdividef(x, y); }
// 1/y to 2^-39 relative (2^-39.9 measured), for 2^-1022 <= |y| < 2^1022: the hardware
// approximation rcp.approx.ftz.f64 refined by one Newton-Raphson step for the
// reciprocal, r1 = r0 + r0 (1 - y r0), written as two fused multiply-adds
// (the FMA form of Newton's iteration of P. Markstein, "Computation of
// elementary functions on the IBM RISC System/6000 processor", IBM J. Res.
// Dev. 34 (1990) 111-119); one step squares the relative error of r0.  Used
// where the result feeds a quantity that tolerates that error (the van Leer
// slope, which enters the trace times an offset below 1; the mixed path's
// FP64 frame, rounded to FP32 afterwards).  pond_check_reciprocal() compares
// it with CUDA's correctly rounded reciprocal.
__device__ __forceinline__ double rcp_nr1(double y) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(y));
  return fma(r, fma(-y, r, 1.0), r);
}

// sign tests on the integer image (no FP64-pipe compare): v > 0 and
// |x| < |y|.  Positive subnormals below 2^-1022 count as zero.
__device__ __forceinline__ bool pos(double v) { return __double2hiint(v) > 0; }
__device__ __forceinline__ bool pos(float v) { return __float_as_int(v) > 0; }
__device__ __forceinline__ bool abs_less(double x, double y) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) < (__double_as_longlong(y) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool abs_less(float x, float y) {
  return (__float_as_int(x) & 0x7fffffff) < (__float_as_int(y) & 0x7fffffff);
}

// The limited slope divided by lf(lim) (lf = 2 for van Leer, 1 for minmod;
// the factor is folded into the trace offsets): van Leer 2xy/(x+y) / 2.  In
// FP64 the quotient takes the reciprocal after one Newton step (no residual
// correction of the quotient): the slope enters the trace times an offset
// below 1, and the step is bound by the FP64 pipe (2 DFMA saved per limit).
template <typename R, typename LT> __device__ __forceinline__ R limiter_factor(LT lim) {
  return lim == LIM_MINMOD ? R(1) : R(2);
}
template <typename R, typename LT>
__device__ __forceinline__ R limit(R x, R y, LT lim) {
  const R p = x * y;
  if (lim == LIM_MINMOD) return pos(p) ? (abs_less(x, y) ? x : y) : R(0);
  if constexpr (std::is_same<R, double>::value) return pos(p) ? p * rcp_nr1(x + y) : R(0);
  else return pos(p) ? div_nr(p, x + y) : R(0);
}

// The limited slope of two lanes at once (the mixed path's trace): the
// differences, product, sum and quotient in the paired FP32 instructions, the
// reciprocal and the sign tests per lane; the same values as limit() on each
// lane to FP32 rounding.
template <typename LT>
__device__ __forceinline__ f2 limit2(f2 x, f2 y, LT lim) {
  const f2 p = x * y;
  if (lim == LIM_MINMOD)
    return f2(pos(p.lo()) ? (abs_less(x.lo(), y.lo()) ? x.lo() : y.lo()) : 0.f,
              pos(p.hi()) ? (abs_less(x.hi(), y.hi()) ? x.hi() : y.hi()) : 0.f);
  const f2 s = x + y;
  const f2 q = p * f2(__fdividef(1.f, s.lo()), __fdividef(1.f, s.hi()));
  return f2(pos(p.lo()) ? q.lo() : 0.f, pos(p.hi()) ? q.hi() : 0.f);
}

// The FP32 instantiation is the mixed-precision path (POND_FP32_MIXED).
template <typename R> constexpr bool is_mixed() { return std::is_same<R, float>::value; }

// The FP64 form of move_frame() for the mixed path, kept out of line: it is
// rarely taken, and one shared copy keeps the FP32 kernel's hot code compact.
template <int DIM, int Q>
__device__ __noinline__ void move_frame_fp64(float usx, float usy, float Ts, float utx, float uty,
                                             float Tt, Blk<float, Q, (DIM == 2 ? Q : 1)> &Y) {
  constexpr int NY = DIM == 2 ? Q : 1;
  Blk<double, Q, NY> Z;
#pragma unroll
  for (int n = 0; n < Q; ++n)
#pragma unroll
    for (int m = 0; m < NY; ++m) Z.v[n][m] = Y.v[n][m];
  const double dT = (double)Ts - (double)Tt, dT3 = 3.0 * dT;
  shift_x(make_dshift((double)usx - (double)utx, dT, dT3), Z);
  if constexpr (DIM == 2) shift_y(make_dshift((double)usy - (double)uty, dT, dT3), Z);
#pragma unroll
  for (int n = 0; n < Q; ++n)
#pragma unroll
    for (int m = 0; m < NY; ++m) Y.v[n][m] = (float)Z.v[n][m];
}

// Moves dimensional Hermite coefficients Y (Q nodes per axis) from the frame
// {us, Ts} to {ut, Tt} (Sec. II.B): per axis the unit-triangular map of
// d = us - ut and Ts - Tt.  On the mixed path a transformation whose source
// nodes land far out in the target frame (max_j |sqrt(Ts) c_j + d| >
// xi_thr sqrt(Tt): large, cancelling coefficients, as at large temperature
// ratios) is built and applied in FP64; sTs, sTt = sqrt(Ts), sqrt(Tt) are read
// only by that test.
template <typename R, int DIM, int Q>
__device__ __forceinline__ void move_frame(const StepConst &K, R usx, R usy, R Ts, R sTs, R utx,
                                           R uty, R Tt, R sTt, Blk<R, Q, (DIM == 2 ? Q : 1)> &Y) {
  const R dx = usx - utx, dy = DIM == 2 ? usy - uty : R(0), dT = Ts - Tt;
  if constexpr (is_mixed<R>()) {
    if (fmaf(sTs, float(Nodes<Q>::cmax), fmaxf(fabsf(dx), fabsf(dy))) > K.xi_thr * sTt) {
      move_frame_fp64<DIM, Q>(usx, usy, Ts, utx, uty, Tt, Y);
      return;
    }
  }
  const R dT3 = R(3) * dT;
  shift_x(make_dshift(dx, dT, dT3), Y);
  if constexpr (DIM == 2) shift_y(make_dshift(dy, dT, dT3), Y);
}

// multiscale projection onto the low-order lattice (Sec. II.E): coefficients of order 3 along an
// axis (and, with the Grad projection, of total order 3) dropped
template <typename R, int Q, int NY>
__device__ __forceinline__ void ms_project(Blk<R, Q, NY> &B, int grad_k) {
#pragma unroll
  for (int a = 0; a < Q; ++a)
#pragma unroll
    for (int b = 0; b < NY; ++b)
      if (a > 2 || b > 2 || (NY > 1 && grad_k && a + b > 2)) B.v[a][b] = R(0);
}

// ---- wall ghosts (Sec. IV.D) -------------------------------------------------
// Walls sit on the y sides in 2D (the x sides then periodic or zero-gradient)
// and on the x sides in 1D, half a cell beyond the last interior cell;
// inflow[side] = (unused, u_w,x, u_w,y, T_w).  The ghost at normal distance m
// reflects the interior cell m - 1 cells from the wall: rho_G = rho_B,
// u_G = 2 u_w - u_B, T_G = 2 T_w - T_B.
template <int DIM> __device__ __forceinline__ bool is_wall_ghost(const StepConst &K, int j, int k) {
  if constexpr (DIM == 2) return (k < 0 && K.bc[2] == BC_WALL) || (k >= K.ny && K.bc[3] == BC_WALL);
  else return (j < 0 && K.bc[0] == BC_WALL) || (j >= K.nx && K.bc[1] == BC_WALL);
}

// rho, ux, uy, T (FP64) at index (j, k): an interior cell (rho = B_00, its
// frame being co-moving), or its reflection across a wall
template <typename R, int DIM>
__device__ __forceinline__ void wall_mac(const StepConst &K, const State<R> &S, int j, int k, double m[4]) {
  if (DIM == 2 && (j < 0 || j >= K.nx)) {
    if (K.bc[j < 0 ? 0 : 1] == BC_PERIODIC) { j %= K.nx; if (j < 0) j += K.nx; }
    else j = j < 0 ? 0 : K.nx - 1;
  }
  int &n = DIM == 2 ? k : j;
  const int nmax = DIM == 2 ? K.ny : K.nx, lo = DIM == 2 ? 2 : 0;
  int side = -1;
  if (n < 0) { side = lo; n = -n - 1; }
  else if (n >= nmax) { side = lo + 1; n = 2 * nmax - 1 - n; }
  const size_t c = (size_t)(DIM == 2 ? k : 0) * K.nx + j;
  m[0] = S.f[c];
  m[1] = S.ux[c];
  m[2] = DIM == 2 ? (double)S.uy[c] : 0.0;
  m[3] = S.T[c];
  if (side >= 0) {
    m[1] = 2.0 * K.inflow[side][1] - m[1];
    m[2] = DIM == 2 ? 2.0 * K.inflow[side][2] - m[2] : 0.0;
    m[3] = 2.0 * K.inflow[side][3] - m[3];
  }
}

// The wall ghost (j, k): dimensional Hermite coefficients of its stored
// variable phi~ in its co-moving frame {u_G, T_G}: the equilibrium plus the
// Chapman-Enskog non-equilibrium of the paper's ghost construction (P^(1),
// Q^(1) for f; M_g0, M_g1, M_g2 for g, as central moments in the ghost frame)
// from second-order centred gradients of the previous step's fields, scaled
// by 1 + dt/(2 tau_1) (phi~ = phi + dt/(2 tau_1) (phi - phi^eq)).  With the
// dimensional Hermite polynomials the central moments are the coefficients:
// B_20 = P_xx, B_11 = P_xy, B_21 = Q_xxy, ... (f, whose non-equilibrium has no
// mass or momentum), and B_00 = M_g0, B_10 = M_g1,x, B_20 = M_g2,xx - T M_g0 (g).
template <typename R, int DIM, int QF1, int QG1 = 3>
__device__ __forceinline__ void wall_ghost(const StepConst &K, const State<R> &S, int j, int k,
                                        Blk<R, QF1, Dims<DIM, QF1>::NYF> &F,
                                        Blk<R, QG1, Dims<DIM, QF1, QG1>::NYG> &G,
                                        R &ux, R &uy, R &Tout) {
  double mG[4], a[4], b[4];
  wall_mac<R, DIM>(K, S, j, k, mG);
  const double rho = mG[0], T = mG[3], cv = K.gfac + 0.5 * DIM;
  if (!(rho > 0.0 && T > 0.0)) {  // T_B > 2 T_w: no physical ghost; poison it (flagged downstream)
#pragma unroll
    for (int p = 0; p < QF1; ++p)
#pragma unroll
      for (int q = 0; q < Dims<DIM, QF1>::NYF; ++q) F.v[p][q] = qnan<R>();
#pragma unroll
    for (int p = 0; p < QG1; ++p)
#pragma unroll
      for (int q = 0; q < Dims<DIM, QF1, QG1>::NYG; ++q) G.v[p][q] = qnan<R>();
    ux = R(mG[1]); uy = R(mG[2]); Tout = qnan<R>();
    return;
  }
  double gu[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, gT[2] = {0.0, 0.0};
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    wall_mac<R, DIM>(K, S, j + (d == 0), k + (d == 1), a);
    wall_mac<R, DIM>(K, S, j - (d == 0), k - (d == 1), b);
    gu[d][0] = (a[1] - b[1]) * K.inv2dx;
    gu[d][1] = (a[2] - b[2]) * K.inv2dx;
    gT[d] = (a[3] - b[3]) * K.inv2dx;
  }
  const double div = DIM == 2 ? gu[0][0] + gu[1][1] : gu[0][0];
  const double sxx = 2.0 * gu[0][0], sxy = gu[0][1] + gu[1][0], syy = 2.0 * gu[1][1];
  const double rT = rho * T, gf = 2.0 * cv - DIM, c1 = -K.tau1 * rT * K.cfac, c2 = -K.tau2 * rT * K.cfac;
  // f: P^(1) (second order), Q^(1) (third order, symmetrised grad T times I)
  const double pxx = c1 * (sxx - div / cv), pxy = c1 * sxy, pyy = c1 * (syy - div / cv);
  const double qxxx = c2 * 3.0 * gT[0], qxxy = c2 * gT[1], qxyy = c2 * gT[0], qyyy = c2 * 3.0 * gT[1];
  // g: M_g0, M_g1, M_g2 (central)
  const double m0 = c1 * gf * div / cv, m1x = c2 * gf * gT[0], m1y = c2 * gf * gT[1];
  const double m2xx = c1 * gf * T * sxx, m2xy = c1 * gf * T * sxy, m2yy = c1 * gf * T * syy;
#pragma unroll
  for (int p = 0; p < QF1; ++p)
#pragma unroll
    for (int q = 0; q < Dims<DIM, QF1>::NYF; ++q) F.v[p][q] = R(0);
#pragma unroll
  for (int p = 0; p < QG1; ++p)
#pragma unroll
    for (int q = 0; q < Dims<DIM, QF1, QG1>::NYG; ++q) G.v[p][q] = R(0);
  F.v[0][0] = R(rho);
  F.v[2][0] = R(pxx);
  F.v[3][0] = R(qxxx);
  G.v[0][0] = R(K.gfac * T * rho + m0);
  G.v[1][0] = R(m1x);
  G.v[2][0] = R(m2xx - T * m0);
  if constexpr (DIM == 2) {
    F.v[1][1] = R(pxy); F.v[0][2] = R(pyy);
    F.v[2][1] = R(qxxy); F.v[1][2] = R(qxyy); F.v[0][3] = R(qyyy);
    G.v[0][1] = R(m1y); G.v[1][1] = R(m2xy); G.v[0][2] = R(m2yy - T * m0);
  }
  ux = R(mG[1]);
  uy = R(mG[2]);
  Tout = R(T);
}

// the interior cell that the wall ghost (j, k) reflects (the x rule first in 2D)
template <int DIM>
__device__ __forceinline__ void wall_source(const StepConst &K, int j, int k, int &sj, int &sk) {
  if (DIM == 2 && (j < 0 || j >= K.nx)) {
    if (K.bc[j < 0 ? 0 : 1] == BC_PERIODIC) { j %= K.nx; if (j < 0) j += K.nx; }
    else j = j < 0 ? 0 : K.nx - 1;
  }
  int &n = DIM == 2 ? k : j;
  const int nmax = DIM == 2 ? K.ny : K.nx;
  n = n < 0 ? -n - 1 : 2 * nmax - 1 - n;
  sj = j; sk = DIM == 2 ? k : 0;
}

// phase A for a wall ghost (out of line: only halo cells across a wall run it):
// phi_bar^+ = kp_a phi~ + kp_b phi^eq, with no quasi-equilibrium step (the
// ghost is built from the cells' macroscopic fields, which it leaves alone).
// low: the multiscale ghost takes the low-order lattice of the cell it
// reflects, and its content of order 3 along an axis is dropped.
template <typename R, int DIM, int QF1, int QG1 = 3>
__device__ __noinline__ void prep_wall_cell(const StepConst &K, const State<R> &S, int j, int k, R *sp,
                                            int NH, int h, bool low = false) {
  using D = Dims<DIM, QF1, QG1>;
  Blk<R, QF1, D::NYF> F;
  Blk<R, QG1, D::NYG> G;
  R ux, uy, T;
  wall_ghost<R, DIM, QF1, QG1>(K, S, j, k, F, G, ux, uy, T);
  if (low) ms_project(F, K.grad_k);
  const R rho = F.v[0][0], ka = kc<R>(K.kp_a, K.cf.kp_a);
#pragma unroll
  for (int a = 0; a < QF1; ++a)
#pragma unroll
    for (int b = 0; b < D::NYF; ++b) F.v[a][b] *= ka;
#pragma unroll
  for (int a = 0; a < QG1; ++a)
#pragma unroll
    for (int b = 0; b < D::NYG; ++b) G.v[a][b] *= ka;
  F.v[0][0] = kc<R>(K.kappa1, K.cf.kappa1) * rho;
  G.v[0][0] += kc<R>(K.kp_b, K.cf.kp_b) * kc<R>(K.gfac, K.cf.gfac) * T * rho;
#pragma unroll
  for (int a = 0; a < QF1; ++a)
#pragma unroll
    for (int b = 0; b < D::NYF; ++b) sp[(a + QF1 * b) * NH + h] = F.v[a][b];
#pragma unroll
  for (int a = 0; a < QG1; ++a)
#pragma unroll
    for (int b = 0; b < D::NYG; ++b) sp[(D::QF + a + QG1 * b) * NH + h] = G.v[a][b];
  sp[D::IUX * NH + h] = ux;
  sp[D::IUY * NH + h] = uy;
  sp[D::IT * NH + h] = T;
  if constexpr (is_mixed<R>()) sp[D::IST * NH + h] = sqrt(T);
}

// ---- multiscale f-lattice (Sec. II.E, Sec. IV.C) -----------------------------
// Each step every cell takes the high-order f-lattice (D1Q4 / D2Q16) where
// the jump of u or T across it exceeds its threshold, else D1Q3 / D2Q9:
// s_u = max_{d,e} |u_e(+d) - u_e(-d)| / (2 sqrt T), s_T = max_d |T(+d) - T(-d)| / (2 T),
// from the step's start fields, neighbours by the ghost rules.  A low cell's
// coefficients of order 3 along an axis are zero in its co-moving frame (the
// lifting's equilibrium completion: odd central moments of a Gaussian
// vanish), and a cell that turns low drops them (the projection).  A face
// takes the higher lattice of its two cells.

// u_x, u_y, T at index (j, k): an interior cell or its ghost (a wall ghost:
// the reflection of Sec. IV.D)
template <int DIM, typename R>
__device__ __forceinline__ void ms_fields(const StepConst &K, const State<R> &S, int j, int k,
                                          double &ux, double &uy, double &T) {
  if (is_wall_ghost<DIM>(K, j, k)) {
    double m[4];
    wall_mac<R, DIM>(K, S, j, k, m);
    ux = m[1]; uy = m[2]; T = m[3];
    return;
  }
  int sj = 0, sk = 0;
  const int side = map_cell<DIM>(K, j, k, sj, sk);
  if (side >= 0) {
    ux = K.inflow[side][1]; uy = DIM == 2 ? K.inflow[side][2] : 0.0; T = K.inflow[side][3];
  } else {
    const size_t c = (size_t)sk * K.nx + sj;
    ux = (double)S.ux[c]; uy = DIM == 2 ? (double)S.uy[c] : 0.0; T = (double)S.T[c];
  }
}
// the lattice of interior cell (j, k) this step: true = high order
template <int DIM, typename R>
__device__ __noinline__ bool ms_high(const StepConst &K, const State<R> &S, int j, int k) {
  double gu = 0.0, gT = 0.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    double pux, puy, pT, mux, muy, mT;
    ms_fields<DIM>(K, S, j + (d == 0), k + (d == 1), pux, puy, pT);
    ms_fields<DIM>(K, S, j - (d == 0), k - (d == 1), mux, muy, mT);
    gu = fmax(gu, fabs(pux - mux));
    if (DIM == 2) gu = fmax(gu, fabs(puy - muy));
    gT = fmax(gT, fabs(pT - mT));
  }
  const double T = (double)S.T[(size_t)k * K.nx + j];
  return 0.5 * gu / sqrt(T) > K.ms_theta_u || 0.5 * gT / T > K.ms_theta_T;
}

// ---- phase A: one halo cell -> shared memory ------------------------------
// MS: multiscale; the cell's lattice goes to lat[h] (1 high, 0 low).
template <typename R, int DIM, int QF1, bool MS = false, int QG1 = 3>
__device__ __forceinline__ void prep_cell(const StepConst &K, const State<R> &S, int j, int k, R *sp,
                                          int NH, int h, unsigned char *lat = nullptr) {
  using D = Dims<DIM, QF1, QG1>;
  Blk<R, QF1, D::NYF> F;
  Blk<R, QG1, D::NYG> G;
  R ux, uy, T;
  int sj = 0, sk = 0;
  if (is_wall_ghost<DIM>(K, j, k)) {
    bool low = false;
    if constexpr (MS) {  // the lattice of the cell the ghost reflects
      int wj = 0, wk = 0;
      wall_source<DIM>(K, j, k, wj, wk);
      low = !ms_high<DIM>(K, S, wj, wk);
      lat[h] = low ? 0 : 1;
    }
    prep_wall_cell<R, DIM, QF1, QG1>(K, S, j, k, sp, NH, h, low);
    return;
  }
  const int side = map_cell<DIM>(K, j, k, sj, sk);
  if (side < 0) {
    const size_t N = (size_t)K.nx * (DIM == 2 ? K.ny : 1);
    const size_t c = (size_t)sk * K.nx + sj;
#pragma unroll
    for (int i = 0; i < D::QF; ++i) F.v[i % QF1][i / QF1] = S.f[i * N + c];
#pragma unroll
    for (int i = 0; i < D::QG; ++i) G.v[i % QG1][i / QG1] = S.g[i * N + c];
    ux = S.ux[c];
    uy = DIM == 2 ? S.uy[c] : R(0);
    T = S.T[c];
    if constexpr (MS) {
      const bool hi = ms_high<DIM>(K, S, sj, sk);
      if (!hi) ms_project(F, K.grad_k);
      lat[h] = hi ? 1 : 0;
    }
    // the first QE half step (qe on the order-3 content of f and order-1 of
    // g) and the kp_a of phi_bar^+ in one scaling per coefficient
    const R rho = F.v[0][0], ka = kc<R>(K.kp_a, K.cf.kp_a), kq = ka * kc<R>(K.qe, K.cf.qe);
#pragma unroll
    for (int a = 0; a < QF1; ++a)
#pragma unroll
      for (int b = 0; b < D::NYF; ++b) F.v[a][b] *= a + b == 3 ? kq : ka;
#pragma unroll
    for (int a = 0; a < QG1; ++a)
#pragma unroll
      for (int b = 0; b < D::NYG; ++b) G.v[a][b] *= a + b == 1 ? kq : ka;
    // phi_bar^+ = kp_a phi~ + kp_b phi^eq; phi^eq = rho W (f), (C_v - D/2) T rho W (g)
    F.v[0][0] = kc<R>(K.kappa1, K.cf.kappa1) * rho;
    G.v[0][0] += kc<R>(K.kp_b, K.cf.kp_b) * kc<R>(K.gfac, K.cf.gfac) * T * rho;
  } else {
    if constexpr (MS) lat[h] = 0;  // an inflow ghost: equilibrium, either lattice
    const R rho = R(K.inflow[side][0]);
    ux = R(K.inflow[side][1]);
    uy = DIM == 2 ? R(K.inflow[side][2]) : R(0);
    T = R(K.inflow[side][3]);
#pragma unroll
    for (int a = 0; a < QF1; ++a)
#pragma unroll
      for (int b = 0; b < D::NYF; ++b) F.v[a][b] = R(0);
#pragma unroll
    for (int a = 0; a < QG1; ++a)
#pragma unroll
      for (int b = 0; b < D::NYG; ++b) G.v[a][b] = R(0);
    F.v[0][0] = kc<R>(K.kappa1, K.cf.kappa1) * rho;
    G.v[0][0] = kc<R>(K.kappa1, K.cf.kappa1) * kc<R>(K.gfac, K.cf.gfac) * T * rho;
  }
#pragma unroll
  for (int a = 0; a < QF1; ++a)
#pragma unroll
    for (int b = 0; b < D::NYF; ++b) sp[(a + QF1 * b) * NH + h] = F.v[a][b];
#pragma unroll
  for (int a = 0; a < QG1; ++a)
#pragma unroll
    for (int b = 0; b < D::NYG; ++b) sp[(D::QF + a + QG1 * b) * NH + h] = G.v[a][b];
  sp[D::IUX * NH + h] = ux;
  sp[D::IUY * NH + h] = uy;
  sp[D::IT * NH + h] = T;
  if constexpr (is_mixed<R>()) sp[D::IST * NH + h] = sqrt(T);
}

// ---- phase B helpers --------------------------------------------------------
// phi_bar^+ of halo cell h (times kappa1) moved into the face frame
// {uF, TF} and synthesised into node values divided by the weights,
// Y[x-node][y-node] (SK: the face frame's synthesis constants).
// GS: 0 for the f coefficients (stride QF1), else the g coefficients (stride
// QG1, the g-lattice's nodes per axis); Q: the lattice the face works on (a
// multiscale face with the low-order f-lattice reads the f coefficients of
// order <= 2 per axis: the projection).
template <typename R, int DIM, int QF1, int Q, int GS, int QG1, typename NHT>
__device__ __forceinline__ void stencil_pops_body(const StepConst &K, const R *sp, NHT NH, int h, R uFx,
                                                  R uFy, R TF, R sTF, const SynK<R, Q> &SK,
                                                  Blk<R, Q, (DIM == 2 ? Q : 1)> &Y) {
  using D = Dims<DIM, QF1, QG1>;
  constexpr int NY = DIM == 2 ? Q : 1;
  constexpr int base = GS ? D::QF : 0, stride = GS ? QG1 : QF1;
#pragma unroll
  for (int n = 0; n < Q; ++n)
#pragma unroll
    for (int m = 0; m < NY; ++m) Y.v[n][m] = sp[(base + n + stride * m) * NH + h];
  move_frame<R, DIM, Q>(K, sp[D::IUX * NH + h], DIM == 2 ? sp[D::IUY * NH + h] : R(0), sp[D::IT * NH + h],
                        is_mixed<R>() ? sp[D::IST * NH + h] : R(0), uFx, uFy, TF, sTF, Y);
  if constexpr (DIM == 2) {
    if (K.grad_k) grad_mask(Y);
  }
  synq_xy(SK, Y);
}
// The mixed path calls one out-of-line copy of the stencil transformation per
// lattice (16 call sites per face direction): the FP32 kernel is bound by
// instruction fetch, not arithmetic, and the shared copy keeps its code
// footprint small.  The FP64 kernel, bound by the FP64 pipe, inlines it.
template <typename R, int DIM, int QF1, int Q, int GS, int QG1, typename NHT>
__device__ __noinline__ Blk<R, Q, (DIM == 2 ? Q : 1)> stencil_pops_call(const StepConst &K, const R *sp,
                                                                      NHT NH, int h, R uFx, R uFy,
                                                                      R TF, R sTF, SynK<R, Q> SK) {
  Blk<R, Q, (DIM == 2 ? Q : 1)> Y;  // returned by value: in registers, not through local memory
  stencil_pops_body<R, DIM, QF1, Q, GS, QG1>(K, sp, NH, h, uFx, uFy, TF, sTF, SK, Y);
  return Y;
}
template <typename R, int DIM, int QF1, int Q, int GS, int QG1, typename NHT>
__device__ __forceinline__ void stencil_pops(const StepConst &K, const R *sp, NHT NH, int h, R uFx,
                                             R uFy, R TF, R sTF, const SynK<R, Q> &SK,
                                             Blk<R, Q, (DIM == 2 ? Q : 1)> &Y) {
  if constexpr (is_mixed<R>())
    Y = stencil_pops_call<R, DIM, QF1, Q, GS, QG1>(K, sp, NH, h, uFx, uFy, TF, sTF, SK);
  else stencil_pops_body<R, DIM, QF1, Q, GS, QG1>(K, sp, NH, h, uFx, uFy, TF, sTF, SK, Y);
}

// The mixed path moves the two cells beside the face (stencil cells 0 and 1)
// together, in one out-of-line call, in the two lanes of the paired FP32
// instructions: the same tensor-product frame change (each lane its own
// shift), Grad projection and synthesis as stencil_pops_body.  A cell whose
// transformation must run in FP64 takes both cells through
// stencil_pops_body instead.
template <typename R, int DIM, int Q> struct TwoBlk {
  Blk<R, Q, (DIM == 2 ? Q : 1)> L, R_;
};
template <int DIM, int QF1, int Q, int GS, int QG1, typename NHT>
__device__ __forceinline__ TwoBlk<float, DIM, Q> stencil_two_body(const StepConst &K, const float *sp, NHT NH,
                                                                 int hL, int hR, float uFx, float uFy, float TF,
                                                                 float sTF, const SynK<float, Q> &SK) {
  using D = Dims<DIM, QF1, QG1>;
  constexpr int NY = DIM == 2 ? Q : 1, base = GS ? D::QF : 0, stride = GS ? QG1 : QF1;
  TwoBlk<float, DIM, Q> out;
  const float uxL = sp[D::IUX * NH + hL], uxR = sp[D::IUX * NH + hR];
  const float uyL = DIM == 2 ? sp[D::IUY * NH + hL] : 0.f, uyR = DIM == 2 ? sp[D::IUY * NH + hR] : 0.f;
  const float TL = sp[D::IT * NH + hL], TR = sp[D::IT * NH + hR];
  const float lim = K.xi_thr * sTF;
  const bool full =
      fmaf(sp[D::IST * NH + hL], float(Nodes<Q>::cmax), fmaxf(fabsf(uxL - uFx), fabsf(uyL - uFy))) > lim ||
      fmaf(sp[D::IST * NH + hR], float(Nodes<Q>::cmax), fmaxf(fabsf(uxR - uFx), fabsf(uyR - uFy))) > lim;
  if (full) {
    stencil_pops_body<float, DIM, QF1, Q, GS, QG1>(K, sp, NH, hL, uFx, uFy, TF, sTF, SK, out.L);
    stencil_pops_body<float, DIM, QF1, Q, GS, QG1>(K, sp, NH, hR, uFx, uFy, TF, sTF, SK, out.R_);
    return out;
  }
  const SynK<f2, Q> S(SK);
  const f2 dT(TL - TF, TR - TF), dT3 = f2(3) * dT;
  Blk<f2, Q, NY> B;
#pragma unroll
  for (int n = 0; n < Q; ++n)
#pragma unroll
    for (int m = 0; m < NY; ++m)
      B.v[n][m] = f2(sp[(base + n + stride * m) * NH + hL], sp[(base + n + stride * m) * NH + hR]);
  shift_x(make_dshift(f2(uxL - uFx, uxR - uFx), dT, dT3), B);
  if constexpr (DIM == 2) {
    shift_y(make_dshift(f2(uyL - uFy, uyR - uFy), dT, dT3), B);
    if (K.grad_k) grad_mask(B);
  }
  synq_xy(S, B);
#pragma unroll
  for (int n = 0; n < Q; ++n)
#pragma unroll
    for (int m = 0; m < NY; ++m) {
      out.L.v[n][m] = B.v[n][m].lo();
      out.R_.v[n][m] = B.v[n][m].hi();
    }
  return out;
}
template <int DIM, int QF1, int Q, int GS, int QG1, typename NHT>
__device__ __noinline__ TwoBlk<float, DIM, Q> stencil_two_call(const StepConst &K, const float *sp, NHT NH,
                                                              int hL, int hR, float uFx, float uFy, float TF,
                                                              float sTF, SynK<float, Q> SK) {
  return stencil_two_body<DIM, QF1, Q, GS, QG1>(K, sp, NH, hL, hR, uFx, uFy, TF, sTF, SK);
}

// ---- a pair of stencil cells of which each normal node needs one ------------
// The trace of a normal node takes its outer neighbour and its two tangential
// neighbours from the upwind side only: cells 2 / 4 / 6 of the stencil where
// the node's v_n > 0 (upwind cell on the left/lower side), cells 3 / 5 / 7
// elsewhere.  So each of the pairs (2, 3), (4, 5), (6, 7) is moved into the
// face frame and synthesised along the normal axis for both cells, the
// selected cell's values are kept per normal node (bit k of upm: node k takes
// hA), and only those are moved and synthesised along the tangential axis,
// with the shift of the cell they came from.  The maps of the two axes act on
// different indices and commute, so every value is the one the full
// transformation of its cell gives (up to rounding order), for a quarter less
// arithmetic.  The Grad projection (zeroing coefficients in the face frame
// between the frame change and the synthesis) and, on the mixed path, a
// cell whose transformation must run in FP64 take both cells' full
// transformations instead (stencil_pair_full, out of line: rare).
template <typename R, int DIM, int QF1, int Q, int GS, int QG1, int DIRN>
__device__ __noinline__ Blk<R, Q, (DIM == 2 ? Q : 1)> stencil_pair_full(const StepConst &K, const R *sp,
                                                                      int NH, int hA, int hB,
                                                                      unsigned upm, R uFx, R uFy, R TF,
                                                                      R sTF, SynK<R, Q> SK) {
  constexpr int NY = DIM == 2 ? Q : 1;
  Blk<R, Q, NY> YA, YB;
  stencil_pops_body<R, DIM, QF1, Q, GS, QG1>(K, sp, NH, hA, uFx, uFy, TF, sTF, SK, YA);
  stencil_pops_body<R, DIM, QF1, Q, GS, QG1>(K, sp, NH, hB, uFx, uFy, TF, sTF, SK, YB);
#pragma unroll
  for (int n = 0; n < Q; ++n)
#pragma unroll
    for (int m = 0; m < NY; ++m) {
      const int k = DIRN == 0 ? n : m;
      YA.v[n][m] = (upm >> k & 1u) ? YA.v[n][m] : YB.v[n][m];
    }
  return YA;
}
template <typename R, int DIM, int QF1, int Q, int GS, int QG1, int DIRN, typename NHT>
__device__ __forceinline__ void stencil_pair_body(const StepConst &K, const R *sp, NHT NH, int hA, int hB,
                                                  unsigned upm, R uFx, R uFy, R TF, R sTF,
                                                  const SynK<R, Q> &SK, Blk<R, Q, (DIM == 2 ? Q : 1)> &Y) {
  if constexpr (DIM == 1) {  // no tangential axis: both cells in full, in line
    Blk<R, Q, 1> YB;
    stencil_pops<R, DIM, QF1, Q, GS, QG1>(K, sp, NH, hA, uFx, uFy, TF, sTF, SK, Y);
    stencil_pops<R, DIM, QF1, Q, GS, QG1>(K, sp, NH, hB, uFx, uFy, TF, sTF, SK, YB);
#pragma unroll
    for (int k = 0; k < Q; ++k) Y.v[k][0] = (upm >> k & 1u) ? Y.v[k][0] : YB.v[k][0];
    return;
  }
  using D = Dims<DIM, QF1, QG1>;
  constexpr int base = GS ? D::QF : 0, stride = GS ? QG1 : QF1;
  constexpr int IN = DIRN == 0 ? D::IUX : D::IUY, IT_ = DIRN == 0 ? D::IUY : D::IUX;
  const R uFn = DIRN == 0 ? uFx : uFy, uFt = DIRN == 0 ? uFy : uFx;
  const R unA = sp[IN * NH + hA], unB = sp[IN * NH + hB];
  const R utA = sp[IT_ * NH + hA], utB = sp[IT_ * NH + hB];
  const R TA = sp[D::IT * NH + hA], TB = sp[D::IT * NH + hB];
  bool full = K.grad_k != 0;
  if constexpr (is_mixed<R>()) {
    const R sTA = sp[D::IST * NH + hA], sTB = sp[D::IST * NH + hB], lim = K.xi_thr * sTF;
    full = full || fmaf(sTA, float(Nodes<Q>::cmax), fmaxf(fabsf(unA - uFn), fabsf(utA - uFt))) > lim ||
           fmaf(sTB, float(Nodes<Q>::cmax), fmaxf(fabsf(unB - uFn), fabsf(utB - uFt))) > lim;
  }
  if (full) {
    Y = stencil_pair_full<R, DIM, QF1, Q, GS, QG1, DIRN>(K, sp, NH, hA, hB, upm, uFx, uFy, TF, sTF, SK);
    return;
  }
  if constexpr (is_mixed<R>()) {
    // the two cells' normal stage in the two lanes of the paired FP32
    // instructions, then the selected values' tangential stage two normal
    // nodes at a time (an odd last node alone)
    const SynK<f2, Q> S(SK);
    const f2 dT(TA - TF, TB - TF), dT3 = f2(3) * dT;
    const DShift<f2> Cn = make_dshift(f2(unA - uFn, unB - uFn), dT, dT3);
    const DShift<f2> Ct = make_dshift(f2(utA - uFt, utB - uFt), dT, dT3);
    float Z[Q][Q];  // [normal node][tangential order]
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      f2 p[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int c = DIRN == 0 ? i + stride * j : j + stride * i;
        p[i] = f2(sp[(base + c) * NH + hA], sp[(base + c) * NH + hB]);
      }
      dshiftq(Cn, p);
      synqq(S, p);
#pragma unroll
      for (int k = 0; k < Q; ++k) Z[k][j] = pick((upm >> k & 1u) != 0u, p[k]);
    }
#pragma unroll
    for (int k = 0; k + 1 < Q; k += 2) {
      const DShift<f2> C = pick_rows((upm >> k & 1u) != 0u, (upm >> (k + 1) & 1u) != 0u, Ct);
      f2 t[Q];
#pragma unroll
      for (int j = 0; j < Q; ++j) t[j] = f2(Z[k][j], Z[k + 1][j]);
      dshiftq(C, t);
      synqq(S, t);
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        Y.v[DIRN == 0 ? k : j][DIRN == 0 ? j : k] = t[j].lo();
        Y.v[DIRN == 0 ? k + 1 : j][DIRN == 0 ? j : k + 1] = t[j].hi();
      }
    }
    if constexpr (Q % 2 == 1) {
      constexpr int k = Q - 1;
      const DShift<float> C = pick_row((upm >> k & 1u) != 0u, Ct);
      float t[Q];
#pragma unroll
      for (int j = 0; j < Q; ++j) t[j] = Z[k][j];
      dshiftq(C, t);
      synqq(SK, t);
#pragma unroll
      for (int j = 0; j < Q; ++j) Y.v[DIRN == 0 ? k : j][DIRN == 0 ? j : k] = t[j];
    }
    return;
  }
  {
    const R dTA = TA - TF, dTB = TB - TF;
    const DShift<R> CnA = make_dshift(unA - uFn, dTA, R(3) * dTA), CnB = make_dshift(unB - uFn, dTB, R(3) * dTB);
    const DShift<R> CtA = make_dshift(utA - uFt, dTA, R(3) * dTA), CtB = make_dshift(utB - uFt, dTB, R(3) * dTB);
    R Z[Q][Q];  // [normal node][tangential order]
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      R a[Q], b[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int c = DIRN == 0 ? i + stride * j : j + stride * i;
        a[i] = sp[(base + c) * NH + hA];
        b[i] = sp[(base + c) * NH + hB];
      }
      dshiftq(CnA, a); synqq(SK, a);
      dshiftq(CnB, b); synqq(SK, b);
#pragma unroll
      for (int k = 0; k < Q; ++k) Z[k][j] = (upm >> k & 1u) ? a[k] : b[k];
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const DShift<R> Ct = select_shift((upm >> k & 1u) != 0u, CtA, CtB);
      dshiftq(Ct, Z[k]);
      synqq(SK, Z[k]);
#pragma unroll
      for (int j = 0; j < Q; ++j) Y.v[DIRN == 0 ? k : j][DIRN == 0 ? j : k] = Z[k][j];
    }
  }
}
template <typename R, int DIM, int QF1, int Q, int GS, int QG1, int DIRN, typename NHT>
__device__ __noinline__ Blk<R, Q, (DIM == 2 ? Q : 1)> stencil_pair_call(const StepConst &K, const R *sp,
                                                                      NHT NH, int hA, int hB,
                                                                      unsigned upm, R uFx, R uFy, R TF,
                                                                      R sTF, SynK<R, Q> SK) {
  Blk<R, Q, (DIM == 2 ? Q : 1)> Y;
  stencil_pair_body<R, DIM, QF1, Q, GS, QG1, DIRN>(K, sp, NH, hA, hB, upm, uFx, uFy, TF, sTF, SK, Y);
  return Y;
}
template <typename R, int DIM, int QF1, int Q, int GS, int QG1, int DIRN, typename NHT>
__device__ __forceinline__ void stencil_pair(const StepConst &K, const R *sp, NHT NH, int hA, int hB,
                                             unsigned upm, R uFx, R uFy, R TF, R sTF, const SynK<R, Q> &SK,
                                             Blk<R, Q, (DIM == 2 ? Q : 1)> &Y) {
  if constexpr (is_mixed<R>())
    Y = stencil_pair_call<R, DIM, QF1, Q, GS, QG1, DIRN>(K, sp, NH, hA, hB, upm, uFx, uFy, TF, sTF, SK);
  else stencil_pair_body<R, DIM, QF1, Q, GS, QG1, DIRN>(K, sp, NH, hA, hB, upm, uFx, uFy, TF, sTF, SK, Y);
}

// v_n == +-0 exactly (a wall at rest puts the zero node of D1Q3 there)
__device__ __forceinline__ bool is_zero(double v) { return (__double_as_longlong(v) << 1) == 0; }
__device__ __forceinline__ bool is_zero(float v) { return (__float_as_int(v) << 1) == 0; }

// The trace of a face with a node at v_n = 0: that node takes the mean of its
// two one-sided traces, so that the face has no preferred side; the others
// take the upwind one as in reconstruct().  Out of line: only such faces run it.
template <typename R, int DIM, int QF1, int DIRN, int Q, int GS, int QG1>
__device__ __noinline__ void reconstruct_tie(const StepConst &K, const R *sp, int NH, const int *st, R uFx,
                                             R uFy, R TF, R sTF, R isTF, Blk<R, Q, (DIM == 2 ? Q : 1)> &out) {
  constexpr int NY = DIM == 2 ? Q : 1, NS = DIM == 2 ? 8 : 4;
  const SynK<R, Q> SK(isTF * isTF, isTF);
  const R uFn = DIRN == 0 ? uFx : uFy, uFt = DIRN == 0 ? uFy : uFx;
  const R lf = limiter_factor<R>(K.limiter);
  const R hl = R(0.5) * kc<R>(K.lam, K.cf.lam) * lf, h0 = R(0.5) * lf;
  const int lim = K.limiter;
  Blk<R, Q, NY> Y[NS];  // stencil: 0 left, 1 right, 2 outer-left, 3 outer-right, 4-7 tangential
#pragma unroll 1
  for (int s = 0; s < NS; ++s) stencil_pops<R, DIM, QF1, Q, GS, QG1>(K, sp, NH, st[s], uFx, uFy, TF, sTF, SK, Y[s]);
#pragma unroll
  for (int n = 0; n < Q; ++n)
#pragma unroll
    for (int m = 0; m < NY; ++m) {
      const int k = DIRN == 0 ? n : m, kt = DIRN == 0 ? m : n;
      const R c = R(Nodes<Q>::c(k)), ct = R(Nodes<Q>::c(kt));
      const R vn = sTF * c + uFn;
      const R offn = h0 - hl * fabs(vn), offt = -hl * (sTF * ct + uFt);
      R t[2];
#pragma unroll
      for (int side = 0; side < 2; ++side) {  // 0: left/lower upwind, 1: right/upper
        const R a = Y[side].v[n][m], b = Y[2 + side].v[n][m], cc = Y[1 - side].v[n][m];
        t[side] = a + offn * limit(a - b, cc - a, lim);
        if constexpr (DIM == 2) {
          const R lo = Y[4 + side].v[n][m], hi = Y[6 + side].v[n][m];
          t[side] += offt * limit(a - lo, hi - a, lim);
        }
      }
      out.v[n][m] = is_zero(vn) ? R(0.5) * (t[0] + t[1]) : (pos(vn) ? t[0] : t[1]);
    }
}

// First stage of the trace (normal limited slope) from the two cells beside
// the face (YL, YR) and the outer cell of the upwind side (Bo): A = the upwind
// value, out = A + offn L(A - Bo, downwind - A); two tangential nodes per paired
// instruction on the mixed path.
template <typename R, int DIM, int DIRN, int Q, typename LT>
__device__ __forceinline__ void trace_normal(const Blk<R, Q, (DIM == 2 ? Q : 1)> &YL,
                                             const Blk<R, Q, (DIM == 2 ? Q : 1)> &YR,
                                             const Blk<R, Q, (DIM == 2 ? Q : 1)> &Bo, unsigned upm,
                                             const R *offn, LT lim, Blk<R, Q, (DIM == 2 ? Q : 1)> &A,
                                             Blk<R, Q, (DIM == 2 ? Q : 1)> &out) {
  constexpr int NY = DIM == 2 ? Q : 1;
  if constexpr (is_mixed<R>() && DIM == 2) {
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const bool up = (upm >> k & 1u) != 0u;
#pragma unroll
      for (int t = 0; t < Q; t += 2) {
        const int n0 = DIRN == 0 ? k : t, m0 = DIRN == 0 ? t : k;
        if (t + 1 < Q) {
          const int n1 = DIRN == 0 ? k : t + 1, m1 = DIRN == 0 ? t + 1 : k;
          const f2 a = up ? f2(YL.v[n0][m0], YL.v[n1][m1]) : f2(YR.v[n0][m0], YR.v[n1][m1]);
          const f2 c = up ? f2(YR.v[n0][m0], YR.v[n1][m1]) : f2(YL.v[n0][m0], YL.v[n1][m1]);
          const f2 o = fma(f2(offn[k]), limit2(a - f2(Bo.v[n0][m0], Bo.v[n1][m1]), c - a, lim), a);
          A.v[n0][m0] = a.lo(); A.v[n1][m1] = a.hi();
          out.v[n0][m0] = o.lo(); out.v[n1][m1] = o.hi();
        } else {
          const R a = up ? YL.v[n0][m0] : YR.v[n0][m0];
          const R c = up ? YR.v[n0][m0] : YL.v[n0][m0];
          A.v[n0][m0] = a;
          out.v[n0][m0] = a + offn[k] * limit(a - Bo.v[n0][m0], c - a, lim);
        }
      }
    }
  } else {
#pragma unroll
    for (int n = 0; n < Q; ++n)
#pragma unroll
      for (int m = 0; m < NY; ++m) {
        const int k = DIRN == 0 ? n : m;
        const bool up = (upm >> k & 1u) != 0u;
        const R a = up ? YL.v[n][m] : YR.v[n][m];
        const R c = up ? YR.v[n][m] : YL.v[n][m];
        A.v[n][m] = a;
        out.v[n][m] = a + offn[k] * limit(a - Bo.v[n][m], c - a, lim);
      }
  }
}

// The zero normal node of an odd lattice has v_n = u_F,n, so v_n = 0 exactly
// wherever the face frame is at rest along the normal (a gas at rest, a wall
// at rest).  reconstruct() then traces that node from the right/upper side
// (pos(+-0) is false); this adds its trace from the left/lower side: the two
// cells beside the face give zl / zr (the node's row, one value per
// tangential node), cells 2 / 4 / 6 of the stencil are moved in full.  Out of
// line: only such faces call it.
template <typename R, int N> struct Row {
  R v[N];
};
template <typename R, int DIM, int QF1, int DIRN, int Q, int GS, int QG1>
__device__ __noinline__ Row<R, (DIM == 2 ? Q : 1)> zero_node_left(
    const StepConst &K, const R *sp, int NH, int hO, int hLo, int hHi, R uFx, R uFy, R TF, R sTF,
    SynK<R, Q> SK, Row<R, (DIM == 2 ? Q : 1)> zl, Row<R, (DIM == 2 ? Q : 1)> zr, R offn,
    Row<R, (DIM == 2 ? Q : 1)> offt, int lim) {
  constexpr int NY = DIM == 2 ? Q : 1, NZ = DIM == 2 ? Q : 1, KZ = Q / 2;
  Row<R, NZ> t;
  Blk<R, Q, NY> Y;
  stencil_pops_body<R, DIM, QF1, Q, GS, QG1>(K, sp, NH, hO, uFx, uFy, TF, sTF, SK, Y);
#pragma unroll
  for (int z = 0; z < NZ; ++z) {
    const R a = zl.v[z], b = DIRN == 0 ? Y.v[KZ][z] : Y.v[z][KZ];
    t.v[z] = a + offn * limit(a - b, zr.v[z] - a, lim);
  }
  if constexpr (DIM == 2) {
    Blk<R, Q, NY> H;
    stencil_pops_body<R, DIM, QF1, Q, GS, QG1>(K, sp, NH, hLo, uFx, uFy, TF, sTF, SK, Y);
    stencil_pops_body<R, DIM, QF1, Q, GS, QG1>(K, sp, NH, hHi, uFx, uFy, TF, sTF, SK, H);
#pragma unroll
    for (int z = 0; z < NZ; ++z) {
      const R a = zl.v[z];
      const R lo = DIRN == 0 ? Y.v[KZ][z] : Y.v[z][KZ], hi = DIRN == 0 ? H.v[KZ][z] : H.v[z][KZ];
      t.v[z] += offt.v[z] * limit(a - lo, hi - a, lim);
    }
  }
  return t;
}

// Limited half-step MUSCL trace of the populations of one lattice (Q nodes
// per axis) to the face (Eq. eq:InterfacePop), on node values divided by
// the weights (the trace is homogeneous of degree 1 in each node's values).  st[] = halo indices of the
// stencil: 0 left, 1 right, 2 outer-left, 3 outer-right, 4/5 lower tangential
// neighbour of left/right, 6/7 upper tangential neighbour of left/right.
// With a = upwind value, b = its outer neighbour, c = the downwind value, the
// trace is a + (1/2 - |v_n| lam/2) L(a - b, c - a) for either upwind side
// (L odd and symmetric), plus the tangential term -v_t lam/2 L(a - lo, hi - a).
// The offsets carry the factor lf of limit().
// TIE: 0 = no node of the face other than an odd lattice's zero node has
// v_n = 0 (checked by the caller), 1 = check here, 2 = the face has one (both
// run reconstruct_tie out of line).  The zero node at v_n = 0 (u_F,n = 0
// exactly) takes the mean of its two one-sided traces here: the right/upper
// one in line, the left/lower one from zero_node_left.
template <typename R, int DIM, int QF1, int DIRN, int Q, int TIE, int GS, int QG1, typename NHT, typename LT>
__device__ __forceinline__ void reconstruct(const StepConst &K, const R *sp, NHT NH, const int *st,
                                            R uFx, R uFy, R TF, R sTF, R isTF,
                                            Blk<R, Q, (DIM == 2 ? Q : 1)> &out, LT lim) {
  if constexpr (TIE == 2) {
    reconstruct_tie<R, DIM, QF1, DIRN, Q, GS, QG1>(K, sp, NH, st, uFx, uFy, TF, sTF, isTF, out);
    return;
  }
  constexpr int NY = DIM == 2 ? Q : 1;
  const SynK<R, Q> SK(isTF * isTF, isTF);
  const R uFn = DIRN == 0 ? uFx : uFy, uFt = DIRN == 0 ? uFy : uFx;
  // lim: K.limiter, or the same value as a compile-time type (CInt)
  const R lf = limiter_factor<R>(lim);
  const R hl = R(0.5) * kc<R>(K.lam, K.cf.lam) * lf, h0 = R(0.5) * lf;
  bool up[Q], tie = false;
  unsigned upm = 0u;
  R offn[Q], offt[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const R c = R(Nodes<Q>::c(k));
    const R vn = sTF * c + uFn;
    up[k] = pos(vn);
    upm |= up[k] ? 1u << k : 0u;
    if constexpr (TIE == 1) {
      if (Q % 2 == 0 || 2 * k != Q - 1) tie |= is_zero(vn);
    }
    offn[k] = h0 - hl * fabs(vn);
    offt[k] = -hl * (sTF * c + uFt);
  }
  if constexpr (TIE == 1) {
    if (tie) {
      reconstruct_tie<R, DIM, QF1, DIRN, Q, GS, QG1>(K, sp, NH, st, uFx, uFy, TF, sTF, isTF, out);
      return;
    }
  }
  // (no node but the zero node has v_n = 0 here: the tie path takes the others)
  constexpr bool ODD = Q % 2 == 1;
  constexpr int KZ = Q / 2, NZ = DIM == 2 ? Q : 1;
  Row<R, NZ> zl, zr;  // the zero node's row in the two cells beside the face
  Blk<R, Q, NY> A;
  {
    Blk<R, Q, NY> YL, YR, Bo;
    if constexpr (is_mixed<R>()) {
      const TwoBlk<float, DIM, Q> two = stencil_two_call<DIM, QF1, Q, GS, QG1>(K, sp, NH, st[0], st[1], uFx, uFy,
                                                                            TF, sTF, SK);
      YL = two.L;
      YR = two.R_;
    } else {
      stencil_pops<R, DIM, QF1, Q, GS, QG1>(K, sp, NH, st[0], uFx, uFy, TF, sTF, SK, YL);
      stencil_pops<R, DIM, QF1, Q, GS, QG1>(K, sp, NH, st[1], uFx, uFy, TF, sTF, SK, YR);
    }
    if constexpr (ODD) {
#pragma unroll
      for (int z = 0; z < NZ; ++z) {
        zl.v[z] = DIRN == 0 ? YL.v[KZ][z] : YL.v[z][KZ];
        zr.v[z] = DIRN == 0 ? YR.v[KZ][z] : YR.v[z][KZ];
      }
    }
    stencil_pair<R, DIM, QF1, Q, GS, QG1, DIRN>(K, sp, NH, st[2], st[3], upm, uFx, uFy, TF, sTF, SK, Bo);
    trace_normal<R, DIM, DIRN, Q>(YL, YR, Bo, upm, offn, lim, A, out);
  }
  if constexpr (DIM == 2) {
    Blk<R, Q, NY> Y, Dl;
    stencil_pair<R, DIM, QF1, Q, GS, QG1, DIRN>(K, sp, NH, st[4], st[5], upm, uFx, uFy, TF, sTF, SK, Y);
#pragma unroll
    for (int n = 0; n < Q; ++n)
#pragma unroll
      for (int m = 0; m < NY; ++m) Dl.v[n][m] = A.v[n][m] - Y.v[n][m];
    stencil_pair<R, DIM, QF1, Q, GS, QG1, DIRN>(K, sp, NH, st[6], st[7], upm, uFx, uFy, TF, sTF, SK, Y);
    if constexpr (is_mixed<R>()) {
#pragma unroll
      for (int k = 0; k < Q; ++k)
#pragma unroll
        for (int t = 0; t < Q; t += 2) {
          const int n0 = DIRN == 0 ? k : t, m0 = DIRN == 0 ? t : k;
          if (t + 1 < Q) {
            const int n1 = DIRN == 0 ? k : t + 1, m1 = DIRN == 0 ? t + 1 : k;
            const f2 a(A.v[n0][m0], A.v[n1][m1]);
            const f2 l = limit2(f2(Dl.v[n0][m0], Dl.v[n1][m1]), f2(Y.v[n0][m0], Y.v[n1][m1]) - a, lim);
            const f2 o = fma(f2(offt[t], offt[t + 1]), l, f2(out.v[n0][m0], out.v[n1][m1]));
            out.v[n0][m0] = o.lo(); out.v[n1][m1] = o.hi();
          } else {
            out.v[n0][m0] += offt[t] * limit(Dl.v[n0][m0], Y.v[n0][m0] - A.v[n0][m0], lim);
          }
        }
    } else {
#pragma unroll
      for (int n = 0; n < Q; ++n)
#pragma unroll
        for (int m = 0; m < NY; ++m) {
          const int kt = DIRN == 0 ? m : n;
          out.v[n][m] += offt[kt] * limit(Dl.v[n][m], Y.v[n][m] - A.v[n][m], lim);
        }
    }
  }
  if constexpr (ODD) {
    if (is_zero(uFn)) {
      Row<R, NZ> ot;
#pragma unroll
      for (int z = 0; z < NZ; ++z) ot.v[z] = offt[z];
      const Row<R, NZ> tl = zero_node_left<R, DIM, QF1, DIRN, Q, GS, QG1>(
          K, sp, NH, st[2], DIM == 2 ? st[4] : 0, DIM == 2 ? st[6] : 0, uFx, uFy, TF, sTF, SK, zl, zr,
          offn[KZ], ot, lim);
#pragma unroll
      for (int z = 0; z < NZ; ++z) {
        R &o = DIRN == 0 ? out.v[KZ][z] : out.v[z][KZ];
        o = R(0.5) * (o + tl.v[z]);
      }
    }
  }
}

// Gaussian expectations E[H_n(mu + X; TF)], X ~ N(0, Tb), n <= 3, with
// dT = Tb - TF: by the addition theorem of the H_n, H_n(mu; TF - Tb), i.e. the
// dimensional Hermite coefficients of an equilibrium {u_b, Tb} seen from the
// face frame (Gauss-Hermite quadrature is exact to degree 2q-1, so rho G W has
// them).
template <typename R, int N = 4>
__device__ __forceinline__ void gauss_he(R mu, R dT, R *e) {
  e[1] = mu;
  e[2] = fma(mu, mu, dT);
  if constexpr (N > 3) e[3] = mu * fma(mu, mu, R(3) * dT);
}
// order 4 (D1Q5): H_4(mu; TF - Tb) = mu^4 + 6 dT mu^2 + 3 dT^2
template <typename R>
__device__ __forceinline__ R gauss_he4(R mu, R dT) {
  const R mm = mu * mu;
  return fma(mm, fma(R(6), dT, mm), R(3) * dT * dT);
}

// ---- phase B: one face --------------------------------------------------------
// ITER: the iterated face frame (the predictor-corrector of the earlier scheme
// that Sec. IV.A.3 replaces by the averaged frame): the face frame is replaced
// by the interface state {u_b, T_b} until max(|u_b - u_F|/sqrt(T_F),
// |T_b - T_F|/T_F) < iter_tol (tested in FP64) or iter_max traces were made;
// a converged face uses the co-moving equilibrium rho W.  An iterate whose
// interface state is nonphysical ends the iteration and the face keeps the
// previous iterate.  Returns true when an iterated frame did not converge;
// ntrace receives the number of traces made (1 for the averaged frame).
// QL: the f-lattice of the face, QF1 or (a multiscale face whose two cells
// are both on the low-order lattice) 3; the face record keeps the storage
// layout of QF1, with zero coefficients beyond QL.
template <typename R, int DIM, int QF1, int DIRN, bool ITER, bool TIE = false, int QL = QF1, int QG1 = 3,
          typename NHT = int, typename LT = int>
__device__ __forceinline__ bool face_flux(const StepConst &K, const R *sp, NHT NH, const int *st,
                                          R *fp, int NFACES, int fidx, int &ntrace, LT lim);

// does a node of either lattice other than an odd lattice's zero node have
// v_n = 0 exactly in the face frame (u_F,n = -c_k sqrt(T_F) to the last bit:
// rare)?  Such a face takes the out-of-line trace, where that node takes the
// mean of its two one-sided traces.  The zero node (v_n = u_F,n: 0 for a gas
// or a wall at rest) is averaged in line by reconstruct().
template <typename R, int QF1, int QG1 = 3>
__device__ __forceinline__ bool face_has_tie(R uFn, R sTF) {
  bool t = false;
#pragma unroll
  for (int k = 0; k < QF1; ++k)
    if (QF1 % 2 == 0 || 2 * k != QF1 - 1) t |= is_zero(sTF * R(Nodes<QF1>::c(k)) + uFn);
#pragma unroll
  for (int k = 0; k < QG1; ++k)
    if (QG1 % 2 == 0 || 2 * k != QG1 - 1) t |= is_zero(sTF * R(Nodes<QG1>::c(k)) + uFn);
  return t;
}
// the averaged-frame face with a node at v_n = 0, out of line (rare)
template <typename R, int DIM, int QF1, int DIRN, int QL, int QG1>
__device__ __noinline__ bool face_flux_tie(const StepConst &K, const R *sp, int NH, const int *st, R *fp,
                                           int NFACES, int fidx, int &ntrace) {
  return face_flux<R, DIM, QF1, DIRN, false, true, QL, QG1>(K, sp, NH, st, fp, NFACES, fidx, ntrace, K.limiter);
}

template <typename R, int DIM, int QF1, int DIRN, bool ITER, bool TIE, int QL, int QG1, typename NHT, typename LT>
__device__ __forceinline__ bool face_flux(const StepConst &K, const R *sp, NHT NH, const int *st,
                                          R *fp, int NFACES, int fidx, int &ntrace, LT lim) {
  static_assert(QL >= QG1, "the equilibrium's Gaussian moments are built to the f-lattice's order");
  using D = Dims<DIM, QF1, QG1>;
  constexpr int NYF = DIM == 2 ? QL : 1, NYG = D::NYG;
  const int hL = st[0], hR = st[1];
  R uFx = R(0.5) * (sp[D::IUX * NH + hL] + sp[D::IUX * NH + hR]);
  R uFy = DIM == 2 ? R(0.5) * (sp[D::IUY * NH + hL] + sp[D::IUY * NH + hR]) : R(0);
  R TF = R(0.5) * (sp[D::IT * NH + hL] + sp[D::IT * NH + hR]);
  R sTF = sqrt(TF), isTF = R(1) / sTF;
  if constexpr (!ITER && !TIE) {
    if (face_has_tie<R, QL, QG1>(DIRN == 0 ? uFx : uFy, sTF))
      return face_flux_tie<R, DIM, QF1, DIRN, QL, QG1>(K, sp, NH, st, fp, NFACES, fidx, ntrace);
  }
  constexpr int TMODE = ITER ? 1 : (TIE ? 2 : 0);

  Blk<R, QL, NYF> Fb;
  Blk<R, QG1, NYG> Gb;
  R rk, mx, my, Tb;
  bool converged = false, noconv = false;
  R pFx = uFx, pFy = uFy, pT = TF;  // previous iterate's frame
  int it = 0;
  bool fallback = false;
  ntrace = 0;
  while (true) {
    ++ntrace;
    reconstruct<R, DIM, QF1, DIRN, QL, TMODE, 0, QG1>(K, sp, NH, st, uFx, uFy, TF, sTF, isTF, Fb, lim);
    reconstruct<R, DIM, QF1, DIRN, QG1, TMODE, 1, QG1>(K, sp, NH, st, uFx, uFy, TF, sTF, isTF, Gb, lim);
    anaq_xy(AnaK<R, QL>(TF, sTF), Fb);
    anaq_xy(AnaK<R, QG1>(TF, sTF), Gb);
    // interface moments in the face frame (all carry the factor kappa1): rho,
    // mu = u - u_F, C_v rho T = (sum |v - u_F|^2 f - rho |mu|^2)/2 + sum g
    rk = Fb.v[0][0];
    const R irk = R(1) / rk;
    mx = Fb.v[1][0] * irk;
    my = R(0);
    R S2 = fma(R(DIM) * TF, rk, Fb.v[2][0]);
    if constexpr (DIM == 2) { my = Fb.v[0][1] * irk; S2 += Fb.v[0][2]; }
    const R ek = R(0.5) * (S2 - rk * (mx * mx + my * my)) + Gb.v[0][0];
    Tb = ek * irk * kc<R>(K.inv_cv, K.cf.inv_cv);
    if constexpr (!ITER) {
      break;
    } else {
      if (fallback) break;
      if (!(rk > R(0) && Tb > R(0) && isfinite(Tb))) {
        if (it > 0) {  // retrace at the previous (physical) iterate
          uFx = pFx; uFy = pFy; TF = pT;
          sTF = sqrt(TF); isTF = R(1) / sTF;
          fallback = true;
          continue;
        }
        break;
      }
      const double mxd = mx, myd = my;
      const double err = fmax(sqrt(mxd * mxd + myd * myd) / sqrt((double)TF),
                              fabs((double)Tb - (double)TF) / (double)TF);
      if (err < K.iter_tol) { converged = true; break; }
      if (++it >= (K.iter_max > 0 ? K.iter_max : 1)) break;
      pFx = uFx; pFy = uFy; pT = TF;
      uFx = uFx + mx;
      if constexpr (DIM == 2) uFy = uFy + my;
      TF = Tb;
      sTF = sqrt(TF); isTF = R(1) / sTF;
    }
  }
  if constexpr (ITER) noconv = !converged;
  const R dTb = Tb - TF;

  // equilibrium (closed form of rho G_{u,T}^{lambda_F} W), weighted by kappa2/kappa1;
  // a converged iterated frame is co-moving: rho W
  R ex[QL], ey[QL];
  ex[0] = R(1); gauss_he<R, QL>(mx, dTb, ex);
  if constexpr (QL == 5) ex[4] = gauss_he4(mx, dTb);
  ey[0] = R(1);
#pragma unroll
  for (int a = 1; a < QL; ++a) ey[a] = R(0);
  if constexpr (DIM == 2) {
    gauss_he<R, QL>(my, dTb, ey);
    if constexpr (QL == 5) ey[4] = gauss_he4(my, dTb);
  }
  if constexpr (ITER) {
    if (converged) {
#pragma unroll
      for (int a = 1; a < QL; ++a) ex[a] = ey[a] = R(0);
    }
  }
  // an interface state with rho <= 0 or T <= 0 has no equilibrium: poison the
  // face so that both adjacent cells are flagged nonphysical
  const bool phys = rk > R(0) && Tb > R(0);
  const bool gk = DIM == 2 && K.grad_k;
  const R re = phys ? kc<R>(K.kr, K.cf.kr) * rk : qnan<R>(), ge = re * kc<R>(K.gfac, K.cf.gfac) * Tb;
  // rho E[H_a] E[H_b] added as (rho E[H_a]) E[H_b]: one multiply-add per coefficient
  R rex[QL], gex[QG1];
#pragma unroll
  for (int a = 0; a < QL; ++a) rex[a] = a == 0 ? re : re * ex[a];
#pragma unroll
  for (int a = 0; a < QG1; ++a) gex[a] = a == 0 ? ge : ge * ex[a];
#pragma unroll
  for (int a = 0; a < QL; ++a)
#pragma unroll
    for (int b = 0; b < NYF; ++b)
      Fb.v[a][b] = b == 0 ? Fb.v[a][b] + ((gk && a > QL - 1) ? R(0) : rex[a])
                          : fma((gk && a + b > QL - 1) ? R(0) : rex[a], ey[b], Fb.v[a][b]);
#pragma unroll
  for (int a = 0; a < QG1; ++a)
#pragma unroll
    for (int b = 0; b < NYG; ++b)
      Gb.v[a][b] = b == 0 ? Gb.v[a][b] + ((gk && a > QG1 - 1) ? R(0) : gex[a])
                          : fma((gk && a + b > QG1 - 1) ? R(0) : gex[a], ey[b], Gb.v[a][b]);
  // Appendix C form: transport v_n^{lambda_F} phi in the face frame
  if (K.appc) {
    const R un = DIRN == 0 ? uFx : uFy;
    vmul<DIRN>(un, TF, Fb);
    vmul<DIRN>(un, TF, Gb);
  }
  if constexpr (is_mixed<R>()) {
    // Mixed path: the face's conserved fluxes (mass, momentum, energy along the
    // normal), evaluated once here so that the two adjacent cells add exactly
    // opposite amounts to their FP64 moment sums.  They are moments of order
    // <= 3 of v_n phi (<= 1 of v_n g), which every frame transformation keeps
    // (Eq. eq:Mcondition), so the face frame gives the same values as the cell
    // frames of Eq. fluxEq.  C = dimensional coefficients of v_n phi (low
    // orders): x H_k = H_{k+1} + k T_F H_{k-1} along the normal.
    // (A multiscale face of two low cells has no order-3 coefficient along
    // the normal: H_3 vanishes on the D1Q3 nodes.  Its energy flux is not
    // used with the main flux form: a low cell takes its own frame's value.)
    const R un = DIRN == 0 ? uFx : uFy;
    R b3 = R(0);
    if constexpr (QL > 3) b3 = DIRN == 0 ? Fb.v[3][0] : Fb.v[0][DIM == 2 ? 3 : 0];
    R C00, C10, C01 = R(0), C20, C02 = R(0), CG;
    if (K.appc) {  // Fb, Gb already hold v_n phi
      C00 = Fb.v[0][0]; C10 = Fb.v[1][0]; C20 = Fb.v[2][0]; CG = Gb.v[0][0];
      if constexpr (DIM == 2) { C01 = Fb.v[0][1]; C02 = Fb.v[0][2]; }
    } else if constexpr (DIRN == 0) {
      C00 = fma(un, Fb.v[0][0], Fb.v[1][0]);
      C10 = fma(un, Fb.v[1][0], fma(TF, Fb.v[0][0], Fb.v[2][0]));
      C20 = fma(un, Fb.v[2][0], fma(TF + TF, Fb.v[1][0], b3));
      CG = fma(un, Gb.v[0][0], Gb.v[1][0]);
      if constexpr (DIM == 2) {
        C01 = fma(un, Fb.v[0][1], Fb.v[1][1]);
        C02 = fma(un, Fb.v[0][2], Fb.v[1][2]);
      }
    } else {
      C00 = fma(un, Fb.v[0][0], Fb.v[0][1]);
      C01 = fma(un, Fb.v[0][1], fma(TF, Fb.v[0][0], Fb.v[0][2]));
      C02 = fma(un, Fb.v[0][2], fma(TF + TF, Fb.v[0][1], b3));
      C10 = fma(un, Fb.v[1][0], Fb.v[1][1]);
      C20 = fma(un, Fb.v[2][0], Fb.v[2][1]);
      CG = fma(un, Gb.v[0][0], Gb.v[0][1]);
    }
    // v = u_F + x: sum v_n phi, sum v v_n phi, sum (|v|^2/2) v_n phi + sum v_n g
    const R c2 = fma(R(DIM) * TF, C00, C20 + C02);
    fp[(D::FJ + 0) * NFACES + fidx] = C00;
    fp[(D::FJ + 1) * NFACES + fidx] = fma(uFx, C00, C10);
    fp[(D::FJ + 2) * NFACES + fidx] = fma(uFy, C00, C01);
    fp[(D::FJ + 3) * NFACES + fidx] =
        R(0.5) * ((uFx * uFx + uFy * uFy) * C00 + R(2) * (uFx * C10 + uFy * C01) + c2) + CG;
    fp[D::FST * NFACES + fidx] = sTF;
  }
#pragma unroll
  for (int a = 0; a < QF1; ++a)
#pragma unroll
    for (int b = 0; b < D::NYF; ++b) {
      if constexpr (QL == QF1) fp[(a + QF1 * b) * NFACES + fidx] = Fb.v[a][b];
      else fp[(a + QF1 * b) * NFACES + fidx] = (a < QL && b < NYF) ? Fb.v[a < QL ? a : 0][b < NYF ? b : 0] : R(0);
    }
#pragma unroll
  for (int a = 0; a < QG1; ++a)
#pragma unroll
    for (int b = 0; b < NYG; ++b) fp[(D::QF + a + QG1 * b) * NFACES + fidx] = Gb.v[a][b];
  fp[D::FUX * NFACES + fidx] = uFx;
  fp[D::FUY * NFACES + fidx] = uFy;
  fp[D::FT * NFACES + fidx] = TF;
  return noconv;
}

// ---- phase C: one cell --------------------------------------------------------
// Mixed path: the conserved moments of each cell (rho, rho u, rho E: Eqs.
// eq::ConservationLaws, eq:E) are kept in FP64 (State::M) and accumulated
// there: -dt/dx times each face's conserved flux (the same FP32 value for both
// cells of a face) is added.  The collision terms conserve them.
struct MomAcc {
  double r, jx, jy, e;
};

// one face's phi (dimensional coefficients in the face frame) moved into the
// cell frame {u, T} (sT = sqrt T, read by the mixed path's FP64 test only)
template <typename R, int DIM, int QF1, int QG1>
__device__ __forceinline__ void face_contrib_body(const StepConst &K, const R *fp, int NFACES, int fidx,
                                                  R ux, R uy, R T, R sT, Blk<R, QF1, Dims<DIM, QF1>::NYF> &X,
                                                  Blk<R, QG1, Dims<DIM, QF1, QG1>::NYG> &Y) {
  using D = Dims<DIM, QF1, QG1>;
#pragma unroll
  for (int a = 0; a < QF1; ++a)
#pragma unroll
    for (int b = 0; b < D::NYF; ++b) X.v[a][b] = fp[(a + QF1 * b) * NFACES + fidx];
#pragma unroll
  for (int a = 0; a < QG1; ++a)
#pragma unroll
    for (int b = 0; b < D::NYG; ++b) Y.v[a][b] = fp[(D::QF + a + QG1 * b) * NFACES + fidx];
  const R uFx = fp[D::FUX * NFACES + fidx], uFy = fp[D::FUY * NFACES + fidx];
  const R TF = fp[D::FT * NFACES + fidx];
  const R sTF = is_mixed<R>() ? fp[D::FST * NFACES + fidx] : R(0);
  move_frame<R, DIM, QF1>(K, uFx, uFy, TF, sTF, ux, uy, T, sT, X);
  move_frame<R, DIM, QG1>(K, uFx, uFy, TF, sTF, ux, uy, T, sT, Y);
  if constexpr (DIM == 2) {
    if (K.grad_k) { grad_mask(X); grad_mask(Y); }
  }
}
// The mixed path moves a face's phi in one out-of-line copy (returned by
// value, in registers), like the stencil transformation.
template <typename R, int DIM, int QF1, int QG1> struct FaceContrib {
  Blk<R, QF1, Dims<DIM, QF1>::NYF> X;
  Blk<R, QG1, Dims<DIM, QF1, QG1>::NYG> Y;
};
template <typename R, int DIM, int QF1, int QG1>
__device__ __noinline__ FaceContrib<R, DIM, QF1, QG1> face_contrib_call(const StepConst &K, const R *fp,
                                                                      int NFACES, int fidx, R ux, R uy, R T,
                                                                      R sT) {
  FaceContrib<R, DIM, QF1, QG1> c;
  face_contrib_body<R, DIM, QF1, QG1>(K, fp, NFACES, fidx, ux, uy, T, sT, c.X, c.Y);
  return c;
}
template <typename R, int DIM, int QF1, int QG1>
__device__ __forceinline__ void face_contrib(const StepConst &K, const R *fp, int NFACES, int fidx, R ux,
                                             R uy, R T, R sT, Blk<R, QF1, Dims<DIM, QF1>::NYF> &X,
                                             Blk<R, QG1, Dims<DIM, QF1, QG1>::NYG> &Y) {
  if constexpr (is_mixed<R>()) {
    const FaceContrib<R, DIM, QF1, QG1> c =
        face_contrib_call<R, DIM, QF1, QG1>(K, fp, NFACES, fidx, ux, uy, T, sT);
    X = c.X;
    Y = c.Y;
  } else {
    face_contrib_body<R, DIM, QF1, QG1>(K, fp, NFACES, fidx, ux, uy, T, sT, X, Y);
  }
}

// The mixed path moves a cell's two faces along one direction into its frame
// in one out-of-line call, the upper face in the low lane and the lower face
// in the high lane of the paired FP32 instructions (each lane its own face
// frame's shift, the same arithmetic as face_contrib_body), and returns their
// difference, upper minus lower.  A face whose transformation must run in
// FP64 takes both faces through face_contrib_body instead.
template <int DIM, int QF1, int QG1, typename NFT>
__device__ __noinline__ FaceContrib<float, DIM, QF1, QG1> face_pair_diff_call(const StepConst &K, const float *fp,
                                                                             NFT NFACES, int flo, int fhi,
                                                                             float ux, float uy, float T,
                                                                             float sT) {
  using D = Dims<DIM, QF1, QG1>;
  constexpr int NYF = D::NYF, NYG = D::NYG;
  FaceContrib<float, DIM, QF1, QG1> out;
  const float uxh = fp[D::FUX * NFACES + fhi], uxl = fp[D::FUX * NFACES + flo];
  const float uyh = DIM == 2 ? fp[D::FUY * NFACES + fhi] : 0.f, uyl = DIM == 2 ? fp[D::FUY * NFACES + flo] : 0.f;
  const float Th = fp[D::FT * NFACES + fhi], Tl = fp[D::FT * NFACES + flo];
  const float lim = K.xi_thr * sT;
  const bool full =
      fmaf(fp[D::FST * NFACES + fhi], float(Nodes<QF1>::cmax), fmaxf(fabsf(uxh - ux), fabsf(uyh - uy))) > lim ||
      fmaf(fp[D::FST * NFACES + flo], float(Nodes<QF1>::cmax), fmaxf(fabsf(uxl - ux), fabsf(uyl - uy))) > lim;
  if (full) {
    Blk<float, QF1, NYF> Xl;
    Blk<float, QG1, NYG> Yl;
    face_contrib_body<float, DIM, QF1, QG1>(K, fp, NFACES, fhi, ux, uy, T, sT, out.X, out.Y);
    face_contrib_body<float, DIM, QF1, QG1>(K, fp, NFACES, flo, ux, uy, T, sT, Xl, Yl);
#pragma unroll
    for (int p = 0; p < QF1; ++p)
#pragma unroll
      for (int q = 0; q < NYF; ++q) out.X.v[p][q] = out.X.v[p][q] - Xl.v[p][q];
#pragma unroll
    for (int p = 0; p < QG1; ++p)
#pragma unroll
      for (int q = 0; q < NYG; ++q) out.Y.v[p][q] = out.Y.v[p][q] - Yl.v[p][q];
    return out;
  }
  Blk<f2, QF1, NYF> X;
  Blk<f2, QG1, NYG> Y;
#pragma unroll
  for (int a = 0; a < QF1; ++a)
#pragma unroll
    for (int b = 0; b < NYF; ++b)
      X.v[a][b] = f2(fp[(a + QF1 * b) * NFACES + fhi], fp[(a + QF1 * b) * NFACES + flo]);
#pragma unroll
  for (int a = 0; a < QG1; ++a)
#pragma unroll
    for (int b = 0; b < NYG; ++b)
      Y.v[a][b] = f2(fp[(D::QF + a + QG1 * b) * NFACES + fhi], fp[(D::QF + a + QG1 * b) * NFACES + flo]);
  const f2 dT(Th - T, Tl - T), dT3 = f2(3) * dT;
  const DShift<f2> Cx = make_dshift(f2(uxh - ux, uxl - ux), dT, dT3);
  shift_x(Cx, X);
  shift_x(Cx, Y);
  if constexpr (DIM == 2) {
    const DShift<f2> Cy = make_dshift(f2(uyh - uy, uyl - uy), dT, dT3);
    shift_y(Cy, X);
    shift_y(Cy, Y);
    if (K.grad_k) { grad_mask(X); grad_mask(Y); }
  }
#pragma unroll
  for (int a = 0; a < QF1; ++a)
#pragma unroll
    for (int b = 0; b < NYF; ++b) out.X.v[a][b] = X.v[a][b].lo() - X.v[a][b].hi();
#pragma unroll
  for (int a = 0; a < QG1; ++a)
#pragma unroll
    for (int b = 0; b < NYG; ++b) out.Y.v[a][b] = Y.v[a][b].lo() - Y.v[a][b].hi();
  return out;
}

// The two faces of the cell along DIRN (lower face flo, upper face fhi):
// F += -dt/dx [(v . n) G phi_hi - (v . n) G phi_lo] (Eq. fluxEq; the
// multiplication by v_n in the cell frame is linear, so it is applied once to
// the difference), or -dt/dx [G (v_F . n phi)_hi - G (v_F . n phi)_lo] in
// the Appendix C form.
// (MS, low: the fluxes are projected onto the cell's low-order lattice before
// the multiplication by v_n, which on that lattice has no order-3 term.)
template <typename R, int DIM, int QF1, int DIRN, bool MS = false, int QG1 = 3, typename NFT = int>
__device__ __forceinline__ void add_faces(const StepConst &K, const R *fp, NFT NFACES, int flo, int fhi,
                                          R ux, R uy, R T, R sT, Blk<R, QF1, Dims<DIM, QF1>::NYF> &F,
                                          Blk<R, QG1, Dims<DIM, QF1, QG1>::NYG> &G, MomAcc &M,
                                          bool low = false) {
  using D = Dims<DIM, QF1, QG1>;
  Blk<R, QF1, D::NYF> DX;
  Blk<R, QG1, D::NYG> DY;
  if constexpr (is_mixed<R>()) {
    const FaceContrib<float, DIM, QF1, QG1> c =
        face_pair_diff_call<DIM, QF1, QG1>(K, fp, NFACES, flo, fhi, ux, uy, T, sT);
    DX = c.X;
    DY = c.Y;
  } else {
    Blk<R, QF1, D::NYF> X;
    Blk<R, QG1, D::NYG> Y;
    face_contrib<R, DIM, QF1, QG1>(K, fp, NFACES, flo, ux, uy, T, sT, DX, DY);
    face_contrib<R, DIM, QF1, QG1>(K, fp, NFACES, fhi, ux, uy, T, sT, X, Y);
#pragma unroll
    for (int p = 0; p < QF1; ++p)
#pragma unroll
      for (int q = 0; q < D::NYF; ++q) DX.v[p][q] = X.v[p][q] - DX.v[p][q];
#pragma unroll
    for (int p = 0; p < QG1; ++p)
#pragma unroll
      for (int q = 0; q < D::NYG; ++q) DY.v[p][q] = Y.v[p][q] - DY.v[p][q];
  }
  if constexpr (MS) {
    if (low) ms_project(DX, K.grad_k);
  }
  if (!K.appc) {
    const R un = DIRN == 0 ? ux : uy;
    vmul<DIRN>(un, T, DX);
    vmul<DIRN>(un, T, DY);
  }
  const R ml = -kc<R>(K.lam, K.cf.lam);
#pragma unroll
  for (int p = 0; p < QF1; ++p)
#pragma unroll
    for (int q = 0; q < D::NYF; ++q) F.v[p][q] = fma(ml, DX.v[p][q], F.v[p][q]);
#pragma unroll
  for (int p = 0; p < QG1; ++p)
#pragma unroll
    for (int q = 0; q < D::NYG; ++q) G.v[p][q] = fma(ml, DY.v[p][q], G.v[p][q]);
  if constexpr (is_mixed<R>()) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (DIM == 1 && j == 2) continue;
      const double d = (double)fp[(D::FJ + j) * NFACES + fhi] - (double)fp[(D::FJ + j) * NFACES + flo];
      double &m = j == 0 ? M.r : (j == 1 ? M.jx : (j == 2 ? M.jy : M.e));
      if (MS && j == 3 && low && !K.appc) continue;
      m = fma(-K.lam, d, m);
    }
    if constexpr (MS) {
      // A low cell with the main flux form: its lattice lacks the third-order
      // moment along the normal that the energy flux takes in another frame,
      // so its energy changes by the cell-frame moment of the projected
      // v_n phi (the FP64 path's and the oracle's value), not the face's:
      // with v = u + x, sum |v|^2/2 v_n phi = (|u|^2 X_0 + 2 u . X_1 +
      // D T X_0 + X_2x + X_2y) / 2, plus sum v_n g = Y_0.
      if (low && !K.appc) {
        const double dux = ux, duy = DIM == 2 ? (double)uy : 0.0, dT = T;
        const double X0 = DX.v[0][0], X1x = DX.v[1][0], X2x = DX.v[2][0];
        const double X1y = DIM == 2 ? (double)DX.v[0][1] : 0.0, X2y = DIM == 2 ? (double)DX.v[0][2] : 0.0;
        const double e = 0.5 * ((dux * dux + duy * duy + DIM * dT) * X0 + 2.0 * (dux * X1x + duy * X1y) +
                                X2x + X2y) + (double)DY.v[0][0];
        M.e = fma(-K.lam, e, M.e);
      }
    }
  }
}

template <typename R, int DIM, int QF1, int BX, int BY, bool MS = false, int QG1 = 3>
__device__ __forceinline__ void update_cell(const StepConst &K, const State<R> &S, const State<R> &O,
                                            const R *fp, int cx, int cy, int j, int k, R &vmax,
                                            unsigned &flags, bool low = false) {
  using D = Dims<DIM, QF1, QG1>;
  using TL = Tile<DIM, BX, BY, QF1, QG1>;
  const size_t N = (size_t)K.nx * (DIM == 2 ? K.ny : 1);
  const size_t c = (size_t)k * K.nx + j;
  Blk<R, QF1, D::NYF> F;
  Blk<R, QG1, D::NYG> G;
#pragma unroll
  for (int i = 0; i < D::QF; ++i) F.v[i % QF1][i / QF1] = S.f[i * N + c];
#pragma unroll
  for (int i = 0; i < D::QG; ++i) G.v[i % QG1][i / QG1] = S.g[i * N + c];
  const R ux = S.ux[c], uy = DIM == 2 ? S.uy[c] : R(0), T = S.T[c];
  const R sT = is_mixed<R>() ? sqrt(T) : R(0);
  if constexpr (MS) {
    if (low) ms_project(F, K.grad_k);
  }
  const R rho = F.v[0][0];
  MomAcc M;
  if constexpr (is_mixed<R>()) {
    // the cell's conserved moments, kept in FP64
    M.r = S.M[c];
    M.jx = S.M[N + c];
    M.jy = DIM == 2 ? S.M[2 * N + c] : 0.0;
    M.e = S.M[3 * N + c];
  }
  // DUGKS update in the cell frame (Eq. eq:FinalUpdateDUGKS):
  // a1 phi~ + a2 phi^eq - dt/dx sum_faces (+-) F, after the first QE half
  // step (qe on the order-3 content of f and order-1 of g): one scaling
  const R a1 = kc<R>(K.a1, K.cf.a1), aq = a1 * kc<R>(K.qe, K.cf.qe);
#pragma unroll
  for (int a = 0; a < QF1; ++a)
#pragma unroll
    for (int b = 0; b < D::NYF; ++b) F.v[a][b] *= a + b == 3 ? aq : a1;
#pragma unroll
  for (int a = 0; a < QG1; ++a)
#pragma unroll
    for (int b = 0; b < D::NYG; ++b) G.v[a][b] *= a + b == 1 ? aq : a1;
  // fluxes through the faces, in a fixed order: x, then y
  add_faces<R, DIM, QF1, 0, MS, QG1>(K, fp, CInt<TL::NFACES>{}, cy * (BX + 1) + cx, cy * (BX + 1) + cx + 1, ux, uy, T, sT, F,
                                G, M, low);
  if constexpr (DIM == 2)
    add_faces<R, DIM, QF1, 1, MS, QG1>(K, fp, CInt<TL::NFACES>{}, TL::NFX + cy * BX + cx, TL::NFX + (cy + 1) * BX + cx, ux, uy,
                                  T, sT, F, G, M, low);
  F.v[0][0] += kc<R>(K.a2, K.cf.a2) * rho;
  G.v[0][0] += kc<R>(K.a2, K.cf.a2) * kc<R>(K.gfac, K.cf.gfac) * T * rho;

  // new moments (Eqs. eq::ConservationLaws, eq:E) and the new co-moving frame
  R uxn, uyn, Tout;
  bool ok;
  if constexpr (!is_mixed<R>()) {
    const R rn = F.v[0][0], irn = R(1) / rn;
    const R mx = F.v[1][0] * irn;
    R my = R(0), S2 = fma(R(DIM) * T, rn, F.v[2][0]);
    if constexpr (DIM == 2) { my = F.v[0][1] * irn; S2 += F.v[0][2]; }
    const R en = R(0.5) * (S2 - rn * (mx * mx + my * my)) + G.v[0][0];
    const R Tn = en * irn * kc<R>(K.inv_cv, K.cf.inv_cv);
    uxn = ux + mx; uyn = DIM == 2 ? uy + my : R(0); Tout = Tn;
    ok = rn > R(0) && Tn > R(0) && isfinite(rn) && isfinite(Tn) && isfinite(uxn) && isfinite(uyn);
    if (ok) {
      const R dT = T - Tn, dT3 = R(3) * dT;
      const DShift<R> Cx = make_dshift(-mx, dT, dT3);
      shift_x(Cx, F); shift_x(Cx, G);
      if constexpr (DIM == 2) {
        const DShift<R> Cy = make_dshift(-my, dT, dT3);
        shift_y(Cy, F); shift_y(Cy, G);
      }
    }
  } else {
    // FP64: the new moments and frame; the frame is stored rounded to FP32
    // and the populations are moved into exactly that stored frame
    const double rn = M.r, irn = rcp_nr1(rn);
    const double ux64 = M.jx * irn, uy64 = DIM == 2 ? M.jy * irn : 0.0;
    const double Tn = (M.e - 0.5 * rn * (ux64 * ux64 + uy64 * uy64)) * irn * K.inv_cv;
    ok = rn > 0.0 && Tn > 0.0 && isfinite(rn) && isfinite(Tn) && isfinite(ux64) && isfinite(uy64);
    uxn = (R)ux64; uyn = (R)uy64; Tout = (R)Tn;
    ok = ok && Tout > R(0) && isfinite(Tout);
    // the conserved coefficients (still in the old frame) are the FP64 sums,
    // rounded once: the FP32 update alone drifts (a1 + a2 != 1 in FP32, and
    // the two cells of a face move its flux through different frames)
    const double cux = ux, cuy = uy, T64 = T;
    const double a10 = fma(-cux, rn, M.jx), a01 = DIM == 2 ? fma(-cuy, rn, M.jy) : 0.0;
    F.v[0][0] = (R)rn;
    F.v[1][0] = (R)a10;
    double c2 = fma(DIM * T64, rn, (double)F.v[2][0]);
    if constexpr (DIM == 2) { F.v[0][1] = (R)a01; c2 += (double)F.v[0][2]; }
    G.v[0][0] = (R)(M.e - 0.5 * ((cux * cux + cuy * cuy) * rn + 2.0 * (cux * a10 + cuy * a01) + c2));
    if (ok) {
      const R sTn = sqrt(Tout);
      move_frame<R, DIM, QF1>(K, ux, uy, T, sT, uxn, uyn, Tout, sTn, F);
      move_frame<R, DIM, QG1>(K, ux, uy, T, sT, uxn, uyn, Tout, sTn, G);
    }
  }
  if (ok) {
    if constexpr (DIM == 2) {
      if (K.grad_k) { grad_mask(F); grad_mask(G); }
    }
    if (K.qe != 1.0) qe_scale(F, G, kc<R>(K.qe, K.cf.qe));  // (BGK: no QE step)
    const R cm = (MS && low) ? R(Nodes<3>::cmax) : R(Nodes<QF1>::cmax);
    vmax = fmax(vmax, fmax(fabs(uxn), fabs(uyn)) + sqrt(Tout) * cm);
  } else {
    flags |= FLAG_NONPHYSICAL;
    uxn = ux; uyn = uy; Tout = T;
  }
  if constexpr (MS) {
    if (low) ms_project(F, K.grad_k);  // back to the low lattice's storage
  }
#pragma unroll
  for (int i = 0; i < D::QF; ++i) O.f[i * N + c] = F.v[i % QF1][i / QF1];
#pragma unroll
  for (int i = 0; i < D::QG; ++i) O.g[i * N + c] = G.v[i % QG1][i / QG1];
  O.ux[c] = uxn;
  if constexpr (DIM == 2) O.uy[c] = uyn;
  O.T[c] = Tout;
  if constexpr (is_mixed<R>()) {
    O.M[c] = M.r;
    O.M[N + c] = M.jx;
    if constexpr (DIM == 2) O.M[2 * N + c] = M.jy;
    O.M[3 * N + c] = M.e;
  }
}

// The right-edge x-face records of the tile just stepped (fx = BX) become the
// left-edge records (fx = 0) of the tile to its right, in the same shared
// memory.  Called by every thread after a barrier that follows the tile's
// phase C; the next tile's phase A writes only the halo records, and its
// barrier orders these copies before phase B.
template <typename R, int DIM, int QF1, int BX, int BY, int NT, int QG1 = 3>
__device__ __forceinline__ void hand_over_x_edge(unsigned char *smem) {
  using D = Dims<DIM, QF1, QG1>;
  using TL = Tile<DIM, BX, BY, QF1, QG1>;
  R *fp = reinterpret_cast<R *>(smem) + (size_t)TL::NH * D::NPREP;
  constexpr int rows = DIM == 2 ? BY : 1, NC = D::template nface<R>();
  for (int w = threadIdx.x; w < rows * NC; w += NT) {
    const int fy = w % rows, c = w / rows;
    fp[c * TL::NFACES + fy * (BX + 1)] = fp[c * TL::NFACES + fy * (BX + 1) + BX];
  }
}

// Phase B of a tile: every face item of the tile (see step_tile).  lim: the
// limiter, K.limiter or (the mixed path) the same value as a compile-time
// type, so that each limited slope compiles to one limiter's code.
template <typename R, int DIM, int QF1, int BX, int BY, int NT, bool ITER, bool MS, int QG1, typename LT>
__device__ __forceinline__ void faces_of_tile(const StepConst &K, const R *sp, R *fp, const unsigned char *lat,
                                              int j0, int k0, bool carry, LT lim, unsigned &noconv,
                                              unsigned &traces, unsigned &evals, unsigned &max_tr) {
  using TL = Tile<DIM, BX, BY, QF1, QG1>;
  const int tid = threadIdx.x;
  constexpr int ROWS = DIM == 2 ? BY : 1;
  const int xw = carry ? BX : BX + 1, x0 = carry ? 1 : 0;
  const int nxi = xw * ROWS, px = (nxi + 31) / 32 * 32;
  for (int w = tid; w < px + TL::NFY; w += NT) {
    int st[8];
    if (w < px) {
      if (w >= nxi) continue;
      const int fx = x0 + w % xw, fy = w / xw, f = fy * (BX + 1) + fx;
      if (j0 + fx - 1 >= K.nx || k0 + fy >= (DIM == 2 ? K.ny : 1)) continue;
      const int r = (fy + TL::OY) * TL::HX;
      st[0] = r + fx + 1; st[1] = r + fx + 2; st[2] = r + fx; st[3] = r + fx + 3;
      if constexpr (DIM == 2) {
        st[4] = r - TL::HX + fx + 1; st[5] = r - TL::HX + fx + 2;
        st[6] = r + TL::HX + fx + 1; st[7] = r + TL::HX + fx + 2;
      }
      int nt;
      bool nc;
      if constexpr (MS) {  // the face's f-lattice: the higher of its two cells'
        if (lat[st[0]] == 0 && lat[st[1]] == 0)
          nc = face_flux<R, DIM, QF1, 0, ITER, false, 3, QG1>(K, sp, CInt<TL::NH>{}, st, fp, TL::NFACES, f, nt, lim);
        else
          nc = face_flux<R, DIM, QF1, 0, ITER, false, QF1, QG1>(K, sp, CInt<TL::NH>{}, st, fp, TL::NFACES, f, nt, lim);
      } else {
        nc = face_flux<R, DIM, QF1, 0, ITER, false, QF1, QG1>(K, sp, CInt<TL::NH>{}, st, fp, TL::NFACES, f, nt, lim);
      }
      if (ITER && (fx > 0 || j0 == 0)) {
        noconv += nc; traces += nt; ++evals; max_tr = max(max_tr, (unsigned)nt);
      }
    } else if constexpr (DIM == 2) {
      const int g = w - px, fx = g % BX, fy = g / BX, f = TL::NFX + g;
      if (j0 + fx >= K.nx || k0 + fy - 1 >= K.ny) continue;
      const int x = fx + 2, H = TL::HX;
      st[0] = (fy + 1) * H + x; st[1] = (fy + 2) * H + x; st[2] = fy * H + x; st[3] = (fy + 3) * H + x;
      st[4] = (fy + 1) * H + x - 1; st[5] = (fy + 2) * H + x - 1;
      st[6] = (fy + 1) * H + x + 1; st[7] = (fy + 2) * H + x + 1;
      int nt;
      bool nc;
      if constexpr (MS) {  // the face's f-lattice: the higher of its two cells'
        if (lat[st[0]] == 0 && lat[st[1]] == 0)
          nc = face_flux<R, DIM, QF1, 1, ITER, false, 3, QG1>(K, sp, CInt<TL::NH>{}, st, fp, TL::NFACES, f, nt, lim);
        else
          nc = face_flux<R, DIM, QF1, 1, ITER, false, QF1, QG1>(K, sp, CInt<TL::NH>{}, st, fp, TL::NFACES, f, nt, lim);
      } else {
        nc = face_flux<R, DIM, QF1, 1, ITER, false, QF1, QG1>(K, sp, CInt<TL::NH>{}, st, fp, TL::NFACES, f, nt, lim);
      }
      if (ITER && (fy > 0 || k0 == 0)) {
        noconv += nc; traces += nt; ++evals; max_tr = max(max_tr, (unsigned)nt);
      }
    }
  }
}

// ---- one tile step (phases A-C) --------------------------------------------------
// The BX x BY tile whose first cell is (j0, k0); smem holds the halo and face
// records.  Every output depends only on its own stencil's arithmetic: for a
// given instantiation the result does not depend on the launch order or on
// which tile a cell falls in (different tile shapes are different machine
// code and may round differently).
// carry: the tile's left-edge x-face records (fx = 0) are already in shared
// memory, handed over by the tile on its left (hand_over_x_edge); phase B
// skips them.
template <typename R, int DIM, int QF1, int BX, int BY, int NT, bool ITER, bool MS = false, int QG1 = 3>
__device__ __forceinline__ void step_tile(const StepConst &K, const State<R> &S, const State<R> &O,
                                          Stats *stats, int j0, int k0, unsigned char *smem,
                                          bool carry = false) {
  using D = Dims<DIM, QF1, QG1>;
  using TL = Tile<DIM, BX, BY, QF1, QG1>;
  R *sp = reinterpret_cast<R *>(smem);
  R *fp = sp + (size_t)TL::NH * D::NPREP;
  unsigned char *lat = reinterpret_cast<unsigned char *>(fp + (size_t)TL::NFACES * D::template nface<R>());
  const int tid = threadIdx.x;

  // A. halo tile
  for (int h = tid; h < TL::NH; h += NT) {
    const int hx = h % TL::HX, hy = h / TL::HX;
    prep_cell<R, DIM, QF1, MS, QG1>(K, S, j0 + hx - 2, k0 + hy - TL::OY, sp, TL::NH, h, lat);
  }
  __syncthreads();

  // B. faces (a face on a tile edge is evaluated by both tiles unless it was
  // handed over; the iterated frame's counts take it from the tile on its
  // right/upper side).  Work items: the x-faces this tile computes (BX + 1 per
  // row, BX when the left edge was handed over), padded to whole warps so that
  // no warp runs both the x-face and the y-face code, then the y-faces.
  unsigned noconv = 0, traces = 0, evals = 0, max_tr = 0;
  // The mixed path, bound by latency rather than arithmetic, runs the faces
  // with the limiter fixed at compile time (one uniform branch per tile
  // instead of one per limited slope); the FP64 path, bound by its FP64
  // pipe, and the iterated frame keep one copy of the face code.
  if constexpr (is_mixed<R>() && !ITER) {
    if (K.limiter == LIM_MINMOD)
      faces_of_tile<R, DIM, QF1, BX, BY, NT, ITER, MS, QG1>(K, sp, fp, lat, j0, k0, carry, CInt<LIM_MINMOD>{},
                                                            noconv, traces, evals, max_tr);
    else
      faces_of_tile<R, DIM, QF1, BX, BY, NT, ITER, MS, QG1>(K, sp, fp, lat, j0, k0, carry, CInt<LIM_VANLEER>{},
                                                            noconv, traces, evals, max_tr);
  } else {
    faces_of_tile<R, DIM, QF1, BX, BY, NT, ITER, MS, QG1>(K, sp, fp, lat, j0, k0, carry, K.limiter, noconv,
                                                          traces, evals, max_tr);
  }
  __syncthreads();

  // C. cells
  R vmax = R(0);
  unsigned flags = 0, nhigh = 0;
  for (int c = tid; c < TL::NCELL; c += NT) {
    const int cx = c % BX, cy = c / BX;
    const int j = j0 + cx, k = k0 + cy;
    if (j >= K.nx || k >= (DIM == 2 ? K.ny : 1)) continue;
    bool low = false;
    if constexpr (MS) {
      low = lat[(cy + TL::OY) * TL::HX + cx + 2] == 0;
      nhigh += !low;
    }
    update_cell<R, DIM, QF1, BX, BY, MS, QG1>(K, S, O, fp, cx, cy, j, k, vmax, flags, low);
  }
  double cfl = (double)vmax * K.lam;
  // warp reduction of the CFL number, flags and counts, one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cfl = fmax(cfl, __shfl_xor_sync(0xffffffffu, cfl, o));
    flags |= __shfl_xor_sync(0xffffffffu, flags, o);
    if constexpr (MS) nhigh += __shfl_xor_sync(0xffffffffu, nhigh, o);
    if constexpr (ITER) {
      noconv += __shfl_xor_sync(0xffffffffu, noconv, o);
      traces += __shfl_xor_sync(0xffffffffu, traces, o);
      evals += __shfl_xor_sync(0xffffffffu, evals, o);
      max_tr = max(max_tr, __shfl_xor_sync(0xffffffffu, max_tr, o));
    }
  }
  if ((tid & 31) == 0) {
    if (cfl > 1.0) flags |= FLAG_CFL;
    if (noconv) {
      flags |= FLAG_NOCONV;
      atomicAdd(&stats->noconv, (unsigned long long)noconv);
    }
    if constexpr (ITER) {
      if (evals) {
        atomicAdd(&stats->traces, (unsigned long long)traces);
        atomicAdd(&stats->face_evals, (unsigned long long)evals);
        atomicMax(&stats->max_traces, max_tr);
      }
    }
    if constexpr (MS) {
      if (nhigh) atomicAdd(&stats->ms_high, (unsigned long long)nhigh);
    }
    if (flags) atomicOr(&stats->flags, flags);
    atomicMax(&stats->max_cfl_bits, (unsigned long long)__double_as_longlong(cfl));
  }
}

// ---- the fused step kernel: one launch = one time step of one grid --------------
template <typename R, int DIM, int QF1, int BX, int BY, int NT, int MINB = 1, bool ITER = false>
__global__ void __launch_bounds__(NT, MINB) step_kernel(const StepConst K, const State<R> S,
                                                        const State<R> O, Stats *stats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  step_tile<R, DIM, QF1, BX, BY, NT, ITER>(K, S, O, stats, blockIdx.x * BX, DIM == 2 ? blockIdx.y * BY : 0,
                                      smem_raw);
}

}  // namespace pond
