// pond_kernels.cuh -- the fused PonD step kernel and its helpers (sm_103a).
//
// One launch advances every cell by one time step of Sec. IV.A.3 of
// arXiv:2302.00310 (with the Strang-split quasi-equilibrium step of Sec. IV.B).
// A CTA owns a BX x BY tile of cells and runs three phases separated by block
// barriers:
//   A. every cell of the halo-2 tile: load phi~ (SoA, coalesced), Hermite
//      analysis in the cell frame, first QE half step, phi_bar^+ of
//      Eq. eq:Fbarplus -> shared memory;
//   B. every face touching the tile: averaged face frame (Eq. eq::AvgFrame),
//      the 8 (2D) / 4 (1D) stencil cells moved into it by the Hermite shift
//      (Sec. II.B), limited MUSCL half-step trace (Eq. eq:InterfacePop),
//      interface moments, non-co-moving equilibrium (Eq. NonComovingEq) in
//      closed form, face phi (inverse of Eq. eq:FluxTransf) -> shared memory;
//   C. every cell of the tile: face phi moved into the cell frame and
//      multiplied by v.n (Eq. fluxEq), DUGKS update (Eq. eq:FinalUpdateDUGKS),
//      new co-moving frame, second QE half step, synthesis, store.
// All linear algebra is done on Hermite coefficients (pond_hermite.cuh);
// populations are synthesised only where the limiter needs them.
#pragma once
#include <cstdint>
#include "pond_hermite.cuh"

namespace pond {

enum { BC_PERIODIC = 0, BC_ZERO_GRADIENT = 1, BC_INFLOW = 2 };
enum { LIM_VANLEER = 0, LIM_MINMOD = 1 };
enum { FLAG_NONPHYSICAL = 1u, FLAG_CFL = 2u, FLAG_NOCONV = 4u };

// Per-run constants, passed by value (kernel parameter space).
struct StepConst {
  int nx, ny;
  int bc[4];
  double inflow[4][4];  // rho, ux, uy, T
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
  int iter_max;
  int grad_k, appc, limiter, iterative;
};

template <typename R> struct State {
  R *f, *g, *ux, *uy, *T;
};

struct Stats {
  unsigned int flags;
  unsigned int pad;
  unsigned long long max_cfl_bits;  // bit pattern of a non-negative double
  unsigned long long noconv;
};

template <int DIM> struct Dims {
  static constexpr int QF = DIM == 2 ? 16 : 4;
  static constexpr int QG = DIM == 2 ? 9 : 3;
  static constexpr int NYF = DIM == 2 ? 4 : 1;
  static constexpr int NYG = DIM == 2 ? 3 : 1;
  // shared-memory record of a halo cell: f coeffs, g coeffs, ux, uy, T, sqrt T
  static constexpr int IUX = QF + QG, IUY = IUX + 1, IT = IUX + 2, IST = IUX + 3;
  static constexpr int NPREP = QF + QG + 4;
  // shared-memory record of a face: f coeffs, g coeffs, uFx, uFy, sqrt TF
  static constexpr int FUX = QF + QG, FUY = FUX + 1, FST = FUX + 2;
  static constexpr int NFACE = QF + QG + 3;
};

template <int DIM, int BX, int BY> struct Tile {
  static constexpr int HX = BX + 4, HY = DIM == 2 ? BY + 4 : 1, OY = DIM == 2 ? 2 : 0;
  static constexpr int NH = HX * HY;
  static constexpr int NFX = (BX + 1) * (DIM == 2 ? BY : 1);
  static constexpr int NFY = DIM == 2 ? BX * (BY + 1) : 0;
  static constexpr int NFACES = NFX + NFY;
  static constexpr int NCELL = BX * (DIM == 2 ? BY : 1);
  template <typename R> static constexpr size_t smem_bytes() {
    return sizeof(R) * ((size_t)NH * Dims<DIM>::NPREP + (size_t)NFACES * Dims<DIM>::NFACE);
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
template <typename R, int NYF, int NYG>
__device__ __forceinline__ void qe_scale(Blk<R, 4, NYF> &F, Blk<R, 3, NYG> &G, R qe) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < NYF; ++b)
      if (a + b == 3) F.v[a][b] *= qe;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < NYG; ++b)
      if (a + b == 1) G.v[a][b] *= qe;
}

template <typename R> __device__ __forceinline__ R qnan();
template <> __device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000LL); }
template <> __device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }

template <typename R>
__device__ __forceinline__ R limit(R x, R y, int lim) {
  const R p = x * y;
  if (lim == LIM_MINMOD) return p > R(0) ? (fabs(x) < fabs(y) ? x : y) : R(0);
  return p > R(0) ? (p + p) / (x + y) : R(0);  // Van Leer: 2xy/(x+y)
}

// ---- phase A: one halo cell -> shared memory ------------------------------
template <typename R, int DIM>
__device__ __forceinline__ void prep_cell(const StepConst &K, const State<R> &S, int j, int k, R *sp,
                                          int NH, int h) {
  using D = Dims<DIM>;
  Blk<R, 4, D::NYF> F;
  Blk<R, 3, D::NYG> G;
  R ux, uy, T;
  int sj = 0, sk = 0;
  const int side = map_cell<DIM>(K, j, k, sj, sk);
  if (side < 0) {
    const size_t N = (size_t)K.nx * (DIM == 2 ? K.ny : 1);
    const size_t c = (size_t)sk * K.nx + sj;
#pragma unroll
    for (int i = 0; i < D::QF; ++i) F.v[i % 4][i / 4] = S.f[i * N + c];
#pragma unroll
    for (int i = 0; i < D::QG; ++i) G.v[i % 3][i / 3] = S.g[i * N + c];
    ux = S.ux[c];
    uy = DIM == 2 ? S.uy[c] : R(0);
    T = S.T[c];
    ana_x(F); ana_y(F); ana_x(G); ana_y(G);
    qe_scale(F, G, R(K.qe));
    const R rho = F.v[0][0], ka = R(K.kp_a);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < D::NYF; ++b) F.v[a][b] *= ka;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < D::NYG; ++b) G.v[a][b] *= ka;
    // phi_bar^+ = kp_a phi~ + kp_b phi^eq; phi^eq = rho W (f), (C_v - D/2) T rho W (g)
    F.v[0][0] = R(K.kappa1) * rho;
    G.v[0][0] += R(K.kp_b) * R(K.gfac) * T * rho;
  } else {
    const R rho = R(K.inflow[side][0]);
    ux = R(K.inflow[side][1]);
    uy = DIM == 2 ? R(K.inflow[side][2]) : R(0);
    T = R(K.inflow[side][3]);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < D::NYF; ++b) F.v[a][b] = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < D::NYG; ++b) G.v[a][b] = R(0);
    F.v[0][0] = R(K.kappa1) * rho;
    G.v[0][0] = R(K.kappa1) * R(K.gfac) * T * rho;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < D::NYF; ++b) sp[(a + 4 * b) * NH + h] = F.v[a][b];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < D::NYG; ++b) sp[(D::QF + a + 3 * b) * NH + h] = G.v[a][b];
  sp[D::IUX * NH + h] = ux;
  sp[D::IUY * NH + h] = uy;
  sp[D::IT * NH + h] = T;
  sp[D::IST * NH + h] = sqrt(T);
}

// ---- phase B helpers --------------------------------------------------------
// phi_bar^+ of halo cell h (times kappa1) moved into the face frame and
// synthesised into populations Y[x-node][y-node].
template <typename R, int DIM, int Q>
__device__ __forceinline__ void stencil_pops(const StepConst &K, const R *sp, int NH, int h, R uFx,
                                             R uFy, R isTF, Blk<R, Q, (DIM == 2 ? Q : 1)> &Y) {
  using D = Dims<DIM>;
  constexpr int NY = DIM == 2 ? Q : 1;
  constexpr int base = Q == 4 ? 0 : D::QF;
#pragma unroll
  for (int n = 0; n < Q; ++n)
#pragma unroll
    for (int m = 0; m < NY; ++m) Y.v[n][m] = sp[(base + n + Q * m) * NH + h];
  const R a = sp[D::IST * NH + h] * isTF;
  shift_x(make_shift(a, (sp[D::IUX * NH + h] - uFx) * isTF), Y);
  if constexpr (DIM == 2) {
    shift_y(make_shift(a, (sp[D::IUY * NH + h] - uFy) * isTF), Y);
    if (K.grad_k) grad_mask(Y);
  }
  syn_x(Y);
  syn_y(Y);
}

// Limited half-step MUSCL trace of the populations of one lattice (Q nodes
// per axis) to the face (Eq. eq:InterfacePop).  st[] = halo indices of the
// stencil: 0 left, 1 right, 2 outer-left, 3 outer-right, 4/5 lower tangential
// neighbour of left/right, 6/7 upper tangential neighbour of left/right.
// With a = upwind value, b = its outer neighbour, c = the downwind value, the
// trace is a + (1/2 - |v_n| lam/2) L(a - b, c - a) for either upwind side
// (L odd and symmetric), plus the tangential term -v_t lam/2 L(a - lo, hi - a).
template <typename R, int DIM, int DIRN, int Q>
__device__ __forceinline__ void reconstruct(const StepConst &K, const R *sp, int NH, const int *st,
                                            R uFx, R uFy, R sTF, R isTF,
                                            Blk<R, Q, (DIM == 2 ? Q : 1)> &out) {
  constexpr int NY = DIM == 2 ? Q : 1;
  const R uFn = DIRN == 0 ? uFx : uFy, uFt = DIRN == 0 ? uFy : uFx;
  const R hl = R(0.5) * R(K.lam);
  bool up[Q];
  R offn[Q], offt[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const R c = R(Nodes<Q>::c(k));
    const R vn = sTF * c + uFn;
    up[k] = vn > R(0);
    offn[k] = R(0.5) - hl * fabs(vn);
    offt[k] = -hl * (sTF * c + uFt);
  }
  Blk<R, Q, NY> YL, YR, A;
  stencil_pops<R, DIM, Q>(K, sp, NH, st[0], uFx, uFy, isTF, YL);
  stencil_pops<R, DIM, Q>(K, sp, NH, st[1], uFx, uFy, isTF, YR);
  {
    Blk<R, Q, NY> Y1, Y2;
    stencil_pops<R, DIM, Q>(K, sp, NH, st[2], uFx, uFy, isTF, Y1);
    stencil_pops<R, DIM, Q>(K, sp, NH, st[3], uFx, uFy, isTF, Y2);
#pragma unroll
    for (int n = 0; n < Q; ++n)
#pragma unroll
      for (int m = 0; m < NY; ++m) {
        const int k = DIRN == 0 ? n : m;
        const R a = up[k] ? YL.v[n][m] : YR.v[n][m];
        const R b = up[k] ? Y1.v[n][m] : Y2.v[n][m];
        const R c = up[k] ? YR.v[n][m] : YL.v[n][m];
        A.v[n][m] = a;
        out.v[n][m] = a + offn[k] * limit(a - b, c - a, K.limiter);
      }
  }
  if constexpr (DIM == 2) {
    Blk<R, Q, NY> Y1, Y2, Dl;
    stencil_pops<R, DIM, Q>(K, sp, NH, st[4], uFx, uFy, isTF, Y1);
    stencil_pops<R, DIM, Q>(K, sp, NH, st[5], uFx, uFy, isTF, Y2);
#pragma unroll
    for (int n = 0; n < Q; ++n)
#pragma unroll
      for (int m = 0; m < NY; ++m) {
        const int k = DIRN == 0 ? n : m;
        Dl.v[n][m] = A.v[n][m] - (up[k] ? Y1.v[n][m] : Y2.v[n][m]);
      }
    stencil_pops<R, DIM, Q>(K, sp, NH, st[6], uFx, uFy, isTF, Y1);
    stencil_pops<R, DIM, Q>(K, sp, NH, st[7], uFx, uFy, isTF, Y2);
#pragma unroll
    for (int n = 0; n < Q; ++n)
#pragma unroll
      for (int m = 0; m < NY; ++m) {
        const int k = DIRN == 0 ? n : m, kt = DIRN == 0 ? m : n;
        const R hi = up[k] ? Y1.v[n][m] : Y2.v[n][m];
        out.v[n][m] += offt[kt] * limit(Dl.v[n][m], hi - A.v[n][m], K.limiter);
      }
  }
}

// Gaussian expectations E[He_n(s Z + mu)], n <= 3, Z ~ N(0,1), s^2 - 1 = sm1:
// the Hermite coefficients of an equilibrium seen from a foreign frame
// (Gauss-Hermite quadrature is exact to degree 2q-1, so rho G W has them).
template <typename R>
__device__ __forceinline__ void gauss_he(R mu, R sm1, R &e1, R &e2, R &e3) {
  const R mu2 = mu * mu;
  e1 = mu;
  e2 = mu2 + sm1;
  e3 = mu * (mu2 + R(3) * sm1);
}

// ---- phase B: one face --------------------------------------------------------
template <typename R, int DIM, int DIRN>
__device__ __forceinline__ void face_flux(const StepConst &K, const R *sp, int NH, const int *st,
                                          R *fp, int NFACES, int fidx) {
  using D = Dims<DIM>;
  constexpr int NYF = D::NYF, NYG = D::NYG;
  const int hL = st[0], hR = st[1];
  const R uFx = R(0.5) * (sp[D::IUX * NH + hL] + sp[D::IUX * NH + hR]);
  const R uFy = DIM == 2 ? R(0.5) * (sp[D::IUY * NH + hL] + sp[D::IUY * NH + hR]) : R(0);
  const R TF = R(0.5) * (sp[D::IT * NH + hL] + sp[D::IT * NH + hR]);
  const R sTF = sqrt(TF), isTF = R(1) / sTF;

  Blk<R, 4, NYF> Fb;
  Blk<R, 3, NYG> Gb;
  reconstruct<R, DIM, DIRN, 4>(K, sp, NH, st, uFx, uFy, sTF, isTF, Fb);
  reconstruct<R, DIM, DIRN, 3>(K, sp, NH, st, uFx, uFy, sTF, isTF, Gb);
  ana_x(Fb); ana_y(Fb); ana_x(Gb); ana_y(Gb);

  // interface moments in the face frame (all carry the factor kappa1):
  // rho, mu = (u - u_F)/sqrt(T_F), C_v rho T = T_F/2 (sum |c|^2 f - rho mu^2) + sum g
  const R rk = Fb.v[0][0], irk = R(1) / rk;
  const R mx = Fb.v[1][0] * irk;
  R my = R(0), S2 = Fb.v[2][0] + R(DIM) * rk;
  if constexpr (DIM == 2) { my = Fb.v[0][1] * irk; S2 += Fb.v[0][2]; }
  const R ek = R(0.5) * TF * (S2 - rk * (mx * mx + my * my)) + Gb.v[0][0];
  const R Tb = ek * irk * R(K.inv_cv);
  const R sm1 = Tb * isTF * isTF - R(1);

  // equilibrium (closed form of rho G_{u,T}^{lambda_F} W), weighted by kappa2/kappa1
  R ex[4], ey[4];
  ex[0] = R(1); gauss_he(mx, sm1, ex[1], ex[2], ex[3]);
  ey[0] = R(1); ey[1] = ey[2] = ey[3] = R(0);
  if constexpr (DIM == 2) gauss_he(my, sm1, ey[1], ey[2], ey[3]);
  // an interface state with rho <= 0 or T <= 0 has no equilibrium: poison the
  // face so that both adjacent cells are flagged nonphysical
  const bool phys = rk > R(0) && Tb > R(0);
  const R re = phys ? R(K.kr) * rk : qnan<R>(), ge = re * R(K.gfac) * Tb;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < NYF; ++b) {
      R e = re * ex[a] * ey[b];
      if (DIM == 2 && K.grad_k && a + b > 3) e = R(0);
      Fb.v[a][b] += e;
    }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < NYG; ++b) {
      R e = ge * ex[a] * ey[b];
      if (DIM == 2 && K.grad_k && a + b > 2) e = R(0);
      Gb.v[a][b] += e;
    }
  // Appendix C form: transport v_n^{lambda_F} phi in the face frame
  if (K.appc) {
    const R un = DIRN == 0 ? uFx : uFy;
    vmul<DIRN>(un, sTF, Fb);
    vmul<DIRN>(un, sTF, Gb);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < NYF; ++b) fp[(a + 4 * b) * NFACES + fidx] = Fb.v[a][b];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < NYG; ++b) fp[(D::QF + a + 3 * b) * NFACES + fidx] = Gb.v[a][b];
  fp[D::FUX * NFACES + fidx] = uFx;
  fp[D::FUY * NFACES + fidx] = uFy;
  fp[D::FST * NFACES + fidx] = sTF;
}

// ---- phase C: one cell --------------------------------------------------------
template <typename R, int DIM, int DIRN>
__device__ __forceinline__ void add_face(const StepConst &K, const R *fp, int NFACES, int fidx,
                                         R sgn, R ux, R uy, R sT, R isT, Blk<R, 4, Dims<DIM>::NYF> &AF,
                                         Blk<R, 3, Dims<DIM>::NYG> &AG) {
  using D = Dims<DIM>;
  Blk<R, 4, D::NYF> X;
  Blk<R, 3, D::NYG> Y;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < D::NYF; ++b) X.v[a][b] = fp[(a + 4 * b) * NFACES + fidx];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < D::NYG; ++b) Y.v[a][b] = fp[(D::QF + a + 3 * b) * NFACES + fidx];
  const R uFx = fp[D::FUX * NFACES + fidx], uFy = fp[D::FUY * NFACES + fidx];
  const R a = fp[D::FST * NFACES + fidx] * isT;
  const Shift<R> Cx = make_shift(a, (uFx - ux) * isT);
  shift_x(Cx, X); shift_x(Cx, Y);
  if constexpr (DIM == 2) {
    const Shift<R> Cy = make_shift(a, (uFy - uy) * isT);
    shift_y(Cy, X); shift_y(Cy, Y);
    if (K.grad_k) { grad_mask(X); grad_mask(Y); }
  }
  // contribution -dt/dx (v^lambda . n) G phi (Eq. fluxEq) or -dt/dx G (v^lambda_F . n phi)
  const R w = -R(K.lam) * sgn;
  if (!K.appc) {
    const R un = DIRN == 0 ? ux : uy;
    vmul<DIRN>(w * un, w * sT, X);
    vmul<DIRN>(w * un, w * sT, Y);
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < D::NYF; ++q) AF.v[p][q] += X.v[p][q];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = 0; q < D::NYG; ++q) AG.v[p][q] += Y.v[p][q];
  } else {
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < D::NYF; ++q) AF.v[p][q] += w * X.v[p][q];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = 0; q < D::NYG; ++q) AG.v[p][q] += w * Y.v[p][q];
  }
}

template <typename R, int DIM, int BX, int BY>
__device__ __forceinline__ void update_cell(const StepConst &K, const State<R> &S, const State<R> &O,
                                            const R *fp, int cx, int cy, int j, int k, double &cfl,
                                            unsigned &flags) {
  using D = Dims<DIM>;
  using TL = Tile<DIM, BX, BY>;
  const size_t N = (size_t)K.nx * (DIM == 2 ? K.ny : 1);
  const size_t c = (size_t)k * K.nx + j;
  Blk<R, 4, D::NYF> F, AF;
  Blk<R, 3, D::NYG> G, AG;
#pragma unroll
  for (int i = 0; i < D::QF; ++i) { F.v[i % 4][i / 4] = S.f[i * N + c]; AF.v[i % 4][i / 4] = R(0); }
#pragma unroll
  for (int i = 0; i < D::QG; ++i) { G.v[i % 3][i / 3] = S.g[i * N + c]; AG.v[i % 3][i / 3] = R(0); }
  const R ux = S.ux[c], uy = DIM == 2 ? S.uy[c] : R(0), T = S.T[c];
  const R sT = sqrt(T), isT = R(1) / sT;
  ana_x(F); ana_y(F); ana_x(G); ana_y(G);
  qe_scale(F, G, R(K.qe));
  const R rho = F.v[0][0];

  // fluxes through the faces, in a fixed order: x-lo, x-hi, y-lo, y-hi
  add_face<R, DIM, 0>(K, fp, TL::NFACES, cy * (BX + 1) + cx, R(-1), ux, uy, sT, isT, AF, AG);
  add_face<R, DIM, 0>(K, fp, TL::NFACES, cy * (BX + 1) + cx + 1, R(1), ux, uy, sT, isT, AF, AG);
  if constexpr (DIM == 2) {
    add_face<R, DIM, 1>(K, fp, TL::NFACES, TL::NFX + cy * BX + cx, R(-1), ux, uy, sT, isT, AF, AG);
    add_face<R, DIM, 1>(K, fp, TL::NFACES, TL::NFX + (cy + 1) * BX + cx, R(1), ux, uy, sT, isT, AF, AG);
  }
  // DUGKS update in the cell frame: a1 phi~ + a2 phi^eq - dt/dx sum F
  const R a1 = R(K.a1);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < D::NYF; ++b) F.v[a][b] = a1 * F.v[a][b] + AF.v[a][b];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < D::NYG; ++b) G.v[a][b] = a1 * G.v[a][b] + AG.v[a][b];
  F.v[0][0] += R(K.a2) * rho;
  G.v[0][0] += R(K.a2) * R(K.gfac) * T * rho;

  // new moments (Eqs. eq::ConservationLaws, eq:E) and the new co-moving frame
  const R rn = F.v[0][0], irn = R(1) / rn;
  const R mx = F.v[1][0] * irn;
  R my = R(0), S2 = F.v[2][0] + R(DIM) * rn;
  if constexpr (DIM == 2) { my = F.v[0][1] * irn; S2 += F.v[0][2]; }
  const R en = R(0.5) * T * (S2 - rn * (mx * mx + my * my)) + G.v[0][0];
  const R Tn = en * irn * R(K.inv_cv);
  R uxn = ux + sT * mx, uyn = DIM == 2 ? uy + sT * my : R(0), Tout = Tn;
  const bool ok = rn > R(0) && Tn > R(0) && isfinite(rn) && isfinite(Tn) && isfinite(uxn) &&
                  isfinite(uyn);
  if (ok) {
    const R sTn = sqrt(Tn), a = sT / sTn;
    const Shift<R> Cx = make_shift(a, -a * mx);
    shift_x(Cx, F); shift_x(Cx, G);
    if constexpr (DIM == 2) {
      const Shift<R> Cy = make_shift(a, -a * my);
      shift_y(Cy, F); shift_y(Cy, G);
      if (K.grad_k) { grad_mask(F); grad_mask(G); }
    }
    qe_scale(F, G, R(K.qe));
    const double vmax = fmax(fabs((double)uxn), fabs((double)uyn)) + (double)sTn * Nodes<4>::cmax;
    cfl = fmax(cfl, vmax * K.lam);
  } else {
    flags |= FLAG_NONPHYSICAL;
    uxn = ux; uyn = uy; Tout = T;
  }
  syn_x(F); syn_y(F); syn_x(G); syn_y(G);
#pragma unroll
  for (int i = 0; i < D::QF; ++i) O.f[i * N + c] = F.v[i % 4][i / 4];
#pragma unroll
  for (int i = 0; i < D::QG; ++i) O.g[i * N + c] = G.v[i % 3][i / 3];
  O.ux[c] = uxn;
  if constexpr (DIM == 2) O.uy[c] = uyn;
  O.T[c] = Tout;
}

// ---- the fused step kernel ------------------------------------------------------
template <typename R, int DIM, int BX, int BY, int NT>
__global__ void __launch_bounds__(NT) step_kernel(const StepConst K, const State<R> S,
                                                  const State<R> O, Stats *stats) {
  using D = Dims<DIM>;
  using TL = Tile<DIM, BX, BY>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *sp = reinterpret_cast<R *>(smem_raw);
  R *fp = sp + (size_t)TL::NH * D::NPREP;
  const int tid = threadIdx.x;
  const int j0 = blockIdx.x * BX, k0 = DIM == 2 ? blockIdx.y * BY : 0;

  // A. halo tile
  for (int h = tid; h < TL::NH; h += NT) {
    const int hx = h % TL::HX, hy = h / TL::HX;
    prep_cell<R, DIM>(K, S, j0 + hx - 2, k0 + hy - TL::OY, sp, TL::NH, h);
  }
  __syncthreads();

  // B. faces
  for (int f = tid; f < TL::NFACES; f += NT) {
    int st[8];
    if (f < TL::NFX) {
      const int fx = f % (BX + 1), fy = f / (BX + 1);
      if (j0 + fx - 1 >= K.nx || k0 + fy >= (DIM == 2 ? K.ny : 1)) continue;
      const int r = (fy + TL::OY) * TL::HX;
      st[0] = r + fx + 1; st[1] = r + fx + 2; st[2] = r + fx; st[3] = r + fx + 3;
      if constexpr (DIM == 2) {
        st[4] = r - TL::HX + fx + 1; st[5] = r - TL::HX + fx + 2;
        st[6] = r + TL::HX + fx + 1; st[7] = r + TL::HX + fx + 2;
      }
      face_flux<R, DIM, 0>(K, sp, TL::NH, st, fp, TL::NFACES, f);
    } else if constexpr (DIM == 2) {
      const int g = f - TL::NFX, fx = g % BX, fy = g / BX;
      if (j0 + fx >= K.nx || k0 + fy - 1 >= K.ny) continue;
      const int x = fx + 2, H = TL::HX;
      st[0] = (fy + 1) * H + x; st[1] = (fy + 2) * H + x; st[2] = fy * H + x; st[3] = (fy + 3) * H + x;
      st[4] = (fy + 1) * H + x - 1; st[5] = (fy + 2) * H + x - 1;
      st[6] = (fy + 1) * H + x + 1; st[7] = (fy + 2) * H + x + 1;
      face_flux<R, DIM, 1>(K, sp, TL::NH, st, fp, TL::NFACES, f);
    }
  }
  __syncthreads();

  // C. cells
  double cfl = 0.0;
  unsigned flags = 0;
  for (int c = tid; c < TL::NCELL; c += NT) {
    const int cx = c % BX, cy = c / BX;
    const int j = j0 + cx, k = k0 + cy;
    if (j >= K.nx || k >= (DIM == 2 ? K.ny : 1)) continue;
    update_cell<R, DIM, BX, BY>(K, S, O, fp, cx, cy, j, k, cfl, flags);
  }
  // warp reduction of the CFL number and flags, one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cfl = fmax(cfl, __shfl_xor_sync(0xffffffffu, cfl, o));
    flags |= __shfl_xor_sync(0xffffffffu, flags, o);
  }
  if ((tid & 31) == 0) {
    if (cfl > 1.0) flags |= FLAG_CFL;
    if (flags) atomicOr(&stats->flags, flags);
    atomicMax(&stats->max_cfl_bits, (unsigned long long)__double_as_longlong(cfl));
  }
}

}  // namespace pond
