/*
 * pond_oracle.c -- plain, slow FP64 CPU reference of one Particles-on-Demand
 * (PonD) time step, Kallikounis & Karlin, arXiv:2302.00310.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * What it computes, in the paper's order (Sec. IV.A.3 "Summary of the
 * algorithm", with the Strang-split quasi-equilibrium step of Sec. IV.B):
 *   1. quasi-equilibrium half relaxation at cell centres  (Sec. IV.B, step 1;
 *      f*, g* of Eq. eq::quasi_f)
 *   2. phi_bar^+ at cell centres                          (Eq. eq:Fbarplus)
 *   3. loop over faces: averaged face frame               (Eq. eq::AvgFrame)
 *      stencil moved into the face frame                  (Sec. II.B, Eq. GradsProjection)
 *      limited slopes + half-step MUSCL trace             (Eq. eq:InterfacePop)
 *      interface rho, rho u, C_v rho T                    (Sec. IV.A.2)
 *      non-co-moving equilibrium rho G W                  (Eq. NonComovingEq)
 *      phi at the face by inverting Eq. eq:FluxTransf
 *   4. loop over cells: face populations moved into the cell frame and summed
 *      (Eq. fluxEq), DUGKS update                         (Eq. eq:FinalUpdateDUGKS(_g))
 *   5. new moments, populations moved into the new co-moving frame
 *      (Sec. IV.A.1: the evolution frame is the co-moving one)
 *   6. quasi-equilibrium half relaxation                  (Sec. IV.B, step 3)
 *
 * The frame transformation is written from its definition (Sec. II.B): the
 * populations in the target frame are the Grad expansion (Eq. GradsProjection)
 * whose coefficients make the moments of order <= K frame invariant (Eq.
 * eq:Mcondition).  By Hermite orthogonality on the Gauss-Hermite nodes the
 * n-th coefficient equals the n-th Hermite moment of the populations measured
 * in the target frame, alpha^(n) = sum_j f_j H^(n)((v_j - u')/sqrt(T')), which
 * is the closed form of Appendix A (the tests pin this against Appendix A's
 * formulas and against the matrix form M(lambda')^-1 M(lambda) of Appendix B).
 *
 * Every floating-point value is a C double.  Loops are over cells and faces,
 * with one explicit transformation per stencil cell per face; there is no
 * tiling or fusion.  OpenMP pragmas only split independent cells/faces over
 * threads; results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXQ1 5
#define ORC_MAXQ (ORC_MAXQ1 * ORC_MAXQ1)

/* Operation counter, compiled in only with ORC_COUNT_OPS (a second build of
 * this file; the everyday build carries none of it): with orc_counting set
 * (single-threaded runs of orc_count_ops), OPS(n) adds the n floating-point
 * operations (+, -, *, /, sqrt; comparisons, fabs and fmax excluded) of the
 * statement beside it.  It covers the step's stages on cells and faces (QE,
 * phi_bar^+, faces, update, CFL), not the construction of ghost cells or the
 * multiscale switching measure. */
#ifdef ORC_COUNT_OPS
static int orc_counting = 0;
static int64_t orc_ops = 0;
#define OPS(n) \
  do { \
    if (orc_counting) orc_ops += (n); \
  } while (0)
#define ORC_UNCOUNTED(stmt) \
  do { \
    const int counting_ = orc_counting; \
    orc_counting = 0; \
    stmt; \
    orc_counting = counting_; \
  } while (0)
#else
#define OPS(n) \
  do { \
  } while (0)
#define ORC_UNCOUNTED(stmt) \
  do { \
    stmt; \
  } while (0)
#endif

enum { ORC_BC_PERIODIC = 0, ORC_BC_ZERO_GRADIENT = 1, ORC_BC_INFLOW = 2, ORC_BC_WALL = 3 };
enum { ORC_LIM_VANLEER = 0, ORC_LIM_MINMOD = 1 };
enum { ORC_FLAG_NONPHYSICAL = 1u, ORC_FLAG_NOCONV = 4u };

/* Parameters of one run.  Field order is mirrored by the Python wrapper. */
typedef struct {
  int D;              /* 1 or 2 */
  int nx, ny;         /* interior cells (ny = 1 when D = 1) */
  int qf, qg;         /* 1D node counts of the f- and g-lattices (4 and 3) */
  double gamma;       /* adiabatic exponent; C_v = 1/(gamma-1) */
  double tau;         /* tau_1 */
  double prandtl;     /* Pr = tau_1/tau_2; 1 switches the QE step off */
  double dx, dt;
  int bc[4];          /* x-lo, x-hi, y-lo, y-hi */
  double inflow[4][4];/* per side: rho, ux, uy, T of the fixed ghost state (a
                         wall: unused, its velocity ux, uy and temperature T) */
  int grad_k;         /* 0: tensor product of 1D transforms, 1: Grad a+b<=K */
  int flux_appc;      /* 0: Eq. fluxEq form, 1: Appendix C form */
  int limiter;        /* ORC_LIM_* */
  int iterative;      /* 0: averaged face frame, 1: iterated face frame */
  double iter_tol;
  int iter_max;
  /* multiscale f-lattice (Sec. II.E, Sec. IV.C): each step every cell takes
   * D1Q4 / D2Q16 where a velocity or temperature jump across it exceeds its
   * threshold, else D1Q3 / D2Q9 */
  int ms;
  double ms_theta_u;  /* on max |u_e(x + dx e_d) - u_e(x - dx e_d)| / (2 sqrt T) */
  double ms_theta_T;  /* on max |T(x + dx e_d) - T(x - dx e_d)| / (2 T) */
} orc_params;

typedef struct {
  uint32_t flags;
  int64_t noconv_faces;
  double max_cfl;
  /* iterated face frame: face evaluations, traces made over them, and the
   * most traces one evaluation made (a trace = one interface state traced in
   * a face frame) */
  int64_t face_evals;
  int64_t traces;
  int32_t max_traces;
  int64_t ms_high;  /* multiscale: cell updates made on the high-order lattice */
} orc_report;

/* ------------------------------------------------------------------ */
/* Lattices: Table I (Gauss-Hermite nodes and weights, T_L = 1).        */
/* ------------------------------------------------------------------ */
typedef struct {
  int q;                 /* nodes per axis */
  int K;                 /* highest frame-invariant order per axis */
  double c[ORC_MAXQ1];
  double w[ORC_MAXQ1];
} orc_lat1;

static void orc_lat1_make(orc_lat1 *L, int q) {
  memset(L, 0, sizeof(*L));
  L->q = q;
  if (q == 3) { /* D1Q3 */
    L->K = 2;
    L->c[0] = -sqrt(3.0); L->c[1] = 0.0; L->c[2] = sqrt(3.0);
    L->w[0] = 1.0 / 6.0;  L->w[1] = 2.0 / 3.0; L->w[2] = 1.0 / 6.0;
  } else if (q == 4) { /* D1Q4 */
    double r1 = sqrt(3.0 - sqrt(6.0)), r2 = sqrt(3.0 + sqrt(6.0));
    L->K = 3;
    L->c[0] = -r2; L->c[1] = -r1; L->c[2] = r1; L->c[3] = r2;
    L->w[0] = (3.0 - sqrt(6.0)) / 12.0; L->w[1] = (3.0 + sqrt(6.0)) / 12.0;
    L->w[2] = L->w[1]; L->w[3] = L->w[0];
  } else { /* D1Q5 */
    double r1 = sqrt(5.0 - sqrt(10.0)), r2 = sqrt(5.0 + sqrt(10.0));
    L->q = 5; L->K = 4;
    L->c[0] = -r2; L->c[1] = -r1; L->c[2] = 0.0; L->c[3] = r1; L->c[4] = r2;
    L->w[0] = (7.0 - 2.0 * sqrt(10.0)) / 60.0; L->w[1] = (7.0 + 2.0 * sqrt(10.0)) / 60.0;
    L->w[2] = 8.0 / 15.0; L->w[3] = L->w[1]; L->w[4] = L->w[0];
  }
}

/* Number of populations on the D-dimensional tensor lattice; population i
 * has node indices ix = i % q, iy = i / q (x fastest). */
static int orc_Q(const orc_lat1 *L, int D) { return D == 1 ? L->q : L->q * L->q; }
static double orc_W(const orc_lat1 *L, int D, int i) { /* Eq. eq:wi */
  OPS(D == 2);
  return D == 1 ? L->w[i] : L->w[i % L->q] * L->w[i / L->q];
}
static double orc_cx(const orc_lat1 *L, int D, int i) { return L->c[D == 1 ? i : i % L->q]; }
static double orc_cy(const orc_lat1 *L, int D, int i) { return D == 1 ? 0.0 : L->c[i / L->q]; }

/* One-dimensional Hermite polynomials of Appendix A (T_L = 1). */
static double orc_He(int n, double x) {
  OPS(n == 2 ? 2 : (n == 3 ? 4 : (n == 4 ? 7 : 0)));
  switch (n) {
  case 0: return 1.0;
  case 1: return x;
  case 2: return x * x - 1.0;
  case 3: return x * x * x - 3.0 * x;
  default: return x * x * x * x - 6.0 * x * x + 3.0;
  }
}
static double orc_fact(int n) {
  double r = 1;
  for (int k = 2; k <= n; ++k) r *= k;
  OPS(n > 1 ? n - 1 : 0);
  return r;
}

/* ------------------------------------------------------------------ */
/* Frame transformation G_{lambda}^{lambda'} (Sec. II.B).              */
/* ------------------------------------------------------------------ */
/* fin: populations in frame lambda = {u, T}; fout: populations in frame
 * lambda' = {up, Tp}.  Coefficients alpha_ab = sum_j f_j He_a(xi_xj) He_b(xi_yj),
 * xi_j = (v_j^lambda - u')/sqrt(T'), v_j^lambda = sqrt(T) c_j + u (Eq. eq:veli).
 * Synthesis f'_i = W_i sum_ab alpha_ab He_a(c_ix) He_b(c_iy) / (a! b!)
 * (Eq. GradsProjection written per axis).  grad_k = 0 keeps every a, b <= K
 * (tensor product of 1D transformations); grad_k = 1 keeps a + b <= K only
 * (the Grad projection of order K used by the paper for D2Q16, Sec. V.A). */
/* orc_transform_x: the same map between two lattices (multiscale, Sec.
 * II.E): the coefficients of order <= K per axis are measured on the source
 * lattice Ls and the Grad expansion is synthesised on the destination lattice
 * Ld, K being Ld's invariant order.  Onto a lattice of lower order it is the
 * projection (the higher coefficients are dropped).  Onto one of higher order
 * it is the lifting with the coefficients Ls does not carry set to zero in the
 * source frame (see orc_ms_switch for why that is the equilibrium completion
 * of Sec. II.E): q-node Gauss-Hermite quadrature is exact to degree 2q - 1, so
 * the source lattice measures the higher moments of its own Grad expansion
 * exactly.  In the same frame the lifting may take K = Ls's order. */
static void orc_transform_x(const orc_lat1 *Ls, const orc_lat1 *Ld, int K, int D, int grad_k,
                            const double *fin, const double u[2], double T, const double up[2],
                            double Tp, double *fout) {
  const int Qs = orc_Q(Ls, D), Qd = orc_Q(Ld, D), Kb = (D == 2) ? K : 0;
  const double sT = sqrt(T), sTp = sqrt(Tp);
  OPS(2);
  double alpha[ORC_MAXQ1][ORC_MAXQ1];
  for (int a = 0; a <= K; ++a)
    for (int b = 0; b <= Kb; ++b) {
      double s = 0.0;
      for (int j = 0; j < Qs; ++j) {
        double xix = (sT * orc_cx(Ls, D, j) + u[0] - up[0]) / sTp;
        double h = orc_He(a, xix);
        if (D == 2) {
          double xiy = (sT * orc_cy(Ls, D, j) + u[1] - up[1]) / sTp;
          h *= orc_He(b, xiy);
        }
        s += fin[j] * h;
        OPS(D == 2 ? 11 : 6);
      }
      alpha[a][b] = s;
    }
  for (int i = 0; i < Qd; ++i) {
    double s = 0.0;
    for (int a = 0; a <= K; ++a)
      for (int b = 0; b <= Kb; ++b) {
        if (grad_k && a + b > K) continue;
        double h = orc_He(a, orc_cx(Ld, D, i));
        if (D == 2) h *= orc_He(b, orc_cy(Ld, D, i));
        s += alpha[a][b] * h / (orc_fact(a) * orc_fact(b));
        OPS(D == 2 ? 5 : 4);
      }
    fout[i] = orc_W(Ld, D, i) * s;
    OPS(1);
  }
}
static void orc_transform(const orc_lat1 *L, int D, int grad_k, const double *fin,
                          const double u[2], double T, const double up[2], double Tp,
                          double *fout) {
  orc_transform_x(L, L, L->K, D, grad_k, fin, u, T, up, Tp, fout);
}

/* Equilibrium of a gas with (rho, u, T) written in a frame lambda' that need
 * not be co-moving: rho G_{u,T}^{lambda'} W (Eq. NonComovingEq). */
static void orc_equilibrium(const orc_lat1 *L, int D, int grad_k, double rho, const double u[2],
                            double T, const double up[2], double Tp, double *feq) {
  double W[ORC_MAXQ];
  const int Q = orc_Q(L, D);
  for (int i = 0; i < Q; ++i) W[i] = rho * orc_W(L, D, i);
  OPS(Q);
  orc_transform(L, D, grad_k, W, u, T, up, Tp, feq);
}

/* ------------------------------------------------------------------ */
/* Macroscopic moments (Eq. eq::ConservationLaws, Eq. eq:E).           */
/* ------------------------------------------------------------------ */
/* f, g given in the frame {uf, Tf}; returns rho, u, T.  Returns 0 if the
 * state is nonphysical (rho <= 0, T <= 0 or not finite). */
static int orc_macro(const orc_lat1 *Lf, const orc_lat1 *Lg, int D, double Cv, const double *f,
                     const double *g, const double uf[2], double Tf, double *rho, double u[2],
                     double *T) {
  const double sT = sqrt(Tf);
  OPS(1 + 15 * orc_Q(Lf, D) + orc_Q(Lg, D) + 10 + (D == 2));
  double r = 0, jx = 0, jy = 0, E2 = 0, G = 0;
  for (int i = 0; i < orc_Q(Lf, D); ++i) {
    double vx = sT * orc_cx(Lf, D, i) + uf[0];
    double vy = sT * orc_cy(Lf, D, i) + uf[1];
    r += f[i];
    jx += vx * f[i];
    jy += vy * f[i];
    E2 += 0.5 * (vx * vx + vy * vy) * f[i];
  }
  for (int i = 0; i < orc_Q(Lg, D); ++i) G += g[i];
  *rho = r;
  u[0] = jx / r;
  u[1] = (D == 2) ? jy / r : 0.0;
  /* C_v rho T = sum v^2/2 f + sum g - rho u^2/2 */
  *T = (E2 + G - 0.5 * r * (u[0] * u[0] + u[1] * u[1])) / (Cv * r);
  return (r > 0 && *T > 0 && isfinite(r) && isfinite(*T) && isfinite(u[0]) && isfinite(u[1]));
}

/* ------------------------------------------------------------------ */
/* Quasi-equilibrium half relaxation (Sec. III.A, Eq. eq::quasi_f;     */
/* Sec. IV.B, Eq. QE_relaxation), in the co-moving frame {u, T}.       */
/* ------------------------------------------------------------------ */
static void orc_qe_half(const orc_lat1 *Lf, const orc_lat1 *Lg, int D, double Cv, double dt,
                        double tau1, double tau2, double *f, double *g, const double u[2],
                        double T) {
  const int Qf = orc_Q(Lf, D), Qg = orc_Q(Lg, D);
  const double sT = sqrt(T);
  double rho = 0;
  for (int i = 0; i < Qf; ++i) rho += f[i];
  OPS(1 + Qf);
  /* Q_{abc} = sum_i e_a e_b e_c (f_i - f_i^eq), f^eq = rho W (Eq. feqPond) */
  double Qt[2][2][2] = {{{0}}};
  for (int i = 0; i < Qf; ++i) {
    double e[2] = {sT * orc_cx(Lf, D, i), sT * orc_cy(Lf, D, i)};
    double fneq = f[i] - rho * orc_W(Lf, D, i);
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b)
        for (int c = 0; c < D; ++c) Qt[a][b][c] += e[a] * e[b] * e[c] * fneq;
    OPS(4 + 4 * D * D * D);
  }
  /* varsigma_a = sum_i e_a (g_i - g_i^eq), g^eq = (C_v - D/2) T rho W (Eq. geqPond) */
  double vs[2] = {0, 0};
  for (int i = 0; i < Qg; ++i) {
    double e[2] = {sT * orc_cx(Lg, D, i), sT * orc_cy(Lg, D, i)};
    double gneq = g[i] - (Cv - 0.5 * D) * T * rho * orc_W(Lg, D, i);
    for (int a = 0; a < D; ++a) vs[a] += e[a] * gneq;
    OPS(2 + 6 + 2 * D);
  }
  const double k = 0.5 * dt * (1.0 / tau1 - 1.0 / tau2);
  OPS(5);
  /* f* - f^eq = W Q : (e e e - 3 T e I) / (6 T^3) */
  for (int i = 0; i < Qf; ++i) {
    double e[2] = {sT * orc_cx(Lf, D, i), sT * orc_cy(Lf, D, i)};
    double s = 0;
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b)
        for (int c = 0; c < D; ++c) {
          double h = e[a] * e[b] * e[c];
          if (b == c) h -= T * e[a];
          if (a == c) h -= T * e[b];
          if (a == b) h -= T * e[c];
          s += Qt[a][b][c] * h;
        }
    double dfs = orc_W(Lf, D, i) * s / (6.0 * T * T * T);
    f[i] += k * dfs;
    OPS(2 + 4 * D * D * D + 6 * D * D + 5 + 2);
  }
  /* g* - g^eq = W varsigma . e / T */
  for (int i = 0; i < Qg; ++i) {
    double e[2] = {sT * orc_cx(Lg, D, i), sT * orc_cy(Lg, D, i)};
    double s = 0;
    for (int a = 0; a < D; ++a) s += vs[a] * e[a];
    g[i] += k * orc_W(Lg, D, i) * s / T;
    OPS(2 + 2 * D + 4);
  }
}

/* ------------------------------------------------------------------ */
/* Grid with two ghost layers (Sec. IV.D: ghost-node boundaries).      */
/* ------------------------------------------------------------------ */
typedef struct {
  const orc_params *p;
  orc_lat1 Lf, Lg;
  orc_lat1 Ll; /* multiscale: the low-order f-lattice (D1Q3) */
  int *lat;    /* multiscale: 1 where a cell takes Lf, 0 where it takes Ll */
  int *xlat, *ylat; /* multiscale: lattice of each face (the higher of its cells') */
  int D, nx, ny, nxp, nyp, gy, Qf, Qg;
  double Cv;
  /* padded cell arrays, population-major: f[i * ncp + cell] */
  double *f, *g, *ux, *uy, *T;
  double *fp, *gp; /* phi_bar^+ at cell centres (frame of each cell) */
  /* faces: phi at the face in the face frame, and the face frame */
  int nfx, nfy;
  double *xff, *xfg, *xlam; /* x-faces: (nx+1)*ny */
  double *yff, *yfg, *ylam; /* y-faces: nx*(ny+1) */
} orc_grid;

static int orc_pidx(const orc_grid *G, int j, int k) { return (k + G->gy) * G->nxp + (j + 2); }
static int orc_ncp(const orc_grid *G) { return G->nxp * G->nyp; }

/* Ghost cell (j,k) -> interior source cell, or a fixed inflow state.  The
 * x-rule is resolved first, then the y-rule.  Returns the inflow side (0..3)
 * or -1 with (*sj,*sk) set. */
static int orc_ghost_map(const orc_params *p, int j, int k, int *sj, int *sk) {
  if (j < 0 || j >= p->nx) {
    int side = j < 0 ? 0 : 1;
    if (p->bc[side] == ORC_BC_INFLOW) return side;
    if (p->bc[side] == ORC_BC_PERIODIC) j = j < 0 ? j + p->nx : j - p->nx;
    else j = j < 0 ? 0 : p->nx - 1;
  }
  if (p->D == 2 && (k < 0 || k >= p->ny)) {
    int side = k < 0 ? 2 : 3;
    if (p->bc[side] == ORC_BC_INFLOW) return side;
    if (p->bc[side] == ORC_BC_PERIODIC) k = k < 0 ? k + p->ny : k - p->ny;
    else k = k < 0 ? 0 : p->ny - 1;
  }
  *sj = j; *sk = k;
  return -1;
}

static void orc_set_equilibrium_cell(orc_grid *G, int c, double rho, double ux, double uy,
                                     double T) {
  /* co-moving equilibrium (Eqs. feqPond, geqPond) and its frame */
  for (int i = 0; i < G->Qf; ++i) G->f[i * orc_ncp(G) + c] = rho * orc_W(&G->Lf, G->D, i);
  for (int i = 0; i < G->Qg; ++i)
    G->g[i * orc_ncp(G) + c] = (G->Cv - 0.5 * G->D) * T * rho * orc_W(&G->Lg, G->D, i);
  G->ux[c] = ux; G->uy[c] = uy; G->T[c] = T;
}

/* ------------------------------------------------------------------ */
/* Wall ghost cells (Sec. IV.D).                                       */
/* ------------------------------------------------------------------ */
/* Walls sit on the y sides in 2D and on the x sides in 1D, half a cell
 * beyond the last interior cell.  inflow[side] = (unused, u_w,x, u_w,y, T_w).
 * The ghost at normal distance m (m = 1, 2 layers) reflects the interior cell
 * m - 1 cells from the wall: rho_G = rho_B (zero normal gradient),
 * u_G = 2 u_w - u_B and T_G = 2 T_w - T_B (fixed values at the wall). */

/* density (sum of the f populations) and frame of interior cell (j, k); the
 * stored frame is the co-moving one, i.e. the cell's u and T */
static void orc_cell_mac(const orc_grid *G, int j, int k, double m[4]) {
  const int c = orc_pidx(G, j, k), ncp = orc_ncp(G);
  double rho = 0.0;
  for (int i = 0; i < G->Qf; ++i) rho += G->f[i * ncp + c];
  m[0] = rho; m[1] = G->ux[c]; m[2] = G->uy[c]; m[3] = G->T[c];
}

/* rho, ux, uy, T at index (j, k): an interior cell, or its reflection across
 * a wall; the tangential index follows the periodic / zero-gradient rule */
static void orc_wall_mac(const orc_grid *G, int j, int k, double m[4]) {
  const orc_params *p = G->p;
  const int D = G->D;
  if (D == 2 && (j < 0 || j >= p->nx)) {
    int side = j < 0 ? 0 : 1;
    if (p->bc[side] == ORC_BC_PERIODIC) j = j < 0 ? j + p->nx : j - p->nx;
    else j = j < 0 ? 0 : p->nx - 1;
  }
  int *n = D == 2 ? &k : &j;
  const int nmax = D == 2 ? p->ny : p->nx, lo = D == 2 ? 2 : 0;
  int side = -1;
  if (*n < 0) { side = lo; *n = -*n - 1; }
  else if (*n >= nmax) { side = lo + 1; *n = 2 * nmax - 1 - *n; }
  orc_cell_mac(G, j, k, m);
  if (side >= 0) {
    m[1] = 2.0 * p->inflow[side][1] - m[1];
    m[2] = D == 2 ? 2.0 * p->inflow[side][2] - m[2] : 0.0;
    m[3] = 2.0 * p->inflow[side][3] - m[3];
  }
}

/* The wall ghost (j, k) into padded cell c: the co-moving equilibrium of its
 * (rho_G, u_G, T_G) plus the Chapman-Enskog non-equilibrium of the paper's
 * ghost construction, P^(1) and Q^(1) for f, M_g0, M_g1, M_g2 for g, from
 * second-order centred gradients of the previous step's fields, expanded by
 * Grad's projection in the ghost frame.  Readings: the non-equilibrium moments
 * are the central ones in the co-moving ghost frame (Q^(1) without its
 * u P^(1) part, which the raw moment adds; M_g1 without M_g0 u; M_g2 the T S
 * term), and the stored variable is phi~ = phi + dt/(2 tau_1) (phi - phi^eq),
 * i.e. the non-equilibrium part scaled by 1 + dt/(2 tau_1). */
static void orc_wall_ghost(orc_grid *G, int j, int k, int c) {
  const orc_params *p = G->p;
  const int D = G->D, ncp = orc_ncp(G);
  double mG[4], a[4], b[4];
  orc_wall_mac(G, j, k, mG);
  const double rho = mG[0], T = mG[3], Cv = G->Cv;
  /* gradients: gu[d][e] = d u_e / d x_d, gT[d] = d T / d x_d */
  double gu[2][2] = {{0, 0}, {0, 0}}, gT[2] = {0, 0};
  const double h = 1.0 / (2.0 * p->dx);
  for (int d = 0; d < D; ++d) {
    if (d == 0) { orc_wall_mac(G, j + 1, k, a); orc_wall_mac(G, j - 1, k, b); }
    else { orc_wall_mac(G, j, k + 1, a); orc_wall_mac(G, j, k - 1, b); }
    gu[d][0] = (a[1] - b[1]) * h;
    gu[d][1] = (a[2] - b[2]) * h;
    gT[d] = (a[3] - b[3]) * h;
  }
  double S[2][2], div = 0.0;
  for (int d = 0; d < D; ++d) div += gu[d][d];
  for (int d = 0; d < 2; ++d)
    for (int e = 0; e < 2; ++e) S[d][e] = gu[d][e] + gu[e][d];
  const double t1 = p->tau, t2 = p->tau / p->prandtl, rT = rho * T, gf = 2.0 * Cv - D;
  double P[2][2], Q[2][2][2], M1[2], M2[2][2];
  const double M0 = -t1 * rT * gf * div / Cv;
  for (int d = 0; d < 2; ++d) {
    M1[d] = -t2 * rT * gf * gT[d];
    for (int e = 0; e < 2; ++e) {
      P[d][e] = -t1 * rT * (S[d][e] - (d == e ? div / Cv : 0.0));
      M2[d][e] = -t1 * rT * gf * T * S[d][e];
      for (int f = 0; f < 2; ++f)
        Q[d][e][f] = -t2 * rT * (gT[d] * (e == f) + gT[e] * (d == f) + gT[f] * (d == e));
    }
  }
  /* Grad expansion in the ghost frame, xi = the lattice node c_i */
  const double cf = 1.0 + p->dt / (2.0 * t1), sT = sqrt(T);
  for (int i = 0; i < G->Qf; ++i) {
    const double xi[2] = {orc_cx(&G->Lf, D, i), orc_cy(&G->Lf, D, i)};
    double s2 = 0.0, s3 = 0.0;
    for (int d = 0; d < D; ++d)
      for (int e = 0; e < D; ++e) {
        s2 += P[d][e] / T * (xi[d] * xi[e] - (d == e));
        for (int f = 0; f < D; ++f)
          s3 += Q[d][e][f] / (T * sT) *
                (xi[d] * xi[e] * xi[f] - xi[d] * (e == f) - xi[e] * (d == f) - xi[f] * (d == e));
      }
    G->f[i * ncp + c] = orc_W(&G->Lf, D, i) * (rho + cf * (s2 / 2.0 + s3 / 6.0));
  }
  for (int i = 0; i < G->Qg; ++i) {
    const double xi[2] = {orc_cx(&G->Lg, D, i), orc_cy(&G->Lg, D, i)};
    double s1 = 0.0, s2 = 0.0;
    for (int d = 0; d < D; ++d) {
      s1 += M1[d] / sT * xi[d];
      for (int e = 0; e < D; ++e) s2 += (M2[d][e] - T * M0 * (d == e)) / T * (xi[d] * xi[e] - (d == e));
    }
    G->g[i * ncp + c] = orc_W(&G->Lg, D, i) * ((Cv - 0.5 * D) * T * rho + cf * (M0 + s1 + s2 / 2.0));
  }
  G->ux[c] = mG[1]; G->uy[c] = D == 2 ? mG[2] : 0.0; G->T[c] = T;
}

/* is (j, k) a ghost across a wall? */
static int orc_is_wall_ghost(const orc_params *p, int j, int k) {
  if (p->D == 2) return (k < 0 && p->bc[2] == ORC_BC_WALL) || (k >= p->ny && p->bc[3] == ORC_BC_WALL);
  return (j < 0 && p->bc[0] == ORC_BC_WALL) || (j >= p->nx && p->bc[1] == ORC_BC_WALL);
}

static void orc_fill_ghosts(orc_grid *G) {
  const orc_params *p = G->p;
  const int ncp = orc_ncp(G);
  const int k0 = (G->D == 2) ? -2 : 0, k1 = (G->D == 2) ? G->ny + 2 : 1;
  for (int k = k0; k < k1; ++k)
    for (int j = -2; j < G->nx + 2; ++j) {
      if (j >= 0 && j < G->nx && k >= 0 && k < G->ny) continue;
      int c = orc_pidx(G, j, k), sj = 0, sk = 0;
      if (orc_is_wall_ghost(p, j, k)) {
        orc_wall_ghost(G, j, k, c);
        continue;
      }
      int side = orc_ghost_map(p, j, k, &sj, &sk);
      if (side >= 0) {
        /* (a 1D state has no u_y: the inflow's u_y slot is unused there) */
        orc_set_equilibrium_cell(G, c, p->inflow[side][0], p->inflow[side][1],
                                 G->D == 2 ? p->inflow[side][2] : 0.0, p->inflow[side][3]);
      } else {
        int s = orc_pidx(G, sj, sk);
        for (int i = 0; i < G->Qf; ++i) G->f[i * ncp + c] = G->f[i * ncp + s];
        for (int i = 0; i < G->Qg; ++i) G->g[i * ncp + c] = G->g[i * ncp + s];
        G->ux[c] = G->ux[s]; G->uy[c] = G->uy[s]; G->T[c] = G->T[s];
      }
    }
}

/* ------------------------------------------------------------------ */
/* Limited slope (Sec. IV.A.2: Van Leer / minmod).                     */
/* ------------------------------------------------------------------ */
static double orc_limit(int limiter, double sl, double sr) {
  OPS(1);
  if (sl * sr <= 0.0) return 0.0;
  if (limiter == ORC_LIM_MINMOD) return fabs(sl) < fabs(sr) ? sl : sr;
  OPS(4);
  return 2.0 * sl * sr / (sl + sr);
}

/* ------------------------------------------------------------------ */
/* One face: phi at (x_b, t_{n+1/2}) in the face frame (Sec. IV.A.2).  */
/* ------------------------------------------------------------------ */
/* Stencil of a face: cn[n], n = 0..3 along the normal (cells -1, 0 (left),
 * 1 (right), 2); ct[t][m] transverse neighbours of the left (t = 0) and right
 * (t = 1) cell, lower (m = 0) and upper (m = 1). */
typedef struct {
  int dir, cn[4], ct[2][2];
} orc_stencil;

/* The stencil's phi_bar^+ moved into the face frame {uF, TF} and the limited
 * half-step trace x' = x_b - v dt/2 of every population to the face (Eq.
 * eq:InterfacePop); the upwind cell is the left one when v_n > 0.  LF is the
 * face's f-lattice (G->Lf, or the low-order one of a multiscale face, onto
 * which the stencil's populations are projected). */
static void orc_face_trace(const orc_grid *G, const orc_stencil *S, const orc_lat1 *LF,
                           const double uF[2], double TF, double *fb, double *gb) {
  const orc_params *p = G->p;
  const int D = G->D, ncp = orc_ncp(G), dir = S->dir;
  const double dt = p->dt, dx = p->dx;
  double tn_f[4][ORC_MAXQ], tn_g[4][ORC_MAXQ], tt_f[2][2][ORC_MAXQ], tt_g[2][2][ORC_MAXQ];
  for (int n = 0; n < 4; ++n) {
    int c = S->cn[n];
    double fin[ORC_MAXQ], gin[ORC_MAXQ], uc[2] = {G->ux[c], G->uy[c]};
    for (int i = 0; i < G->Qf; ++i) fin[i] = G->fp[i * ncp + c];
    for (int i = 0; i < G->Qg; ++i) gin[i] = G->gp[i * ncp + c];
    orc_transform_x(&G->Lf, LF, LF->K, D, p->grad_k, fin, uc, G->T[c], uF, TF, tn_f[n]);
    orc_transform(&G->Lg, D, p->grad_k, gin, uc, G->T[c], uF, TF, tn_g[n]);
  }
  if (D == 2)
    for (int t = 0; t < 2; ++t)
      for (int m = 0; m < 2; ++m) {
        int c = S->ct[t][m];
        double fin[ORC_MAXQ], gin[ORC_MAXQ], uc[2] = {G->ux[c], G->uy[c]};
        for (int i = 0; i < G->Qf; ++i) fin[i] = G->fp[i * ncp + c];
        for (int i = 0; i < G->Qg; ++i) gin[i] = G->gp[i * ncp + c];
        orc_transform_x(&G->Lf, LF, LF->K, D, p->grad_k, fin, uc, G->T[c], uF, TF, tt_f[t][m]);
        orc_transform(&G->Lg, D, p->grad_k, gin, uc, G->T[c], uF, TF, tt_g[t][m]);
      }
  for (int pop = 0; pop < 2; ++pop) {
    const orc_lat1 *L = pop == 0 ? LF : &G->Lg;
    double *out = pop == 0 ? fb : gb;
    for (int i = 0; i < orc_Q(L, D); ++i) {
      double vx = sqrt(TF) * orc_cx(L, D, i) + uF[0];
      double vy = sqrt(TF) * orc_cy(L, D, i) + uF[1];
      double vn = dir == 0 ? vx : vy, vt = dir == 0 ? vy : vx;
      OPS(6);
      /* upwind: t = 0 left/lower, 1 right/upper; with v_n = 0 exactly (a
       * wall at rest puts the zero node of D1Q3 there) the mean of the two
       * one-sided traces, so that the face has no preferred side */
      double val = 0.0;
      const int t0 = vn < 0.0 ? 1 : 0, t1 = vn > 0.0 ? 0 : 1;
      for (int t = t0; t <= t1; ++t) {
        int s = 1 + t; /* stencil position of the upwind cell */
        double ps = pop == 0 ? tn_f[s][i] : tn_g[s][i];
        double pm = pop == 0 ? tn_f[s - 1][i] : tn_g[s - 1][i];
        double pp = pop == 0 ? tn_f[s + 1][i] : tn_g[s + 1][i];
        double sig_n = orc_limit(p->limiter, (ps - pm) / dx, (pp - ps) / dx);
        /* offset of the departure point from the upwind cell centre */
        double dn = (t == 0 ? 0.5 * dx : -0.5 * dx) - vn * 0.5 * dt;
        double v1 = ps + dn * sig_n;
        OPS(4 + 4 + 2);
        if (D == 2) {
          double qm = pop == 0 ? tt_f[t][0][i] : tt_g[t][0][i];
          double qp = pop == 0 ? tt_f[t][1][i] : tt_g[t][1][i];
          double sig_t = orc_limit(p->limiter, (ps - qm) / dx, (qp - ps) / dx);
          v1 += (-vt * 0.5 * dt) * sig_t;
          OPS(4 + 4);
        }
        val += t0 == t1 ? v1 : 0.5 * v1;
        OPS(t0 == t1 ? 1 : 2);
      }
      out[i] = val;
    }
  }
}

/* dir = 0: x-face between cells (j,k) and (j+1,k); dir = 1: y-face between
 * (j,k) and (j,k+1).  lam is set to the face frame {u_x, u_y, T} actually
 * used; returns 1 if the iterated frame did not converge; *ntrace receives the
 * number of interface traces made; *lat the face's f-lattice (multiscale: 1
 * for G->Lf, 0 for the low-order one; phi_f then holds its populations). */
static int orc_face(orc_grid *G, int dir, int j, int k, double *phi_f, double *phi_g,
                    double lam[3], int *ntrace, int *lat) {
  const orc_params *p = G->p;
  const int D = G->D;
  const double dt = p->dt, tau = p->tau, h = 0.5 * dt;
  OPS(1);
  orc_stencil S;
  S.dir = dir;
  for (int n = 0; n < 4; ++n)
    S.cn[n] = dir == 0 ? orc_pidx(G, j - 1 + n, k) : orc_pidx(G, j, k - 1 + n);
  for (int t = 0; t < 2; ++t)
    for (int m = 0; m < 2; ++m) {
      S.ct[t][m] = -1;
      if (D == 2)
        S.ct[t][m] = dir == 0 ? orc_pidx(G, j + t, k - 1 + 2 * m) : orc_pidx(G, j - 1 + 2 * m, k + t);
    }
  const int cL = S.cn[1], cR = S.cn[2];
  /* multiscale: the face takes the higher lattice of its two cells, so that a
   * face flux only ever moves onto a lattice of equal or lower order */
  *lat = p->ms ? (G->lat[cL] | G->lat[cR]) : 1;
  const orc_lat1 *LF = *lat ? &G->Lf : &G->Ll;
  const int QF = orc_Q(LF, D);
  /* face frame, Eq. eq::AvgFrame */
  double uF[2] = {0.5 * (G->ux[cL] + G->ux[cR]), 0.5 * (G->uy[cL] + G->uy[cR])};
  double TF = 0.5 * (G->T[cL] + G->T[cR]);
  OPS(6);
  int noconv = 0;

  double fb[ORC_MAXQ], gb[ORC_MAXQ];
  double rho = 0, ub[2] = {0, 0}, Tb = 0;
  /* iterated face frame (the predictor-corrector of the earlier scheme, Sec.
   * IV.A.3): the face frame is replaced by the interface state until the two
   * agree to iter_tol or iter_max traces were made.  An iterate whose
   * interface state is nonphysical ends the iteration and the face keeps the
   * previous (physical) iterate. */
  const int nit = p->iterative ? (p->iter_max > 0 ? p->iter_max : 1) : 1;
  int converged = 0;
  double uP[2] = {uF[0], uF[1]}, TP = TF;
  *ntrace = 0;
  for (int it = 0; it < nit; ++it) {
    orc_face_trace(G, &S, LF, uF, TF, fb, gb);
    ++*ntrace;
    /* interface macroscopic fields (rho, rho u, C_v rho T) in the face frame */
    int ok = orc_macro(LF, &G->Lg, D, G->Cv, fb, gb, uF, TF, &rho, ub, &Tb);
    if (!ok) {
      if (p->iterative && it > 0) {
        uF[0] = uP[0]; uF[1] = uP[1]; TF = TP;
        orc_face_trace(G, &S, LF, uF, TF, fb, gb);
        ++*ntrace;
        orc_macro(LF, &G->Lg, D, G->Cv, fb, gb, uF, TF, &rho, ub, &Tb);
      }
      break;
    }
    if (!p->iterative) break;
    double du = sqrt((ub[0] - uF[0]) * (ub[0] - uF[0]) + (ub[1] - uF[1]) * (ub[1] - uF[1]));
    double err = fmax(du / sqrt(TF), fabs(Tb - TF) / TF);
    OPS(8 + 4);
    if (err < p->iter_tol) { converged = 1; break; }
    if (it + 1 < nit) {
      uP[0] = uF[0]; uP[1] = uF[1]; TP = TF;
      uF[0] = ub[0]; uF[1] = (D == 2) ? ub[1] : 0.0; TF = Tb;
    }
  }
  if (p->iterative && !converged) noconv = 1;

  /* equilibrium at the face in the face frame, Eq. NonComovingEq; with a
   * converged iterated frame the face frame is the co-moving one and the
   * equilibrium is rho W (Eqs. feqPond, geqPond). */
  double feq[ORC_MAXQ], geq[ORC_MAXQ];
  if (p->iterative && converged) {
    for (int i = 0; i < QF; ++i) feq[i] = rho * orc_W(LF, D, i);
    for (int i = 0; i < G->Qg; ++i) geq[i] = (G->Cv - 0.5 * D) * Tb * rho * orc_W(&G->Lg, D, i);
    OPS(QF + 5 * G->Qg);
  } else {
    double gscale = (G->Cv - 0.5 * D) * Tb;
    orc_equilibrium(LF, D, p->grad_k, rho, ub, Tb, uF, TF, feq);
    orc_equilibrium(&G->Lg, D, p->grad_k, rho * gscale, ub, Tb, uF, TF, geq);
    OPS(3 + 1);
  }
  /* invert Eq. eq:FluxTransf: phi_bar = phi - (h/2) (phi^eq - phi)/tau, h = dt/2 */
  const double r = h / (2.0 * tau);
  for (int i = 0; i < QF; ++i) phi_f[i] = (fb[i] + r * feq[i]) / (1.0 + r);
  for (int i = 0; i < G->Qg; ++i) phi_g[i] = (gb[i] + r * geq[i]) / (1.0 + r);
  OPS(2 + 4 * (QF + G->Qg));
  lam[0] = uF[0]; lam[1] = uF[1]; lam[2] = TF;
  return noconv;
}

/* ------------------------------------------------------------------ */
/* Multiscale lattice switching (Sec. II.E, Sec. IV.C).                */
/* ------------------------------------------------------------------ */
/* Jumps of u and T across interior cell (j, k), from the padded fields
 * (ghosts filled): s_u = max_{d,e} |u_e(+d) - u_e(-d)| / (2 sqrt T),
 * s_T = max_d |T(+d) - T(-d)| / (2 T), centred over the two neighbours (in
 * 1D u_x only: an inflow ghost's u_y is not part of the 1D state). */
static void orc_ms_measure(const orc_grid *G, int j, int k, double *su, double *sT) {
  const int c = orc_pidx(G, j, k);
  double gu = 0.0, gT = 0.0;
  for (int d = 0; d < G->D; ++d) {
    const int cp = orc_pidx(G, j + (d == 0), k + (d == 1));
    const int cm = orc_pidx(G, j - (d == 0), k - (d == 1));
    gu = fmax(gu, fabs(G->ux[cp] - G->ux[cm]));
    if (G->D == 2) gu = fmax(gu, fabs(G->uy[cp] - G->uy[cm]));
    gT = fmax(gT, fabs(G->T[cp] - G->T[cm]));
  }
  *su = 0.5 * gu / sqrt(G->T[c]);
  *sT = 0.5 * gT / G->T[c];
}

/* The switch at the start of a step.  Every interior cell takes the high
 * lattice where s_u > theta_u or s_T > theta_T, else the low one.  A cell's
 * populations are always stored on the high lattice: a low cell's as the
 * high-lattice populations with its own Hermite coefficients of order <= 2
 * per axis (its frame being co-moving) and none above.  That storage is the
 * lifting of Sec. II.E: the moments the low lattice lacks are set to their
 * equilibrium values, and in the cell's co-moving frame every Hermite
 * coefficient of order 3 along an axis of a Maxwellian centred on the cell's
 * velocity is zero (odd central moments of a Gaussian).  A cell that turns
 * low is projected: its coefficients of order 3 are dropped. */
static void orc_ms_switch(orc_grid *G) {
  const orc_params *p = G->p;
  const int ncp = orc_ncp(G), D = G->D;
  orc_fill_ghosts(G);
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < G->ny; ++k)
    for (int j = 0; j < G->nx; ++j) {
      const int c = orc_pidx(G, j, k);
      double su, sT;
      orc_ms_measure(G, j, k, &su, &sT);
      G->lat[c] = (su > p->ms_theta_u || sT > p->ms_theta_T) ? 1 : 0;
      if (G->lat[c]) continue;
      double f[ORC_MAXQ], fo[ORC_MAXQ], u[2] = {G->ux[c], G->uy[c]};
      for (int i = 0; i < G->Qf; ++i) f[i] = G->f[i * ncp + c];
      orc_transform_x(&G->Lf, &G->Lf, G->Ll.K, D, p->grad_k, f, u, G->T[c], u, G->T[c], fo);
      for (int i = 0; i < G->Qf; ++i) G->f[i * ncp + c] = fo[i];
    }
}

/* Lattices of the ghost cells: that of their source cell; an inflow ghost
 * (a co-moving equilibrium, the same on both lattices) the low one.  A wall
 * ghost's source is the interior cell it reflects (Sec. IV.D), and a low wall
 * ghost is projected like a low interior cell: its Chapman-Enskog content of
 * order 3 along an axis is dropped in its co-moving frame. */
static void orc_ms_ghost_lattices(orc_grid *G) {
  const orc_params *p = G->p;
  const int D = G->D, ncp = orc_ncp(G);
  const int k0 = (D == 2) ? -2 : 0, k1 = (D == 2) ? G->ny + 2 : 1;
  for (int k = k0; k < k1; ++k)
    for (int j = -2; j < G->nx + 2; ++j) {
      if (j >= 0 && j < G->nx && k >= 0 && k < G->ny) continue;
      const int c = orc_pidx(G, j, k);
      if (orc_is_wall_ghost(p, j, k)) {
        int sj = j, sk = k;
        if (D == 2 && (sj < 0 || sj >= p->nx)) {
          if (p->bc[sj < 0 ? 0 : 1] == ORC_BC_PERIODIC) sj = sj < 0 ? sj + p->nx : sj - p->nx;
          else sj = sj < 0 ? 0 : p->nx - 1;
        }
        int *n = D == 2 ? &sk : &sj;
        const int nmax = D == 2 ? p->ny : p->nx;
        *n = *n < 0 ? -*n - 1 : 2 * nmax - 1 - *n;
        G->lat[c] = G->lat[orc_pidx(G, sj, sk)];
        if (!G->lat[c]) {
          double f[ORC_MAXQ], fo[ORC_MAXQ], u[2] = {G->ux[c], G->uy[c]};
          for (int i = 0; i < G->Qf; ++i) f[i] = G->f[i * ncp + c];
          orc_transform_x(&G->Lf, &G->Lf, G->Ll.K, D, p->grad_k, f, u, G->T[c], u, G->T[c], fo);
          for (int i = 0; i < G->Qf; ++i) G->f[i * ncp + c] = fo[i];
        }
        continue;
      }
      int sj = 0, sk = 0;
      const int side = orc_ghost_map(p, j, k, &sj, &sk);
      G->lat[c] = side >= 0 ? 0 : G->lat[orc_pidx(G, sj, sk)];
    }
}

/* ------------------------------------------------------------------ */
/* One time step.                                                      */
/* ------------------------------------------------------------------ */
static int orc_step_once(orc_grid *G, orc_report *rep) {
  const orc_params *p = G->p;
  const int D = G->D, ncp = orc_ncp(G), Qf = G->Qf, Qg = G->Qg;
  const double dt = p->dt, dx = p->dx, tau = p->tau;
  const double tau2 = p->tau / p->prandtl;
  const int qe = p->prandtl != 1.0;
  uint32_t flags = 0;
  int64_t noconv = 0, traces = 0, evals = 0, ms_high = 0;
  int max_tr = 0;

  /* 0. multiscale: each cell's lattice for this step, from its current fields */
  if (p->ms) ORC_UNCOUNTED(orc_ms_switch(G)); /* the switching is not counted */

  /* 1. quasi-equilibrium half relaxation in the cell centres */
  if (qe) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < G->ny; ++k)
      for (int j = 0; j < G->nx; ++j) {
        int c = orc_pidx(G, j, k);
        double f[ORC_MAXQ], g[ORC_MAXQ], u[2] = {G->ux[c], G->uy[c]};
        for (int i = 0; i < Qf; ++i) f[i] = G->f[i * ncp + c];
        for (int i = 0; i < Qg; ++i) g[i] = G->g[i * ncp + c];
        orc_qe_half(&G->Lf, &G->Lg, D, G->Cv, dt, tau, tau2, f, g, u, G->T[c]);
        for (int i = 0; i < Qf; ++i) G->f[i * ncp + c] = f[i];
        for (int i = 0; i < Qg; ++i) G->g[i * ncp + c] = g[i];
      }
  }
  ORC_UNCOUNTED(orc_fill_ghosts(G)); /* ghost construction is not counted */
  if (p->ms) orc_ms_ghost_lattices(G);

  /* 2. phi_bar^+ in every cell (ghosts included), Eq. eq:Fbarplus, from the
   * stored variable of Eq. eq:variableTransform; the cell is in its
   * co-moving frame, so phi^eq is rho W (and (C_v - D/2) T rho W for g). */
#pragma omp parallel for schedule(static)
  for (int c = 0; c < ncp; ++c) {
    double rho = 0;
    for (int i = 0; i < Qf; ++i) rho += G->f[i * ncp + c];
    OPS(Qf + 4);
    for (int pop = 0; pop < 2; ++pop) {
      const orc_lat1 *L = pop == 0 ? &G->Lf : &G->Lg;
      const double *st = pop == 0 ? G->f : G->g;
      double *out = pop == 0 ? G->fp : G->gp;
      const double scale = pop == 0 ? rho : (G->Cv - 0.5 * D) * G->T[c] * rho;
      for (int i = 0; i < orc_Q(L, D); ++i) {
        double eq = scale * orc_W(L, D, i);
        /* phi from phi~ = phi - dt/(2 tau) (phi^eq - phi) */
        double ph = (st[i * ncp + c] + dt / (2.0 * tau) * eq) / (1.0 + dt / (2.0 * tau));
        /* phi_bar^+ = phi + (dt/4) (phi^eq - phi)/tau */
        out[i * ncp + c] = ph + 0.25 * dt * (eq - ph) / tau;
        OPS(1 + 8 + 5);
      }
    }
  }

  /* 3. fluxes: loop over faces */
#pragma omp parallel for collapse(2) schedule(static) reduction(+ : noconv, traces, evals) \
    reduction(max : max_tr)
  for (int k = 0; k < G->ny; ++k)
    for (int j = -1; j < G->nx; ++j) {
      int fi = k * (G->nx + 1) + (j + 1), nt = 0;
      noconv += orc_face(G, 0, j, k, G->xff + (size_t)fi * Qf, G->xfg + (size_t)fi * Qg,
                         G->xlam + 3 * (size_t)fi, &nt, G->xlat + fi);
      traces += nt;
      evals += 1;
      if (nt > max_tr) max_tr = nt;
    }
  if (D == 2) {
#pragma omp parallel for collapse(2) schedule(static) reduction(+ : noconv, traces, evals) \
    reduction(max : max_tr)
    for (int k = -1; k < G->ny; ++k)
      for (int j = 0; j < G->nx; ++j) {
        int fi = (k + 1) * G->nx + j, nt = 0;
        noconv += orc_face(G, 1, j, k, G->yff + (size_t)fi * Qf, G->yfg + (size_t)fi * Qg,
                           G->ylam + 3 * (size_t)fi, &nt, G->ylat + fi);
        traces += nt;
        evals += 1;
        if (nt > max_tr) max_tr = nt;
      }
  }

  /* 4.-5. loop over cells: flux in the cell frame (Eq. fluxEq), DUGKS update
   * (Eqs. eq:FinalUpdateDUGKS, eq:FinalUpdateDUGKS_g), new co-moving frame */
  const double a1 = (2.0 * tau - dt) / (2.0 * tau + dt), a2 = 2.0 * dt / (2.0 * tau + dt);
  OPS(9);
  double maxcfl = 0.0;
#pragma omp parallel for collapse(2) schedule(static) reduction(| : flags) reduction(max : maxcfl) \
    reduction(+ : ms_high)
  for (int k = 0; k < G->ny; ++k)
    for (int j = 0; j < G->nx; ++j) {
      int c = orc_pidx(G, j, k);
      double uc[2] = {G->ux[c], G->uy[c]}, Tc = G->T[c], sT = sqrt(Tc);
      OPS(1);
      double Ff[ORC_MAXQ] = {0}, Fg[ORC_MAXQ] = {0};
      /* the cell's f-lattice and its populations on it (a multiscale low cell:
       * from its high-lattice storage, an exact change of nodes) */
      const int low = p->ms && !G->lat[c];
      const orc_lat1 *Lc = low ? &G->Ll : &G->Lf;
      const int Qc = orc_Q(Lc, D);
      double fc[ORC_MAXQ];
      if (low) {
        double fs[ORC_MAXQ];
        for (int i = 0; i < Qf; ++i) fs[i] = G->f[i * ncp + c];
        orc_transform_x(&G->Lf, Lc, Lc->K, D, p->grad_k, fs, uc, Tc, uc, Tc, fc);
      } else {
        for (int i = 0; i < Qf; ++i) fc[i] = G->f[i * ncp + c];
      }
      ms_high += p->ms && !low;
      /* faces: (normal direction, face index, outward sign) */
      int nf = D == 2 ? 4 : 2;
      for (int face = 0; face < nf; ++face) {
        int dir = face / 2, sgn = (face % 2) ? +1 : -1;
        const double *pf, *pg, *lam;
        int flat;
        if (dir == 0) {
          int fi = k * (G->nx + 1) + (sgn > 0 ? j + 1 : j);
          pf = G->xff + (size_t)fi * Qf; pg = G->xfg + (size_t)fi * Qg; lam = G->xlam + 3 * (size_t)fi;
          flat = G->xlat[fi];
        } else {
          int fi = (sgn > 0 ? k + 1 : k) * G->nx + j;
          pf = G->yff + (size_t)fi * Qf; pg = G->yfg + (size_t)fi * Qg; lam = G->ylam + 3 * (size_t)fi;
          flat = G->ylat[fi];
        }
        double uF[2] = {lam[0], lam[1]}, TF = lam[2];
        for (int pop = 0; pop < 2; ++pop) {
          /* LS: the face's lattice, L: the cell's (multiscale: a high face
           * flux entering a low cell is projected onto it) */
          const orc_lat1 *LS = pop == 0 ? ((p->ms && !flat) ? &G->Ll : &G->Lf) : &G->Lg;
          const orc_lat1 *L = pop == 0 ? Lc : &G->Lg;
          const double *src = pop == 0 ? pf : pg;
          double *acc = pop == 0 ? Ff : Fg;
          const int Q = orc_Q(L, D), QS = orc_Q(LS, D);
          double tr[ORC_MAXQ];
          if (!p->flux_appc) {
            /* Eq. fluxEq: (v_i^lambda . n) G_{lambda_F}^{lambda} phi */
            orc_transform_x(LS, L, L->K, D, p->grad_k, src, uF, TF, uc, Tc, tr);
            for (int i = 0; i < Q; ++i) {
              double vn = dir == 0 ? sT * orc_cx(L, D, i) + uc[0] : sT * orc_cy(L, D, i) + uc[1];
              acc[i] += sgn * vn * tr[i];
            }
            OPS(5 * Q);
          } else {
            /* Appendix C: G_{lambda_F}^{lambda} (v^{lambda_F} . n phi) */
            double fl[ORC_MAXQ];
            for (int i = 0; i < QS; ++i) {
              double vn = dir == 0 ? sqrt(TF) * orc_cx(LS, D, i) + uF[0]
                                   : sqrt(TF) * orc_cy(LS, D, i) + uF[1];
              fl[i] = vn * src[i];
            }
            orc_transform_x(LS, L, L->K, D, p->grad_k, fl, uF, TF, uc, Tc, tr);
            for (int i = 0; i < Q; ++i) acc[i] += sgn * tr[i];
            OPS(4 * QS + 2 * Q);
          }
        }
      }
      double rho = 0;
      for (int i = 0; i < Qc; ++i) rho += fc[i];
      double f[ORC_MAXQ], g[ORC_MAXQ];
      /* V_j = dx^D, face area dx^(D-1): dt/V * area = dt/dx */
      for (int i = 0; i < Qc; ++i) f[i] = a1 * fc[i] + a2 * rho * orc_W(Lc, D, i) - dt / dx * Ff[i];
      OPS(Qc + 7 * Qc + 11 * Qg);
      for (int i = 0; i < Qg; ++i)
        g[i] = a1 * G->g[i * ncp + c] + a2 * (G->Cv - 0.5 * D) * Tc * rho * orc_W(&G->Lg, D, i) -
               dt / dx * Fg[i];
      /* new moments and the new co-moving frame */
      double rn, un[2], Tn;
      if (!orc_macro(Lc, &G->Lg, D, G->Cv, f, g, uc, Tc, &rn, un, &Tn)) {
        flags |= ORC_FLAG_NONPHYSICAL;
        if (low) {
          double fs[ORC_MAXQ];
          orc_transform_x(Lc, &G->Lf, Lc->K, D, p->grad_k, f, uc, Tc, uc, Tc, fs);
          for (int i = 0; i < Qf; ++i) G->f[i * ncp + c] = fs[i];
        } else {
          for (int i = 0; i < Qf; ++i) G->f[i * ncp + c] = f[i];
        }
        for (int i = 0; i < Qg; ++i) G->g[i * ncp + c] = g[i];
        continue;
      }
      double fn[ORC_MAXQ], gn[ORC_MAXQ];
      orc_transform(Lc, D, p->grad_k, f, uc, Tc, un, Tn, fn);
      orc_transform(&G->Lg, D, p->grad_k, g, uc, Tc, un, Tn, gn);
      /* 6. second quasi-equilibrium half relaxation, in the new frame, on the
       * cell's own f-lattice (a multiscale low cell: its third-order content
       * is what D2Q9 / D1Q3 resolves; the first half acts on the lifted
       * storage, whose coefficients of order 3 along an axis are zero) */
      if (qe) orc_qe_half(Lc, &G->Lg, D, G->Cv, dt, tau, tau2, fn, gn, un, Tn);
      if (low) { /* back to the high-lattice storage (lifting, in the new frame) */
        double fs[ORC_MAXQ];
        orc_transform_x(Lc, &G->Lf, Lc->K, D, p->grad_k, fn, un, Tn, un, Tn, fs);
        for (int i = 0; i < Qf; ++i) fn[i] = fs[i];
      }
      for (int i = 0; i < Qf; ++i) G->f[i * ncp + c] = fn[i];
      for (int i = 0; i < Qg; ++i) G->g[i * ncp + c] = gn[i];
      G->ux[c] = un[0]; G->uy[c] = D == 2 ? un[1] : 0.0; G->T[c] = Tn;
      /* CFL = max |v_i alpha| dt/dx (Sec. V) */
      double cmax = Lc->c[Lc->q - 1];
      double vmax = fmax(fabs(un[0]), fabs(D == 2 ? un[1] : 0.0)) + sqrt(Tn) * cmax;
      double cfl = vmax * dt / dx;
      OPS(5);
      if (cfl > maxcfl) maxcfl = cfl;
    }
  /* an iterated face frame that reached iter_max unconverged is reported as
   * a sticky flag beside the count of such face evaluations */
  if (noconv) flags |= ORC_FLAG_NOCONV;
  rep->flags |= flags;
  rep->noconv_faces += noconv;
  if (p->iterative) {
    rep->face_evals += evals;
    rep->traces += traces;
    if (max_tr > rep->max_traces) rep->max_traces = max_tr;
  }
  if (maxcfl > rep->max_cfl) rep->max_cfl = maxcfl;
  rep->ms_high += ms_high;
  return 0;
}

static int orc_grid_alloc(orc_grid *G, const orc_params *p) {
  memset(G, 0, sizeof(*G));
  G->p = p;
  G->D = p->D;
  orc_lat1_make(&G->Lf, p->qf);
  orc_lat1_make(&G->Lg, p->qg);
  orc_lat1_make(&G->Ll, 3);
  G->nx = p->nx; G->ny = p->D == 2 ? p->ny : 1;
  G->nxp = G->nx + 4; G->nyp = p->D == 2 ? G->ny + 4 : 1; G->gy = p->D == 2 ? 2 : 0;
  G->Qf = orc_Q(&G->Lf, G->D); G->Qg = orc_Q(&G->Lg, G->D);
  G->Cv = 1.0 / (p->gamma - 1.0);
  size_t ncp = (size_t)orc_ncp(G);
  G->f = calloc(ncp * G->Qf, sizeof(double)); G->g = calloc(ncp * G->Qg, sizeof(double));
  G->fp = calloc(ncp * G->Qf, sizeof(double)); G->gp = calloc(ncp * G->Qg, sizeof(double));
  G->ux = calloc(ncp, sizeof(double)); G->uy = calloc(ncp, sizeof(double));
  G->T = calloc(ncp, sizeof(double));
  size_t nfx = (size_t)(G->nx + 1) * G->ny, nfy = p->D == 2 ? (size_t)G->nx * (G->ny + 1) : 1;
  G->xff = calloc(nfx * G->Qf, sizeof(double)); G->xfg = calloc(nfx * G->Qg, sizeof(double));
  G->xlam = calloc(nfx * 3, sizeof(double));
  G->yff = calloc(nfy * G->Qf, sizeof(double)); G->yfg = calloc(nfy * G->Qg, sizeof(double));
  G->ylam = calloc(nfy * 3, sizeof(double));
  G->lat = calloc(ncp, sizeof(int));
  G->xlat = calloc(nfx, sizeof(int)); G->ylat = calloc(nfy, sizeof(int));
  return G->f && G->g && G->fp && G->gp && G->ux && G->uy && G->T && G->xff && G->xfg &&
         G->xlam && G->yff && G->yfg && G->ylam && G->lat && G->xlat && G->ylat;
}

static void orc_grid_free(orc_grid *G) {
  free(G->f); free(G->g); free(G->fp); free(G->gp); free(G->ux); free(G->uy); free(G->T);
  free(G->xff); free(G->xfg); free(G->xlam); free(G->yff); free(G->yfg); free(G->ylam);
  free(G->lat); free(G->xlat); free(G->ylat);
}

static int orc_check(const orc_params *p) {
  if (!p || (p->D != 1 && p->D != 2)) return 0;
  if (p->nx < 2 || (p->D == 2 && p->ny < 2)) return 0;
  if (!(p->qf == 3 || p->qf == 4 || p->qf == 5) || !(p->qg == 3 || p->qg == 4 || p->qg == 5))
    return 0;
  if (!(p->tau > 0) || !(p->dt > 0) || !(p->dx > 0) || !(p->prandtl > 0) || !(p->gamma > 1))
    return 0;
  /* walls: on the y sides in 2D (x sides periodic or zero-gradient), on the x
   * sides in 1D, with at least three cells across */
  for (int s = 0; s < 4; ++s) {
    if (p->bc[s] < ORC_BC_PERIODIC || p->bc[s] > ORC_BC_WALL) return 0;
    if (p->bc[s] != ORC_BC_WALL) continue;
    if (p->D == 2 && (s < 2 || p->ny < 3 || p->bc[0] == ORC_BC_INFLOW || p->bc[1] == ORC_BC_INFLOW))
      return 0;
    if (p->D == 1 && (s > 1 || p->nx < 3)) return 0;
  }
  /* multiscale: D1Q3/D1Q4 (D2Q9/D2Q16) f-lattices, averaged face frame */
  if (p->ms) {
    if (p->qf != 4 || p->qg != 3 || p->iterative) return 0;
  }
  return 1;
}

/* ================================================================== */
/* Exported entry points (called through ctypes by the test-suite).    */
/* Array layouts: populations [i][ny][nx] with i = iy*q + ix, fields    */
/* [ny][nx]; all FP64, host memory, caller-owned.                       */
/* ================================================================== */

/* Lattice nodes/weights of Table I. */
int orc_lattice(int q, double *c, double *w) {
  orc_lat1 L;
  orc_lat1_make(&L, q);
  for (int i = 0; i < L.q; ++i) { c[i] = L.c[i]; w[i] = L.w[i]; }
  return L.K;
}

/* Frame transformation of one population vector on the q-node lattice in D
 * dimensions: fin in {u, T} -> fout in {up, Tp}. */
void orc_transform_pub(int q, int D, int grad_k, const double *fin, const double *u, double T,
                       const double *up, double Tp, double *fout) {
  orc_lat1 L;
  orc_lat1_make(&L, q);
  double uu[2] = {u[0], D == 2 ? u[1] : 0.0}, uup[2] = {up[0], D == 2 ? up[1] : 0.0};
  orc_transform(&L, D, grad_k, fin, uu, T, uup, Tp, fout);
}

/* The frame transformation between lattices (multiscale lifting or
 * projection, Sec. II.E): fin on the qs-node lattice in {u, T} -> fout on the
 * qd-node lattice in {up, Tp}, coefficients of order <= K per axis. */
void orc_transform_x_pub(int qs, int qd, int K, int D, int grad_k, const double *fin,
                         const double *u, double T, const double *up, double Tp, double *fout) {
  orc_lat1 Ls, Ld;
  orc_lat1_make(&Ls, qs);
  orc_lat1_make(&Ld, qd);
  double uu[2] = {u[0], D == 2 ? u[1] : 0.0}, uup[2] = {up[0], D == 2 ? up[1] : 0.0};
  orc_transform_x(&Ls, &Ld, K, D, grad_k, fin, uu, T, uup, Tp, fout);
}

/* Equilibrium rho G_{u,T}^{up,Tp} W (Eq. NonComovingEq). */
void orc_equilibrium_pub(int q, int D, int grad_k, double rho, const double *u, double T,
                         const double *up, double Tp, double *feq) {
  orc_lat1 L;
  orc_lat1_make(&L, q);
  double uu[2] = {u[0], D == 2 ? u[1] : 0.0}, uup[2] = {up[0], D == 2 ? up[1] : 0.0};
  orc_equilibrium(&L, D, grad_k, rho, uu, T, uup, Tp, feq);
}

/* One quasi-equilibrium half relaxation of a single cell, in place. */
void orc_qe_half_pub(int qf, int qg, int D, double gamma, double dt, double tau1, double tau2,
                     double *f, double *g, const double *u, double T) {
  orc_lat1 Lf, Lg;
  orc_lat1_make(&Lf, qf);
  orc_lat1_make(&Lg, qg);
  double uu[2] = {u[0], D == 2 ? u[1] : 0.0};
  orc_qe_half(&Lf, &Lg, D, 1.0 / (gamma - 1.0), dt, tau1, tau2, f, g, uu, T);
}

/* Macroscopic rho, u, T of a single cell whose populations are given in the
 * frame {uf, Tf}.  Returns 1 if physical. */
int orc_macro_pub(int qf, int qg, int D, double gamma, const double *f, const double *g,
                  const double *uf, double Tf, double *out /* rho, ux, uy, T */) {
  orc_lat1 Lf, Lg;
  orc_lat1_make(&Lf, qf);
  orc_lat1_make(&Lg, qg);
  double uu[2] = {uf[0], D == 2 ? uf[1] : 0.0}, u[2], rho, T;
  int ok = orc_macro(&Lf, &Lg, D, 1.0 / (gamma - 1.0), f, g, uu, Tf, &rho, u, &T);
  out[0] = rho; out[1] = u[0]; out[2] = u[1]; out[3] = T;
  return ok;
}

/* Co-moving equilibrium initial state from primitive fields. */
int orc_init(const orc_params *p, const double *rho, const double *ux, const double *uy,
             const double *T, double *f, double *g, double *gux, double *guy, double *gT) {
  if (!orc_check(p)) return 1;
  orc_lat1 Lf, Lg;
  orc_lat1_make(&Lf, p->qf);
  orc_lat1_make(&Lg, p->qg);
  const int D = p->D, ny = D == 2 ? p->ny : 1;
  const size_t n = (size_t)p->nx * ny;
  const double Cv = 1.0 / (p->gamma - 1.0);
  for (size_t c = 0; c < n; ++c) {
    for (int i = 0; i < orc_Q(&Lf, D); ++i) f[i * n + c] = rho[c] * orc_W(&Lf, D, i);
    for (int i = 0; i < orc_Q(&Lg, D); ++i)
      g[i * n + c] = (Cv - 0.5 * D) * T[c] * rho[c] * orc_W(&Lg, D, i);
    gux[c] = ux[c]; guy[c] = D == 2 ? uy[c] : 0.0; gT[c] = T[c];
  }
  return 0;
}

/* Advance the state (f, g, gauge) by nsteps steps, in place. */
int orc_run(const orc_params *p, double *f, double *g, double *ux, double *uy, double *T,
            int64_t nsteps, orc_report *rep) {
  if (!orc_check(p)) return 1;
  orc_grid G;
  if (!orc_grid_alloc(&G, p)) { orc_grid_free(&G); return 2; }
  const int ncp = orc_ncp(&G);
  const size_t n = (size_t)G.nx * G.ny;
  memset(rep, 0, sizeof(*rep));
  for (int k = 0; k < G.ny; ++k)
    for (int j = 0; j < G.nx; ++j) {
      size_t s = (size_t)k * G.nx + j;
      int c = orc_pidx(&G, j, k);
      for (int i = 0; i < G.Qf; ++i) G.f[i * ncp + c] = f[i * n + s];
      for (int i = 0; i < G.Qg; ++i) G.g[i * ncp + c] = g[i * n + s];
      G.ux[c] = ux[s]; G.uy[c] = p->D == 2 ? uy[s] : 0.0; G.T[c] = T[s];
    }
  for (int64_t s = 0; s < nsteps; ++s) orc_step_once(&G, rep);
  for (int k = 0; k < G.ny; ++k)
    for (int j = 0; j < G.nx; ++j) {
      size_t s = (size_t)k * G.nx + j;
      int c = orc_pidx(&G, j, k);
      for (int i = 0; i < G.Qf; ++i) f[i * n + s] = G.f[i * ncp + c];
      for (int i = 0; i < G.Qg; ++i) g[i * n + s] = G.g[i * ncp + c];
      ux[s] = G.ux[c]; if (p->D == 2) uy[s] = G.uy[c]; T[s] = G.T[c];
    }
  orc_grid_free(&G);
  return 0;
}

/* The ghost cell (j, k) of the padded grid (two layers beyond the interior)
 * built from the interior state (f, g, ux, uy, T) by the run's boundary
 * rules: its populations fout[Qf], gout[Qg] and frame (ux, uy, T) in frame[3].
 * Returns 1 for invalid parameters, 2 on allocation failure, 3 if (j, k) is
 * not a ghost of the padded grid. */
int orc_ghost_pub(const orc_params *p, const double *f, const double *g, const double *ux,
                  const double *uy, const double *T, int j, int k, double *fout, double *gout,
                  double *frame) {
  if (!orc_check(p)) return 1;
  const int ny = p->D == 2 ? p->ny : 1, klo = p->D == 2 ? -2 : 0, khi = p->D == 2 ? ny + 2 : 1;
  if (j < -2 || j >= p->nx + 2 || k < klo || k >= khi || (j >= 0 && j < p->nx && k >= 0 && k < ny))
    return 3;
  orc_grid G;
  if (!orc_grid_alloc(&G, p)) { orc_grid_free(&G); return 2; }
  const int ncp = orc_ncp(&G);
  const size_t n = (size_t)G.nx * G.ny;
  for (int kk = 0; kk < G.ny; ++kk)
    for (int jj = 0; jj < G.nx; ++jj) {
      size_t s = (size_t)kk * G.nx + jj;
      int c = orc_pidx(&G, jj, kk);
      for (int i = 0; i < G.Qf; ++i) G.f[i * ncp + c] = f[i * n + s];
      for (int i = 0; i < G.Qg; ++i) G.g[i * ncp + c] = g[i * n + s];
      G.ux[c] = ux[s]; G.uy[c] = p->D == 2 ? uy[s] : 0.0; G.T[c] = T[s];
    }
  orc_fill_ghosts(&G);
  const int c = orc_pidx(&G, j, k);
  for (int i = 0; i < G.Qf; ++i) fout[i] = G.f[i * ncp + c];
  for (int i = 0; i < G.Qg; ++i) gout[i] = G.g[i * ncp + c];
  frame[0] = G.ux[c]; frame[1] = G.uy[c]; frame[2] = G.T[c];
  orc_grid_free(&G);
  return 0;
}

/* Multiscale switching measures s_u, s_T of every interior cell of the
 * fields (ux, uy, T) under the run's boundary rules. */
int orc_ms_measure_pub(const orc_params *p, const double *ux, const double *uy, const double *T,
                       double *su, double *sT) {
  if (!orc_check(p)) return 1;
  orc_grid G;
  if (!orc_grid_alloc(&G, p)) { orc_grid_free(&G); return 2; }
  for (int k = 0; k < G.ny; ++k)
    for (int j = 0; j < G.nx; ++j) {
      size_t s = (size_t)k * G.nx + j;
      int c = orc_pidx(&G, j, k);
      G.ux[c] = ux[s]; G.uy[c] = p->D == 2 ? uy[s] : 0.0; G.T[c] = T[s];
      G.f[c] = 1.0; /* a density for the inflow-free ghost copies */
    }
  orc_fill_ghosts(&G);
  for (int k = 0; k < G.ny; ++k)
    for (int j = 0; j < G.nx; ++j)
      orc_ms_measure(&G, j, k, su + (size_t)k * G.nx + j, sT + (size_t)k * G.nx + j);
  orc_grid_free(&G);
  return 0;
}

#ifdef ORC_COUNT_OPS
/* The floating-point operations of nsteps steps (OPS above), counted on one
 * thread; the state is advanced in place as by orc_run. */
int orc_count_ops(const orc_params *p, double *f, double *g, double *ux, double *uy, double *T,
                  int64_t nsteps, orc_report *rep, int64_t *ops) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  extern void omp_set_num_threads(int);
  const int nt = omp_get_max_threads();
  omp_set_num_threads(1);
#endif
  orc_ops = 0;
  orc_counting = 1;
  const int rc = orc_run(p, f, g, ux, uy, T, nsteps, rep);
  orc_counting = 0;
  *ops = orc_ops;
#ifdef _OPENMP
  omp_set_num_threads(nt);
#endif
  return rc;
}
#endif

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int orc_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Sets the number of OpenMP threads for later runs (no effect without OpenMP). */
void orc_set_threads(int n) {
#ifdef _OPENMP
  extern void omp_set_num_threads(int);
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
