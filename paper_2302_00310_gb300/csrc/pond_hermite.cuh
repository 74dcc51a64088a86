// pond_hermite.cuh -- per-axis Hermite algebra of the PonD frame transformation
// on the Gauss-Hermite lattices of Table I (arXiv:2302.00310), for sm_103a.
//
// Representation.  A population vector p_j on a q-node axis, in the frame
// {u, T} (velocities v_j = u + sqrt(T) c_j), is kept as its q dimensional
// Hermite coefficients B_n = sum_j p_j H_n(v_j - u; T), where
// H_n(x; T) = T^(n/2) He_n(x / sqrt(T)) (H_0 = 1, H_1 = x, H_2 = x^2 - T,
// H_3 = x^3 - 3 T x) and He_n are the probabilists' Hermite polynomials of
// Appendix A.  B_n = T^(n/2) A_n with A_n the Hermite coefficients of the
// populations, so the map is invertible on the lattice (Eq. GradsProjection
// restricted to one axis: p_j = w_j sum_n He_n(c_j) A_n / n!, the nodes being
// the roots of He_q).
//
// Frame transformation.  The generating function exp(t x - T t^2 / 2) of the
// H_n factorises, so H_n(x + d; T') = sum_k binom(n, k) H_k(x; T) H_{n-k}(d; T' - T).
// Moving populations from {u, T} to {u', T'} with the moments of order <= q-1
// invariant (Eq. eq:Mcondition) therefore maps the coefficients by the unit
// lower-triangular B'_n = sum_k binom(n, k) h_{n-k} B_k, with d = u - u' and
// h_0 = 1, h_1 = d, h_2 = d^2 + (T - T'), h_3 = d (d^2 + 3 (T - T')): six
// fused multiply-adds per 4-vector and no square root.  In 2D the
// transformation is the tensor product of the per-axis maps; the Grad
// projection of total order K (Sec. V.A) additionally zeroes coefficients
// with a + b > K.
//
// Everything here is templated on the arithmetic type R (double or float).
#pragma once

namespace pond {

// ---- Table I constants --------------------------------------------------
// D1Q4 nodes -R2, -R1, R1, R2 with R1,2 = sqrt(3 -+ sqrt 6), weights W2, W1, W1, W2.
constexpr double R1 = 0.7419637843027258;
constexpr double R2 = 2.3344142183389773;
constexpr double W1 = 0.4541241452319315;   // (3 + sqrt 6)/12
constexpr double W2 = 0.04587585476806849;  // (3 - sqrt 6)/12
constexpr double H2R1 = -0.4494897427831781; // He_2(R1) = 2 - sqrt 6
constexpr double H2R2 = 4.449489742783178;   // He_2(R2) = 2 + sqrt 6
constexpr double H3R1 = -1.8174326791661175; // He_3(R1) = -sqrt 6 R1
constexpr double H3R2 = 5.718123683228535;   // He_3(R2) =  sqrt 6 R2
// synthesis coefficients w_r He_n(r)/n! for r = R1, R2
constexpr double SE0_1 = 0.4541241452319315;
constexpr double SE2_1 = -0.10206207261596575;
constexpr double SO1_1 = 0.3369436693395246;
constexpr double SO3_1 = -0.13755667699048205;
constexpr double SE0_2 = 0.04587585476806849;
constexpr double SE2_2 = 0.10206207261596575;
constexpr double SO1_2 = 0.10709324764903305;
constexpr double SO3_2 = 0.04372063527294086;
// D1Q3 nodes -sqrt 3, 0, sqrt 3 with weights 1/6, 2/3, 1/6
constexpr double SQ3 = 1.7320508075688772;
constexpr double SQ3_6 = 0.28867513459481287;

template <int Q> struct Nodes;
template <> struct Nodes<4> {
  __device__ __forceinline__ static double c(int k) {
    return k == 0 ? -R2 : (k == 1 ? -R1 : (k == 2 ? R1 : R2));
  }
  static constexpr double cmax = R2;
};
template <> struct Nodes<3> {
  __device__ __forceinline__ static double c(int k) { return k == 0 ? -SQ3 : (k == 1 ? 0.0 : SQ3); }
  static constexpr double cmax = SQ3;
};

// ---- one axis: populations <-> thermal coefficients A_n = B_n T^(-n/2) ------
// (the change of basis at the library boundary)
template <typename R>
__device__ __forceinline__ void syn4(R &a0, R &a1, R &a2, R &a3) {
  const R e1 = R(SE0_1) * a0 + R(SE2_1) * a2, o1 = R(SO1_1) * a1 + R(SO3_1) * a3;
  const R e2 = R(SE0_2) * a0 + R(SE2_2) * a2, o2 = R(SO1_2) * a1 + R(SO3_2) * a3;
  a0 = e2 - o2; a1 = e1 - o1; a2 = e1 + o1; a3 = e2 + o2;
}
template <typename R>
__device__ __forceinline__ void ana4(R &p0, R &p1, R &p2, R &p3) {
  const R s1 = p2 + p1, d1 = p2 - p1, s2 = p3 + p0, d2 = p3 - p0;
  p0 = s1 + s2;
  p1 = R(R1) * d1 + R(R2) * d2;
  p2 = R(H2R1) * s1 + R(H2R2) * s2;
  p3 = R(H3R1) * d1 + R(H3R2) * d2;
}
template <typename R>
__device__ __forceinline__ void syn3(R &a0, R &a1, R &a2) {
  const R mid = R(2.0 / 3.0) * a0 - R(1.0 / 3.0) * a2;
  const R e = R(1.0 / 6.0) * (a0 + a2), o = R(SQ3_6) * a1;
  a0 = e - o; a1 = mid; a2 = e + o;
}
template <typename R>
__device__ __forceinline__ void ana3(R &p0, R &p1, R &p2) {
  const R s = p0 + p2, d = p2 - p0;
  const R A0 = s + p1, A1 = R(SQ3) * d, A2 = R(2) * s - p1;
  p0 = A0; p1 = A1; p2 = A2;
}

// ---- one axis: values at the nodes of a frame, divided by the weights -----
// q_j = p_j / w_j = sum_n He_n(c_j) T^(-n/2) B_n / n! at the nodes of the frame
// with temperature T.  The constants depend only on the frame: with
// iT = 1/T and isT = 1/sqrt(T), D1Q4 (nodes -R2, -R1, R1, R2):
//   q(+-R_r) = (B_0 + He_2(R_r)/2 iT B_2) +- R_r isT (B_1 -+ sqrt6/6 iT B_3)
// (He_3(R_r)/6 = R_r (R_r^2 - 3)/6 = -+ R_r sqrt6/6); D1Q3 (nodes -sqrt3, 0, sqrt3):
//   q(+-sqrt3) = B_0 + iT B_2 +- sqrt3 isT B_1,  q(0) = B_0 - iT/2 B_2.
constexpr double K6 = 0.408248290463863;  // sqrt(6)/6
template <typename R, int Q> struct SynK;
// (the converting constructors copy another arithmetic type's constants, e.g.
// the same frame's FP32 constants into both lanes of a packed pair)
template <typename R> struct SynK<R, 4> {
  R h1, h2, k, r1, r2;
  __device__ __forceinline__ SynK(R iT, R isT)
      : h1(R(0.5 * H2R1) * iT), h2(R(0.5 * H2R2) * iT), k(R(K6) * iT), r1(R(R1) * isT), r2(R(R2) * isT) {}
  template <typename S>
  __device__ __forceinline__ explicit SynK(const SynK<S, 4> &o)
      : h1(R(o.h1)), h2(R(o.h2)), k(R(o.k)), r1(R(o.r1)), r2(R(o.r2)) {}
};
template <typename R> struct SynK<R, 3> {
  R e, z, r;
  __device__ __forceinline__ SynK(R iT, R isT) : e(iT), z(R(-0.5) * iT), r(R(SQ3) * isT) {}
  template <typename S>
  __device__ __forceinline__ explicit SynK(const SynK<S, 3> &o) : e(R(o.e)), z(R(o.z)), r(R(o.r)) {}
};
template <typename R>
__device__ __forceinline__ void synq(const SynK<R, 4> &S, R &m0, R &m1, R &m2, R &m3) {
  const R e1 = fma(S.h1, m2, m0), e2 = fma(S.h2, m2, m0);
  const R t1 = fma(-S.k, m3, m1), t2 = fma(S.k, m3, m1);
  m0 = fma(-S.r2, t2, e2); m1 = fma(-S.r1, t1, e1); m2 = fma(S.r1, t1, e1); m3 = fma(S.r2, t2, e2);
}
template <typename R>
__device__ __forceinline__ void synq(const SynK<R, 3> &S, R &m0, R &m1, R &m2) {
  const R e = fma(S.e, m2, m0), mid = fma(S.z, m2, m0);
  const R lo = fma(-S.r, m1, e), hi = fma(S.r, m1, e);
  m0 = lo; m1 = mid; m2 = hi;
}

// ---- one axis: dimensional coefficients from node values q_j = p_j / w_j -------
// B_n = T^(n/2) sum_j w_j He_n(c_j) q_j in the frame with temperature T.
template <typename R, int Q> struct AnaK;
template <typename R> struct AnaK<R, 4> {
  R b11, b12, b21, b22, b31, b32;
  __device__ __forceinline__ AnaK(R T, R sT)
      : b11(R(W1 * R1) * sT), b12(R(W2 * R2) * sT), b21(R(W1 * H2R1) * T), b22(R(W2 * H2R2) * T),
        b31(R(W1 * H3R1) * (T * sT)), b32(R(W2 * H3R2) * (T * sT)) {}
};
template <typename R> struct AnaK<R, 3> {
  R b1, b2s, b2m;
  __device__ __forceinline__ AnaK(R T, R sT)
      : b1(R(SQ3 / 6.0) * sT), b2s(R(1.0 / 3.0) * T), b2m(R(-2.0 / 3.0) * T) {}
};
template <typename R>
__device__ __forceinline__ void anaq(const AnaK<R, 4> &A, R &q0, R &q1, R &q2, R &q3) {
  const R s1 = q2 + q1, d1 = q2 - q1, s2 = q3 + q0, d2 = q3 - q0;
  q0 = fma(R(W2), s2, R(W1) * s1);
  q1 = fma(A.b12, d2, A.b11 * d1);
  q2 = fma(A.b22, s2, A.b21 * s1);
  q3 = fma(A.b32, d2, A.b31 * d1);
}
template <typename R>
__device__ __forceinline__ void anaq(const AnaK<R, 3> &A, R &q0, R &q1, R &q2) {
  const R s = q0 + q2, d = q2 - q0;
  const R B0 = fma(R(2.0 / 3.0), q1, R(1.0 / 6.0) * s), B2 = fma(A.b2m, q1, A.b2s * s);
  q0 = B0; q1 = A.b1 * d; q2 = B2;
}

// ---- one axis: the frame change of dimensional coefficients ---------------
// d = u - u', dT = T - T' (dT3 = 3 dT, shared by the axes of one change)
template <typename R> struct DShift {
  R d, d2, d3, g2, g2x3, g3;
  R d4, g2x6, g3x4, g4;  // order 4 (D1Q5 only; unused members cost nothing)
};
template <typename R>
__device__ __forceinline__ DShift<R> make_dshift(R d, R dT, R dT3) {
  DShift<R> C;
  C.d = d; C.d2 = d + d; C.d3 = R(3) * d;
  C.g2 = fma(d, d, dT); C.g2x3 = R(3) * C.g2;
  C.g3 = d * fma(d, d, dT3);
  C.d4 = R(4) * d; C.g2x6 = R(6) * C.g2; C.g3x4 = R(4) * C.g3;
  const R dd = d * d;
  C.g4 = fma(dd, fma(R(6), dT, dd), R(3) * dT * dT);
  return C;
}
template <typename R>
__device__ __forceinline__ void dshift4(const DShift<R> &C, R &m0, R &m1, R &m2, R &m3) {
  m3 = fma(C.g3, m0, fma(C.g2x3, m1, fma(C.d3, m2, m3)));
  m2 = fma(C.g2, m0, fma(C.d2, m1, m2));
  m1 = fma(C.d, m0, m1);
}
template <typename R>
__device__ __forceinline__ void dshift3(const DShift<R> &C, R &m0, R &m1, R &m2) {
  m2 = fma(C.g2, m0, fma(C.d2, m1, m2));
  m1 = fma(C.d, m0, m1);
}

// ---- one axis: multiplication of the populations by v = u + x --------------
// x H_k(x; T) = H_{k+1} + k T H_{k-1}, and H_q(., T) vanishes on the q nodes of
// the frame, so on the lattice the coefficients of v p are
// u B_k + B_{k+1} + k T B_{k-1} (B_q = 0).
template <typename R>
__device__ __forceinline__ void dvmul4(R u, R T, R &a0, R &a1, R &a2, R &a3) {
  const R b0 = fma(u, a0, a1), b1 = fma(u, a1, fma(T, a0, a2));
  const R b2 = fma(u, a2, fma(T + T, a1, a3)), b3 = fma(u, a3, (R(3) * T) * a2);
  a0 = b0; a1 = b1; a2 = b2; a3 = b3;
}
template <typename R>
__device__ __forceinline__ void dvmul3(R u, R T, R &a0, R &a1, R &a2) {
  const R b0 = fma(u, a0, a1), b1 = fma(u, a1, fma(T, a0, a2)), b2 = fma(u, a2, (T + T) * a1);
  a0 = b0; a1 = b1; a2 = b2;
}

// ---- D1Q5 (the f-lattice of D2Q25): nodes -R2q, -R1q, 0, R1q, R2q, the roots
// of He_5 (R1q,2q = sqrt(5 -+ sqrt 10)), weights W2q, W1q, W0q, W1q, W2q --------
constexpr double R1Q = 1.355626179974266;
constexpr double R2Q = 2.8569700138728056;
constexpr double W0Q = 0.5333333333333333;   // 8/15
constexpr double W1Q = 0.2220759220056127;   // (7 + 2 sqrt 10)/60
constexpr double W2Q = 0.011257411327720691; // (7 - 2 sqrt 10)/60
template <> struct Nodes<5> {
  __device__ __forceinline__ static double c(int k) {
    return k == 0 ? -R2Q : (k == 1 ? -R1Q : (k == 2 ? 0.0 : (k == 3 ? R1Q : R2Q)));
  }
  static constexpr double cmax = R2Q;
};
// He_n at the D1Q5 nodes, n = 2, 3, 4
__host__ __device__ constexpr double he2(double c) { return c * c - 1.0; }
__host__ __device__ constexpr double he3(double c) { return c * c * c - 3.0 * c; }
__host__ __device__ constexpr double he4(double c) { return c * c * c * c - 6.0 * c * c + 3.0; }

// populations <-> thermal coefficients (library boundary): A_n = sum_j p_j He_n(c_j),
// p_j = w_j sum_n He_n(c_j) A_n / n!
template <typename R>
__device__ __forceinline__ void syn5(R &a0, R &a1, R &a2, R &a3, R &a4) {
  const double cs[5] = {-R2Q, -R1Q, 0.0, R1Q, R2Q}, ws[5] = {W2Q, W1Q, W0Q, W1Q, W2Q};
  const R A[5] = {a0, a1, a2, a3, a4};
  R p[5];
#pragma unroll
  for (int j = 0; j < 5; ++j)
    p[j] = R(ws[j]) * (A[0] + R(cs[j]) * A[1] + R(he2(cs[j]) / 2.0) * A[2] + R(he3(cs[j]) / 6.0) * A[3] +
                       R(he4(cs[j]) / 24.0) * A[4]);
  a0 = p[0]; a1 = p[1]; a2 = p[2]; a3 = p[3]; a4 = p[4];
}
template <typename R>
__device__ __forceinline__ void ana5(R &p0, R &p1, R &p2, R &p3, R &p4) {
  const double cs[5] = {-R2Q, -R1Q, 0.0, R1Q, R2Q};
  const R P[5] = {p0, p1, p2, p3, p4};
  R A[5] = {R(0), R(0), R(0), R(0), R(0)};
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    A[0] += P[j];
    A[1] += R(cs[j]) * P[j];
    A[2] += R(he2(cs[j])) * P[j];
    A[3] += R(he3(cs[j])) * P[j];
    A[4] += R(he4(cs[j])) * P[j];
  }
  p0 = A[0]; p1 = A[1]; p2 = A[2]; p3 = A[3]; p4 = A[4];
}

// node values over weights in the frame with temperature T (iT = 1/T, isT = 1/sqrt T):
// q(+-R) = E_R +- R isT (B_1 + k_R iT B_3), E_R = B_0 + He_2(R)/2 iT B_2 + He_4(R)/24 iT^2 B_4,
// q(0) = B_0 - iT/2 B_2 + iT^2/8 B_4 (k_R = (R^2 - 3)/6)
template <typename R> struct SynK<R, 5> {
  R h21, h41, k1, r1, nr1, h22, h42, k2, r2, nr2, z2, z4;
  __device__ __forceinline__ SynK(R iT, R isT)
      : h21(R(0.5 * he2(R1Q)) * iT), h41(R(he4(R1Q) / 24.0) * (iT * iT)), k1(R((R1Q * R1Q - 3.0) / 6.0) * iT),
        r1(R(R1Q) * isT), nr1(R(-R1Q) * isT), h22(R(0.5 * he2(R2Q)) * iT),
        h42(R(he4(R2Q) / 24.0) * (iT * iT)), k2(R((R2Q * R2Q - 3.0) / 6.0) * iT), r2(R(R2Q) * isT),
        nr2(R(-R2Q) * isT), z2(R(-0.5) * iT), z4(R(0.125) * (iT * iT)) {}
  template <typename S>
  __device__ __forceinline__ explicit SynK(const SynK<S, 5> &o)
      : h21(R(o.h21)), h41(R(o.h41)), k1(R(o.k1)), r1(R(o.r1)), nr1(R(o.nr1)), h22(R(o.h22)), h42(R(o.h42)),
        k2(R(o.k2)), r2(R(o.r2)), nr2(R(o.nr2)), z2(R(o.z2)), z4(R(o.z4)) {}
};
template <typename R>
__device__ __forceinline__ void synq(const SynK<R, 5> &S, R &m0, R &m1, R &m2, R &m3, R &m4) {
  const R e1 = fma(S.h41, m4, fma(S.h21, m2, m0)), e2 = fma(S.h42, m4, fma(S.h22, m2, m0));
  const R t1 = fma(S.k1, m3, m1), t2 = fma(S.k2, m3, m1);
  const R c0 = fma(S.z4, m4, fma(S.z2, m2, m0));
  m0 = fma(S.nr2, t2, e2); m1 = fma(S.nr1, t1, e1); m2 = c0; m3 = fma(S.r1, t1, e1); m4 = fma(S.r2, t2, e2);
}
// dimensional coefficients from node values over weights: B_n = T^(n/2) sum_j w_j He_n(c_j) q_j
template <typename R> struct AnaK<R, 5> {
  R b11, b12, b20, b21, b22, b31, b32, b40, b41, b42;
  __device__ __forceinline__ AnaK(R T, R sT)
      : b11(R(W1Q * R1Q) * sT), b12(R(W2Q * R2Q) * sT), b20(R(-W0Q) * T), b21(R(W1Q * he2(R1Q)) * T),
        b22(R(W2Q * he2(R2Q)) * T), b31(R(W1Q * he3(R1Q)) * (T * sT)), b32(R(W2Q * he3(R2Q)) * (T * sT)),
        b40(R(3.0 * W0Q) * (T * T)), b41(R(W1Q * he4(R1Q)) * (T * T)), b42(R(W2Q * he4(R2Q)) * (T * T)) {}
};
template <typename R>
__device__ __forceinline__ void anaq(const AnaK<R, 5> &A, R &q0, R &q1, R &q2, R &q3, R &q4) {
  const R s1 = q3 + q1, d1 = q3 - q1, s2 = q4 + q0, d2 = q4 - q0, c = q2;
  const R B0 = fma(R(W2Q), s2, fma(R(W1Q), s1, R(W0Q) * c));
  const R B1 = fma(A.b12, d2, A.b11 * d1);
  const R B2 = fma(A.b22, s2, fma(A.b21, s1, A.b20 * c));
  const R B3 = fma(A.b32, d2, A.b31 * d1);
  const R B4 = fma(A.b42, s2, fma(A.b41, s1, A.b40 * c));
  q0 = B0; q1 = B1; q2 = B2; q3 = B3; q4 = B4;
}
// frame change, order 4: B'_4 = B_4 + 4 d B_3 + 6 h_2 B_2 + 4 h_3 B_1 + h_4 B_0,
// h_4 = H_4(d; T' - T) = d^4 + 6 (T - T') d^2 + 3 (T - T')^2
template <typename R>
__device__ __forceinline__ void dshift5(const DShift<R> &C, R &m0, R &m1, R &m2, R &m3, R &m4) {
  m4 = fma(C.g4, m0, fma(C.g3x4, m1, fma(C.g2x6, m2, fma(C.d4, m3, m4))));
  m3 = fma(C.g3, m0, fma(C.g2x3, m1, fma(C.d3, m2, m3)));
  m2 = fma(C.g2, m0, fma(C.d2, m1, m2));
  m1 = fma(C.d, m0, m1);
}
// v = u + x: coefficients u B_k + B_{k+1} + k T B_{k-1}, B_5 = 0 on the five nodes
template <typename R>
__device__ __forceinline__ void dvmul5(R u, R T, R &a0, R &a1, R &a2, R &a3, R &a4) {
  const R b0 = fma(u, a0, a1), b1 = fma(u, a1, fma(T, a0, a2)), b2 = fma(u, a2, fma(T + T, a1, a3));
  const R b3 = fma(u, a3, fma(R(3) * T, a2, a4)), b4 = fma(u, a4, (R(4) * T) * a3);
  a0 = b0; a1 = b1; a2 = b2; a3 = b3; a4 = b4;
}

// ---- coefficient blocks: A[x-order][y-order], NY = 1 in 1D ---------------
template <typename R, int Q, int NY> struct Blk {
  R v[Q][NY];
};

template <typename R, int Q, int NY>
__device__ __forceinline__ void syn_x(Blk<R, Q, NY> &B) {
#pragma unroll
  for (int m = 0; m < NY; ++m) {
    if constexpr (Q == 5) syn5(B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m], B.v[4][m]);
    else if constexpr (Q == 4) syn4(B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m]);
    else syn3(B.v[0][m], B.v[1][m], B.v[2][m]);
  }
}
template <typename R, int Q, int NY>
__device__ __forceinline__ void syn_y(Blk<R, Q, NY> &B) {
  if constexpr (NY > 1) {
#pragma unroll
    for (int n = 0; n < Q; ++n) {
      if constexpr (Q == 5) syn5(B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3], B.v[n][4]);
      else if constexpr (Q == 4) syn4(B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3]);
      else syn3(B.v[n][0], B.v[n][1], B.v[n][2]);
    }
  }
}
template <typename R, int Q, int NY>
__device__ __forceinline__ void ana_x(Blk<R, Q, NY> &B) {
#pragma unroll
  for (int m = 0; m < NY; ++m) {
    if constexpr (Q == 5) ana5(B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m], B.v[4][m]);
    else if constexpr (Q == 4) ana4(B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m]);
    else ana3(B.v[0][m], B.v[1][m], B.v[2][m]);
  }
}
template <typename R, int Q, int NY>
__device__ __forceinline__ void ana_y(Blk<R, Q, NY> &B) {
  if constexpr (NY > 1) {
#pragma unroll
    for (int n = 0; n < Q; ++n) {
      if constexpr (Q == 5) ana5(B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3], B.v[n][4]);
      else if constexpr (Q == 4) ana4(B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3]);
      else ana3(B.v[n][0], B.v[n][1], B.v[n][2]);
    }
  }
}
template <typename R, int Q, int NY>
__device__ __forceinline__ void shift_x(const DShift<R> &C, Blk<R, Q, NY> &B) {
#pragma unroll
  for (int m = 0; m < NY; ++m) {
    if constexpr (Q == 5) dshift5(C, B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m], B.v[4][m]);
    else if constexpr (Q == 4) dshift4(C, B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m]);
    else dshift3(C, B.v[0][m], B.v[1][m], B.v[2][m]);
  }
}
template <typename R, int Q, int NY>
__device__ __forceinline__ void shift_y(const DShift<R> &C, Blk<R, Q, NY> &B) {
  if constexpr (NY > 1) {
#pragma unroll
    for (int n = 0; n < Q; ++n) {
      if constexpr (Q == 5) dshift5(C, B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3], B.v[n][4]);
      else if constexpr (Q == 4) dshift4(C, B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3]);
      else dshift3(C, B.v[n][0], B.v[n][1], B.v[n][2]);
    }
  }
}
// one Q-vector along either axis: the frame change and the synthesis at the
// nodes (the per-axis maps that the tensor-product transformation composes)
template <typename R, int Q>
__device__ __forceinline__ void dshiftq(const DShift<R> &C, R (&m)[Q]) {
  if constexpr (Q == 5) dshift5(C, m[0], m[1], m[2], m[3], m[4]);
  else if constexpr (Q == 4) dshift4(C, m[0], m[1], m[2], m[3]);
  else dshift3(C, m[0], m[1], m[2]);
}
template <typename R, int Q>
__device__ __forceinline__ void synqq(const SynK<R, Q> &S, R (&m)[Q]) {
  if constexpr (Q == 5) synq(S, m[0], m[1], m[2], m[3], m[4]);
  else if constexpr (Q == 4) synq(S, m[0], m[1], m[2], m[3]);
  else synq(S, m[0], m[1], m[2]);
}
// the constants of c ? A : B, member by member (the members Q does not use
// are dead code)
template <typename R>
__device__ __forceinline__ DShift<R> select_shift(bool c, const DShift<R> &A, const DShift<R> &B) {
  DShift<R> C;
  C.d = c ? A.d : B.d; C.d2 = c ? A.d2 : B.d2; C.d3 = c ? A.d3 : B.d3;
  C.g2 = c ? A.g2 : B.g2; C.g2x3 = c ? A.g2x3 : B.g2x3; C.g3 = c ? A.g3 : B.g3;
  C.d4 = c ? A.d4 : B.d4; C.g2x6 = c ? A.g2x6 : B.g2x6; C.g3x4 = c ? A.g3x4 : B.g3x4;
  C.g4 = c ? A.g4 : B.g4;
  return C;
}

// node values / weights in the frame of S, x then y
template <typename R, int Q, int NY>
__device__ __forceinline__ void synq_xy(const SynK<R, Q> &S, Blk<R, Q, NY> &B) {
#pragma unroll
  for (int m = 0; m < NY; ++m) {
    if constexpr (Q == 5) synq(S, B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m], B.v[4][m]);
    else if constexpr (Q == 4) synq(S, B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m]);
    else synq(S, B.v[0][m], B.v[1][m], B.v[2][m]);
  }
  if constexpr (NY > 1) {
#pragma unroll
    for (int n = 0; n < Q; ++n) {
      if constexpr (Q == 5) synq(S, B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3], B.v[n][4]);
      else if constexpr (Q == 4) synq(S, B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3]);
      else synq(S, B.v[n][0], B.v[n][1], B.v[n][2]);
    }
  }
}
// dimensional coefficients in the frame of A from node values / weights
template <typename R, int Q, int NY>
__device__ __forceinline__ void anaq_xy(const AnaK<R, Q> &A, Blk<R, Q, NY> &B) {
#pragma unroll
  for (int m = 0; m < NY; ++m) {
    if constexpr (Q == 5) anaq(A, B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m], B.v[4][m]);
    else if constexpr (Q == 4) anaq(A, B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m]);
    else anaq(A, B.v[0][m], B.v[1][m], B.v[2][m]);
  }
  if constexpr (NY > 1) {
#pragma unroll
    for (int n = 0; n < Q; ++n) {
      if constexpr (Q == 5) anaq(A, B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3], B.v[n][4]);
      else if constexpr (Q == 4) anaq(A, B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3]);
      else anaq(A, B.v[n][0], B.v[n][1], B.v[n][2]);
    }
  }
}
// multiply by v_axis = u + x in the frame with temperature T
template <int AX, typename R, int Q, int NY>
__device__ __forceinline__ void vmul(R u, R T, Blk<R, Q, NY> &B) {
  if constexpr (AX == 0) {
#pragma unroll
    for (int m = 0; m < NY; ++m) {
      if constexpr (Q == 5) dvmul5(u, T, B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m], B.v[4][m]);
      else if constexpr (Q == 4) dvmul4(u, T, B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m]);
      else dvmul3(u, T, B.v[0][m], B.v[1][m], B.v[2][m]);
    }
  } else {
#pragma unroll
    for (int n = 0; n < Q; ++n) {
      if constexpr (Q == 5) dvmul5(u, T, B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3], B.v[n][4]);
      else if constexpr (Q == 4) dvmul4(u, T, B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3]);
      else dvmul3(u, T, B.v[n][0], B.v[n][1], B.v[n][2]);
    }
  }
}
// scale coefficient B_ab by s^(a+b) (between thermal and dimensional units)
template <typename R, int Q, int NY>
__device__ __forceinline__ void scale_orders(R s, Blk<R, Q, NY> &B) {
  R p[2 * Q - 1];
  p[0] = R(1);
#pragma unroll
  for (int i = 1; i < 2 * Q - 1; ++i) p[i] = p[i - 1] * s;
#pragma unroll
  for (int n = 0; n < Q; ++n)
#pragma unroll
    for (int m = 0; m < NY; ++m) B.v[n][m] *= p[n + m];
}
// Grad projection of total order Q-1: drop coefficients with a + b > Q-1
template <typename R, int Q, int NY>
__device__ __forceinline__ void grad_mask(Blk<R, Q, NY> &B) {
  if constexpr (NY > 1) {
#pragma unroll
    for (int n = 0; n < Q; ++n)
#pragma unroll
      for (int m = 0; m < NY; ++m)
        if (n + m > Q - 1) B.v[n][m] = R(0);
  }
}

}  // namespace pond
