// pond_hermite.cuh -- per-axis Hermite algebra of the PonD frame transformation
// on the Gauss-Hermite lattices of Table I (arXiv:2302.00310), for sm_103a.
//
// Representation.  A population vector on a q-node axis is kept as its q
// Hermite coefficients A_n = sum_j p_j He_n(c_j) (probabilists' Hermite
// polynomials of Appendix A).  Because the nodes are the roots of He_q, the
// map is invertible on the lattice: p_j = w_j sum_n He_n(c_j) A_n / n!
// (Eq. GradsProjection restricted to one axis).
//
// Frame transformation.  Moving populations from frame {u, T} to {u', T'}
// with moments up to order K = q-1 invariant (Eq. eq:Mcondition) maps the
// coefficients by A'_n = sum_k C_nk(a, b) A_k, with a = sqrt(T/T'),
// b = (u - u')/sqrt(T') and He_n(a x + b) = sum_k C_nk He_k(x) (a lower
// triangular matrix with polynomial entries).  In 2D the transformation is
// the tensor product of the per-axis maps; the Grad projection of total order
// K (Sec. V.A) additionally zeroes coefficients with a + b > K.
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

// ---- one axis: synthesis / analysis --------------------------------------
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

// ---- one axis: Hermite shift/scale matrix C(a, b) -------------------------
template <typename R> struct Shift {
  R a, b, c20, c21, c22, c30, c31, c32, c33;
};
template <typename R>
__device__ __forceinline__ Shift<R> make_shift(R a, R b) {
  Shift<R> C;
  const R a2 = a * a, b2 = b * b, am1 = a2 - R(1), t = am1 + b2;
  C.a = a; C.b = b;
  C.c20 = t; C.c21 = R(2) * a * b; C.c22 = a2;
  C.c30 = b * (b2 + R(3) * am1); C.c31 = R(3) * a * t; C.c32 = R(3) * a2 * b; C.c33 = a2 * a;
  return C;
}
template <typename R>
__device__ __forceinline__ void shift4(const Shift<R> &C, R &m0, R &m1, R &m2, R &m3) {
  const R n3 = C.c30 * m0 + C.c31 * m1 + C.c32 * m2 + C.c33 * m3;
  const R n2 = C.c20 * m0 + C.c21 * m1 + C.c22 * m2;
  const R n1 = C.b * m0 + C.a * m1;
  m1 = n1; m2 = n2; m3 = n3;
}
template <typename R>
__device__ __forceinline__ void shift3(const Shift<R> &C, R &m0, R &m1, R &m2) {
  const R n2 = C.c20 * m0 + C.c21 * m1 + C.c22 * m2;
  const R n1 = C.b * m0 + C.a * m1;
  m1 = n1; m2 = n2;
}

// ---- one axis: multiplication of the populations by v = u + s c ----------
// c He_n = He_{n+1} + n He_{n-1}; He_q vanishes on the q nodes, so the map is
// exact on the lattice: B_k = k A_{k-1} + A_{k+1} (A_q = 0).
template <typename R>
__device__ __forceinline__ void vmul4(R u, R s, R &a0, R &a1, R &a2, R &a3) {
  const R b0 = a1, b1 = a0 + a2, b2 = R(2) * a1 + a3, b3 = R(3) * a2;
  a0 = u * a0 + s * b0; a1 = u * a1 + s * b1; a2 = u * a2 + s * b2; a3 = u * a3 + s * b3;
}
template <typename R>
__device__ __forceinline__ void vmul3(R u, R s, R &a0, R &a1, R &a2) {
  const R b0 = a1, b1 = a0 + a2, b2 = R(2) * a1;
  a0 = u * a0 + s * b0; a1 = u * a1 + s * b1; a2 = u * a2 + s * b2;
}

// ---- coefficient blocks: A[x-order][y-order], NY = 1 in 1D ---------------
template <typename R, int Q, int NY> struct Blk {
  R v[Q][NY];
};

template <typename R, int Q, int NY>
__device__ __forceinline__ void syn_x(Blk<R, Q, NY> &B) {
#pragma unroll
  for (int m = 0; m < NY; ++m) {
    if constexpr (Q == 4) syn4(B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m]);
    else syn3(B.v[0][m], B.v[1][m], B.v[2][m]);
  }
}
template <typename R, int Q, int NY>
__device__ __forceinline__ void syn_y(Blk<R, Q, NY> &B) {
  if constexpr (NY > 1) {
#pragma unroll
    for (int n = 0; n < Q; ++n) {
      if constexpr (Q == 4) syn4(B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3]);
      else syn3(B.v[n][0], B.v[n][1], B.v[n][2]);
    }
  }
}
template <typename R, int Q, int NY>
__device__ __forceinline__ void ana_x(Blk<R, Q, NY> &B) {
#pragma unroll
  for (int m = 0; m < NY; ++m) {
    if constexpr (Q == 4) ana4(B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m]);
    else ana3(B.v[0][m], B.v[1][m], B.v[2][m]);
  }
}
template <typename R, int Q, int NY>
__device__ __forceinline__ void ana_y(Blk<R, Q, NY> &B) {
  if constexpr (NY > 1) {
#pragma unroll
    for (int n = 0; n < Q; ++n) {
      if constexpr (Q == 4) ana4(B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3]);
      else ana3(B.v[n][0], B.v[n][1], B.v[n][2]);
    }
  }
}
template <typename R, int Q, int NY>
__device__ __forceinline__ void shift_x(const Shift<R> &C, Blk<R, Q, NY> &B) {
#pragma unroll
  for (int m = 0; m < NY; ++m) {
    if constexpr (Q == 4) shift4(C, B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m]);
    else shift3(C, B.v[0][m], B.v[1][m], B.v[2][m]);
  }
}
template <typename R, int Q, int NY>
__device__ __forceinline__ void shift_y(const Shift<R> &C, Blk<R, Q, NY> &B) {
  if constexpr (NY > 1) {
#pragma unroll
    for (int n = 0; n < Q; ++n) {
      if constexpr (Q == 4) shift4(C, B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3]);
      else shift3(C, B.v[n][0], B.v[n][1], B.v[n][2]);
    }
  }
}
// multiply by v_axis = u + s c_axis
template <int AX, typename R, int Q, int NY>
__device__ __forceinline__ void vmul(R u, R s, Blk<R, Q, NY> &B) {
  if constexpr (AX == 0) {
#pragma unroll
    for (int m = 0; m < NY; ++m) {
      if constexpr (Q == 4) vmul4(u, s, B.v[0][m], B.v[1][m], B.v[2][m], B.v[3][m]);
      else vmul3(u, s, B.v[0][m], B.v[1][m], B.v[2][m]);
    }
  } else {
#pragma unroll
    for (int n = 0; n < Q; ++n) {
      if constexpr (Q == 4) vmul4(u, s, B.v[n][0], B.v[n][1], B.v[n][2], B.v[n][3]);
      else vmul3(u, s, B.v[n][0], B.v[n][1], B.v[n][2]);
    }
  }
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
