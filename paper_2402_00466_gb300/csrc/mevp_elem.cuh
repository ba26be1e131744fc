// mevp_elem.cuh -- per-element arithmetic of the mEVP subcycle, templated on
// the working precision T (double for the FP64 path, float for the mixed
// path).  All reference-element constants come from mevp_ref.cuh as
// compile-time values, so zero entries vanish and unit entries become adds.
//
// On a rectangle hx x hy the inverse local mass matrix and the Jacobian
// weights cancel (orthogonal DG basis), so every stage reduces to the
// reference operators scaled by 1/hx, 1/hy:
//   strain      E = M^-1 int phi eps(v)               (rows dxi, deta)
//   stress      S <- (1-1/alpha) S + M^-1 int phi s_vp / alpha    (Listing 1)
//   divergence  f_j = -int sigma : grad phi_j          (rows gxi, geta)
//
// The viscous-plastic law is evaluated in invariant form.  With
// p = e11 + e22, Q = (e11 - e22)/e, G = 2 e12/e (e the ellipse ratio),
//   Delta^2 = Delta_min^2 + p^2 + Q^2 + G^2,
//   s11 = X (p + Q/e) - P/2,  s22 = X (p - Q/e) - P/2,  s12 = X G/e,
// with X = P/(2 Delta).  Expanding p, Q, G gives back exactly
// Delta^2 = Delta_min^2 + (1+1/e^2)(e11^2+e22^2) + 2(1-1/e^2) e11 e22
// + (4/e^2) e12^2 and the coefficients 5/8, 3/8, 1/4 of Listing 1 at e = 2.
// The isotropic -P/2 term projects onto the constant DG function only.
#pragma once

#include "mevp_internal.cuh"
#include "mevp_ref.cuh"

namespace mevp {

__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

// DG index of the basis function p_kx(xi) p_ky(eta), or -1 if not in the space.
template <int NS> __host__ __device__ constexpr int sidx(int kx, int ky) {
  return (kx == 0 && ky == 0) ? 0
       : (kx == 1 && ky == 0) ? 1
       : (kx == 0 && ky == 1) ? 2
       : (NS >= 6 && kx == 2 && ky == 0) ? 3
       : (NS >= 6 && kx == 1 && ky == 1) ? 4
       : (NS >= 6 && kx == 0 && ky == 2) ? 5
       : (NS == 8 && kx == 2 && ky == 1) ? 6
       : (NS == 8 && kx == 1 && ky == 2) ? 7
                                         : -1;
}

template <typename T>
__device__ __forceinline__ T cmul_acc(double c, T x, T acc) {
  // acc + c*x with c a compile-time constant (1 folds to an add)
  return c == 1.0 ? acc + x : (c == -1.0 ? acc - x : fma((T)c, x, acc));
}

// Projected reference derivatives of the 9 nodal values w:
// Wxi[s] = sum_j dxi(s,j) w_j, Weta[s] = sum_j deta(s,j) w_j.
template <int NS, typename T>
__device__ __forceinline__ void ref_derivs(const T w[9], T Wxi[NS], T Weta[NS]) {
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    T a = T(-0.0), b = T(-0.0);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const double cx = dxi(s, j), ce = deta(s, j);
      if (cx != 0.0) a = cmul_acc(cx, w[j], a);
      if (ce != 0.0) b = cmul_acc(ce, w[j], b);
    }
    Wxi[s] = a;
    Weta[s] = b;
  }
}

// Strain invariants (DG coefficients) from the nodal velocities:
// p = E11 + E22, Q = (E11 - E22)/e, G = 2 E12/e.
template <int NS, typename T>
__device__ __forceinline__ void strain_invariants(const T u[9], const T v[9], T ihx, T ihy,
                                                  T ie, T Pc[NS], T Qc[NS], T Gc[NS]) {
  T Uxi[NS], Ueta[NS], Vxi[NS], Veta[NS];
  ref_derivs<NS>(u, Uxi, Ueta);
  ref_derivs<NS>(v, Vxi, Veta);
  const T cxe = ihx * ie, cye = ihy * ie;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    Pc[s] = fma(ihx, Uxi[s], ihy * Veta[s]);
    Qc[s] = fma(cxe, Uxi[s], -(cye * Veta[s]));
    Gc[s] = fma(cye, Ueta[s], cxe * Vxi[s]);
  }
}

// Sum-factorised evaluation of a DG field at the NGP x NGP Gauss points
// (g = gx + NGP*gy): c_kx(gy) = sum_ky F(kx,ky) p_ky(gy), then
// f(gx,gy) = sum_kx p_kx(gx) c_kx(gy).
template <int NS, typename T>
__device__ __forceinline__ void gauss_eval(const T F[NS], T out[DgSpace<NS>::NGP * DgSpace<NS>::NGP]) {
  constexpr int N = DgSpace<NS>::NGP;
  T c[3][N];
#pragma unroll
  for (int kx = 0; kx < 3; ++kx)
#pragma unroll
    for (int gy = 0; gy < N; ++gy) {
      T acc = T(-0.0);
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const int s = sidx<NS>(kx, ky);
        if (s < 0) continue;
        const double pv = pg<N>(ky, gy);
        if (pv != 0.0) acc = cmul_acc(pv, F[s], acc);
      }
      c[kx][gy] = acc;
    }
#pragma unroll
  for (int gy = 0; gy < N; ++gy)
#pragma unroll
    for (int gx = 0; gx < N; ++gx) {
      T acc = T(-0.0);
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        if (sidx<NS>(kx, 0) < 0) continue;
        const double pv = pg<N>(kx, gx);
        if (pv != 0.0) acc = cmul_acc(pv, c[kx][gy], acc);
      }
      out[gx + N * gy] = acc;
    }
}

// Relaxed stress update from the strain invariants (coefficients) and the
// ice strength: Ph = P/(2 alpha) per element (DG0 H, A; VAR = false) or
// Phg[g] per Gauss point (DG1/DG2 H, A; VAR = true), fac = 1 - 1/alpha,
// ie = 1/e.  With a constant P the isotropic -P/2 term projects onto the
// constant DG function alone; a varying one is projected with the rest.
template <int NS, bool VAR, typename T>
__device__ __forceinline__ void relax_stress_p(T S11[NS], T S12[NS], T S22[NS], const T Pc[NS],
                                               const T Qc[NS], const T Gc[NS], T Ph,
                                               const T *Phg, T dmin2, T fac, T ie) {
  constexpr int NG = DgSpace<NS>::NGP * DgSpace<NS>::NGP;
  T pgv[NG], qgv[NG], ggv[NG];
  gauss_eval<NS>(Pc, pgv);
  gauss_eval<NS>(Qc, qgv);
  gauss_eval<NS>(Gc, ggv);
  T Ap[NS], AQ[NS], AG[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) Ap[s] = AQ[s] = AG[s] = T(-0.0);
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const T d2 = fma(ggv[g], ggv[g], fma(qgv[g], qgv[g], fma(pgv[g], pgv[g], dmin2)));
    const T Pg = VAR ? Phg[g] : Ph;
    const T X = Pg * rsqrt_t(d2);
    const T xp = VAR ? fma(X, pgv[g], -Pg) : X * pgv[g];
    const T xq = X * qgv[g], xg = X * ggv[g];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const double w = proj<NS>(s, g);
      if (w != 0.0) {
        Ap[s] = fma((T)w, xp, Ap[s]);
        AQ[s] = fma((T)w, xq, AQ[s]);
        AG[s] = fma((T)w, xg, AG[s]);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const T base = (!VAR && s == 0) ? Ap[s] - Ph : Ap[s];
    const T q = ie * AQ[s];
    S11[s] = fma(fac, S11[s], base + q);
    S22[s] = fma(fac, S22[s], base - q);
    S12[s] = fma(fac, S12[s], ie * AG[s]);
  }
}

template <int NS, typename T>
__device__ __forceinline__ void relax_stress(T S11[NS], T S12[NS], T S22[NS], const T Pc[NS],
                                             const T Qc[NS], const T Gc[NS], T Ph, T dmin2,
                                             T fac, T ie) {
  relax_stress_p<NS, false, T>(S11, S12, S22, Pc, Qc, Gc, Ph, nullptr, dmin2, fac, ie);
}

// Element forces f_j = -int sigma : grad phi_j on a rectangle hx x hy
// (fx[j], fy[j] for the 9 local Q2 nodes).
template <int NS, typename T>
__device__ __forceinline__ void element_forces_t(const T S11[NS], const T S12[NS],
                                                 const T S22[NS], T hx, T hy, T fx[9], T fy[9]) {
  T a11[NS], a12x[NS], a12y[NS], a22[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    a11[s] = -hy * S11[s];
    a12x[s] = -hx * S12[s];
    a12y[s] = -hy * S12[s];
    a22[s] = -hx * S22[s];
  }
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    T x = T(-0.0), y = T(-0.0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const double gx = gxi(j, s), ge = geta(j, s);
      if (gx != 0.0) {
        x = cmul_acc(gx, a11[s], x);
        y = cmul_acc(gx, a12y[s], y);
      }
      if (ge != 0.0) {
        x = cmul_acc(ge, a12x[s], x);
        y = cmul_acc(ge, a22[s], y);
      }
    }
    fx[j] = x;
    fy[j] = y;
  }
}

}  // namespace mevp
