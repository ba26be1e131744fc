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

// Projected reference derivatives of the 9 nodal values w (j = a + 3b):
// Wxi[s] = sum_j dxi(s,j) w_j, Weta[s] = sum_j deta(s,j) w_j.  Both operators
// are products of 1-D moments, dxi(s,j) = idr(kx,a) ib(ky,b) / mass_s with
// (kx, ky) the degrees of DG function s, so they are applied in two 1-D
// passes (sum factorisation): the derivative moments along the
// differentiated direction, then the value moments along the other one.
template <int NS, typename T>
__device__ __forceinline__ void ref_derivs(const T w[9], T Wxi[NS], T Weta[NS]) {
  // dx[k][b] = sum_a idr(k,a) w(a,b),  de[k][a] = sum_b idr(k,b) w(a,b);
  // idr(2, .) = 0 (the derivative of a Q2 function is linear)
  T dx[2][3], de[2][3];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T x = T(-0.0), y = T(-0.0);
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const double c = idr(k, t);
        if (c != 0.0) {
          x = cmul_acc(c, w[t + 3 * i], x);
          y = cmul_acc(c, w[i + 3 * t], y);
        }
      }
      dx[k][i] = x;
      de[k][i] = y;
    }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    constexpr int K2 = 2;
    const int kx = dgx(s), ky = dgy(s);
    T x = T(-0.0), y = T(-0.0);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      if (kx < K2) {
        const double c = ib(ky, t) / dgmass(s);
        if (c != 0.0) x = cmul_acc(c, dx[kx < K2 ? kx : 0][t], x);
      }
      if (ky < K2) {
        const double c = ib(kx, t) / dgmass(s);
        if (c != 0.0) y = cmul_acc(c, de[ky < K2 ? ky : 0][t], y);
      }
    }
    Wxi[s] = x;
    Weta[s] = y;
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
// (fx[j], fy[j] for the 9 local Q2 nodes j = a + 3b).  The moments
// gxi(j,s) = idr(kx,a) ib(ky,b) and geta(j,s) = ib(kx,a) idr(ky,b) are
// products of 1-D moments, so the sums over the DG functions are taken in
// two passes (sum factorisation): along the undifferentiated direction
// first, then the derivative moments along the differentiated one.
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
  // X*[k][b] = sum over the DG functions of degree k in xi of ib(ky_s, b) a*_s
  // (xi-derivative terms); Y*[k][a] = sum over degree k in eta of
  // ib(kx_s, a) a*_s (eta-derivative terms); k < 2 (idr(2, .) = 0)
  T X11[2][3], X12[2][3], Y12[2][3], Y22[2][3];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T p = T(-0.0), q = T(-0.0), r = T(-0.0), u = T(-0.0);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (dgx(s) == k) {
          const double c = ib(dgy(s), i);
          if (c != 0.0) {
            p = cmul_acc(c, a11[s], p);
            q = cmul_acc(c, a12y[s], q);
          }
        }
        if (dgy(s) == k) {
          const double c = ib(dgx(s), i);
          if (c != 0.0) {
            r = cmul_acc(c, a12x[s], r);
            u = cmul_acc(c, a22[s], u);
          }
        }
      }
      X11[k][i] = p;
      X12[k][i] = q;
      Y12[k][i] = r;
      Y22[k][i] = u;
    }
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T x = T(-0.0), y = T(-0.0);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const double cx = idr(k, a), ce = idr(k, b);
        if (cx != 0.0) {
          x = cmul_acc(cx, X11[k][b], x);
          y = cmul_acc(cx, X12[k][b], y);
        }
        if (ce != 0.0) {
          x = cmul_acc(ce, Y12[k][a], x);
          y = cmul_acc(ce, Y22[k][a], y);
        }
      }
      fx[a + 3 * b] = x;
      fy[a + 3 * b] = y;
    }
}

}  // namespace mevp
