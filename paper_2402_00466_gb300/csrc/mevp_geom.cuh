// mevp_geom.cuh -- per-element arithmetic of the FP64 subcycle on general
// (non-affine) quadrilateral meshes.
//
// Every element is the image of the reference square under the bilinear (Q1)
// map of its four vertices, evaluated on the fly at the Gauss points (the
// paper's "on-the-fly map", Sec. 3.2; the map from 4 vertices with 2 values
// each).  In centred coordinates xh = xi - 1/2, eh = eta - 1/2 the map is
//   x(xh, eh) = x_c + A xh + B eh + c xh eh,
//   A = (bottom + top edge)/2, B = (left + right edge)/2,
//   c = top edge - bottom edge,
// so the Jacobian columns are dx/dxi = A + c eh and dx/deta = B + c xh, and
// det J = d0 + d1 xh + d2 eh is affine in the reference coordinates.
//
// With that:
//   * strain: the L2 projection E = M^-1 int psi eps(v) detJ.  detJ cancels
//     against the inverse Jacobian inside the integrand, e.g.
//     detJ du/dx = J11 du/dxi - J10 du/deta, so no division is needed;
//   * stress: S <- (1-1/alpha) S + M^-1 int psi detJ s_vp / alpha (Listing 1
//     with the element's own iMJwPSI, factored rather than stored);
//   * divergence: f_j = -int sigma : grad phi_j detJ, where detJ again
//     cancels: f_x = -sum_g w_g [(s11 J11 - s12 J01) dphi/dxi
//                              + (s12 J00 - s11 J10) dphi/deta];
//   * the local DG mass matrix M = d0 diag(mass) + d1 MX + d2 MY uses the
//     exact moment tables of mevp_ref.cuh (the Gauss rule of App. A
//     integrates these products exactly) and is factored as L D L^T per
//     element.
// Every sum over Gauss points is sum-factorised along the two directions.
#pragma once

#include "mevp_elem.cuh"
#include "mevp_internal.cuh"
#include "mevp_ref.cuh"

namespace mevp {

// The 9 values of a CG2 nodal field f[0, nn) on element (kx, ky), local node
// a + 3b (flags, nn: bounds checks of checked builds).
__device__ __forceinline__ void gather9(const double *__restrict__ f, int nw, int kx, int ky,
                                        double out[9], int *flags, long long nn) {
  const long long base = (long long)(2 * ky) * nw + 2 * kx;
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a)
      out[a + 3 * b] = ck_ldg(flags, f, base + (long long)b * nw + a, nn, 102);
}

// Centred bilinear map of one element, in working precision T.
template <typename T> struct QuadMapT {
  T Ax, Ay, Bx, By, cx, cy;
  // det J = d0 + d1 xh + d2 eh
  __device__ __forceinline__ T d0() const { return fma(Ax, By, -(Bx * Ay)); }
  __device__ __forceinline__ T d1() const { return fma(Ax, cy, -(cx * Ay)); }
  __device__ __forceinline__ T d2() const { return fma(cx, By, -(Bx * cy)); }
};
using QuadMap = QuadMapT<double>;

__device__ __forceinline__ QuadMap quad_map(const double2 *__restrict__ xy, int nx, int kx,
                                            int ky, int *flags = nullptr, long long nv = 0) {
  const long long vw = (long long)nx + 1;
#ifdef MEVP_CHECKED
  const double2 p00 = ck_ld(flags, xy, ky * vw + kx, nv, 141);
  const double2 p10 = ck_ld(flags, xy, ky * vw + kx + 1, nv, 141);
  const double2 p01 = ck_ld(flags, xy, (ky + 1) * vw + kx, nv, 141);
  const double2 p11 = ck_ld(flags, xy, (ky + 1) * vw + kx + 1, nv, 141);
#else
  (void)flags; (void)nv;
  const double2 p00 = xy[ky * vw + kx], p10 = xy[ky * vw + kx + 1];
  const double2 p01 = xy[(ky + 1) * vw + kx], p11 = xy[(ky + 1) * vw + kx + 1];
#endif
  const double bx = p10.x - p00.x, by = p10.y - p00.y;  // bottom edge
  const double tx = p11.x - p01.x, ty = p11.y - p01.y;  // top edge
  const double lx = p01.x - p00.x, ly = p01.y - p00.y;  // left edge
  const double rx = p11.x - p10.x, ry = p11.y - p10.y;  // right edge
  QuadMap m;
  m.Ax = 0.5 * (bx + tx);
  m.Ay = 0.5 * (by + ty);
  m.Bx = 0.5 * (lx + rx);
  m.By = 0.5 * (ly + ry);
  m.cx = tx - bx;
  m.cy = ty - by;
  return m;
}

// Jacobian entries at 2-D Gauss point (gx, gy) of an NGP rule.
template <int N, typename T>
__device__ __forceinline__ void jac_at(const QuadMapT<T> &m, int gx, int gy, T &j00, T &j01,
                                       T &j10, T &j11) {
  const double xh = Gauss<N>::xh(gx), eh = Gauss<N>::xh(gy);
  j00 = eh == 0.0 ? m.Ax : fma(m.cx, (T)eh, m.Ax);
  j10 = eh == 0.0 ? m.Ay : fma(m.cy, (T)eh, m.Ay);
  j01 = xh == 0.0 ? m.Bx : fma(m.cx, (T)xh, m.Bx);
  j11 = xh == 0.0 ? m.By : fma(m.cy, (T)xh, m.By);
}

// Isoparametric (Q2) element: the element map is the CG2 interpolant of the
// element's 9 node positions (Sec. 2.1: the map from the velocity's space).
// Its Jacobian at the N x N Gauss points is formed once per element and kept
// in shared memory, one column per thread: entry q (J00, J01, J10, J11) of
// point g at sJ[(q * N * N + g) * stride].
template <int N, typename T> struct IsoGeo {
  const T *sJ;
  int stride;
};

template <int N, typename T>
__device__ __forceinline__ void jac_at(const IsoGeo<N, T> &m, int gx, int gy, T &j00, T &j01,
                                       T &j10, T &j11) {
  const int g = gx + N * gy, NG = N * N;
  j00 = m.sJ[(0 * NG + g) * m.stride];
  j01 = m.sJ[(1 * NG + g) * m.stride];
  j10 = m.sJ[(2 * NG + g) * m.stride];
  j11 = m.sJ[(3 * NG + g) * m.stride];
}

// The same Jacobians read from per-element records in global memory:
// entry q of point g of element K at J[(q * N * N + g) * ne] (J = base + K).
template <int N, typename T> struct IsoGeoG {
  const T *__restrict__ J;
  size_t ne;
};

// A read-only load that the compiler may not merge with an earlier one of
// the same address: each stage re-reads J (an L1 hit) instead of keeping all
// 4 N^2 values live in registers between the stages.
__device__ __forceinline__ double ld_nc_fresh(const double *p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

template <int N>
__device__ __forceinline__ void jac_at(const IsoGeoG<N, double> &m, int gx, int gy, double &j00,
                                       double &j01, double &j10, double &j11) {
  const int g = gx + N * gy, NG = N * N;
  j00 = ld_nc_fresh(m.J + (size_t)(0 * NG + g) * m.ne);
  j01 = ld_nc_fresh(m.J + (size_t)(1 * NG + g) * m.ne);
  j10 = ld_nc_fresh(m.J + (size_t)(2 * NG + g) * m.ne);
  j11 = ld_nc_fresh(m.J + (size_t)(3 * NG + g) * m.ne);
}

// Reference gradients (d/dxi, d/deta) of a Q2 field at the N x N Gauss
// points, sum-factorised: row sums along xi, then columns along eta.
template <int N, typename T>
__device__ __forceinline__ void ref_grad_gauss(const T w[9], T gxi[N * N], T geta[N * N]) {
  T rd[3][N], r0[3][N];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int gx = 0; gx < N; ++gx) {
      T a1 = T(-0.0), a0 = T(-0.0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double cd = dlq<N>(a, gx), c0 = lq<N>(a, gx);
        if (cd != 0.0) a1 = cmul_acc(cd, w[a + 3 * b], a1);
        if (c0 != 0.0) a0 = cmul_acc(c0, w[a + 3 * b], a0);
      }
      rd[b][gx] = a1;
      r0[b][gx] = a0;
    }
#pragma unroll
  for (int gy = 0; gy < N; ++gy)
#pragma unroll
    for (int gx = 0; gx < N; ++gx) {
      T s1 = T(-0.0), s2 = T(-0.0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const double c0 = lq<N>(b, gy), cd = dlq<N>(b, gy);
        if (c0 != 0.0) s1 = cmul_acc(c0, rd[b][gx], s1);
        if (cd != 0.0) s2 = cmul_acc(cd, r0[b][gx], s2);
      }
      gxi[gx + N * gy] = s1;
      geta[gx + N * gy] = s2;
    }
}

// Moments R_s = sum_g w_g psi_s(g) D_g of Gauss-point values D (no mass
// scaling), sum-factorised.
template <int NS, typename T>
__device__ __forceinline__ void gauss_moments(const T D[DgSpace<NS>::NGP * DgSpace<NS>::NGP],
                                              T R[NS]) {
  constexpr int N = DgSpace<NS>::NGP;
  T t[3][N];
#pragma unroll
  for (int kx = 0; kx < 3; ++kx)
#pragma unroll
    for (int gy = 0; gy < N; ++gy) {
      T acc = T(-0.0);
      if (sidx<NS>(kx, 0) >= 0) {
#pragma unroll
        for (int gx = 0; gx < N; ++gx) {
          const double c = Gauss<N>::w(gx) * pg<N>(kx, gx);
          if (c != 0.0) acc = cmul_acc(c, D[gx + N * gy], acc);
        }
      }
      t[kx][gy] = acc;
    }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    T acc = T(-0.0);
#pragma unroll
    for (int gy = 0; gy < N; ++gy) {
      const double c = Gauss<N>::w(gy) * pg<N>(dgy(s), gy);
      if (c != 0.0) acc = cmul_acc(c, t[dgx(s)][gy], acc);
    }
    R[s] = acc;
  }
}

// L D L^T factor of the local DG mass matrix of a bilinear element: the
// strict lower triangle of L, row by row (L(i,k) at i(i-1)/2 + k; the unit
// diagonal is implicit), and 1/D.
template <int NS, typename T = double> struct MassFactor {
  T L[NS * (NS - 1) / 2];
  T Dinv[NS];
  __device__ __forceinline__ T &at(int i, int k) { return L[i * (i - 1) / 2 + k]; }
  __device__ __forceinline__ T at(int i, int k) const { return L[i * (i - 1) / 2 + k]; }
};

// L D L^T of a symmetric positive definite NS x NS matrix given by the
// functor Mij(i, j) (i >= j).
template <int NS, typename T, typename MF>
__device__ __forceinline__ void ldl_factor(const MF &Mij, MassFactor<NS, T> &F) {
  T D[NS];
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    T dj = Mij(j, j);
#pragma unroll
    for (int k = 0; k < j; ++k) dj = fma(-F.at(j, k) * D[k], F.at(j, k), dj);
    D[j] = dj;
    F.Dinv[j] = T(1) / dj;
#pragma unroll
    for (int i = j + 1; i < NS; ++i) {
      T a = Mij(i, j);
#pragma unroll
      for (int k = 0; k < j; ++k) a = fma(-F.at(i, k) * D[k], F.at(j, k), a);
      F.at(i, j) = a * F.Dinv[j];
    }
  }
}

// Bilinear element: M = d0 diag(mass) + d1 MX + d2 MY with the exact moments.
template <int NS, typename T>
__device__ __forceinline__ void mass_factor(const QuadMapT<T> &m, MassFactor<NS, T> &F) {
  const T d0 = m.d0(), d1 = m.d1(), d2 = m.d2();
  ldl_factor<NS, T>(
      [&](int i, int j) -> T {
        if (i == j) return d0 * (T)dgmass(j);
        T a = T(0);
        if (mx(i, j) != 0.0) a = d1 * (T)mx(i, j);
        if (my(i, j) != 0.0) a = fma(d2, (T)my(i, j), a);
        return a;
      },
      F);
}

// Isoparametric element: M = sum_g w_g det J_g psi psi^T with the Gauss rule
// of the stress space (the map makes det J rational-free but of higher
// degree, so the rule is the method's own, as in the paper's iMJwPSI).
template <int NS, typename T>
__device__ __forceinline__ void mass_factor(const IsoGeo<DgSpace<NS>::NGP, T> &m,
                                            MassFactor<NS, T> &F) {
  constexpr int N = DgSpace<NS>::NGP, NG = N * N;
  T wd[NG];
#pragma unroll
  for (int gy = 0; gy < N; ++gy)
#pragma unroll
    for (int gx = 0; gx < N; ++gx) {
      T j00, j01, j10, j11;
      jac_at<N>(m, gx, gy, j00, j01, j10, j11);
      wd[gx + N * gy] = (T)(Gauss<N>::w(gx) * Gauss<N>::w(gy)) * fma(j00, j11, -(j01 * j10));
    }
  ldl_factor<NS, T>(
      [&](int i, int j) -> T {
        T a = T(-0.0);
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          const double c = psi<NS>(i, g) * psi<NS>(j, g);
          if (c != 0.0) a = cmul_acc(c, wd[g], a);
        }
        return a;
      },
      F);
}

// A factor in a [NS (NS + 1) / 2][ne] array of element records: L row by
// row, then 1/D (SoA, entry i of element K at f[i * ne + K]).
template <int NS> constexpr int mass_factor_words() { return NS * (NS + 1) / 2; }

// x <- M^-1 x with the factor above.
template <int NS, typename T>
__device__ __forceinline__ void mass_solve(const MassFactor<NS, T> &F, T x[NS]) {
#pragma unroll
  for (int i = 1; i < NS; ++i)
#pragma unroll
    for (int k = 0; k < i; ++k) x[i] = fma(-F.at(i, k), x[k], x[i]);
#pragma unroll
  for (int i = 0; i < NS; ++i) x[i] *= F.Dinv[i];
#pragma unroll
  for (int ii = 0; ii < NS - 1; ++ii) {
    const int i = NS - 2 - ii;
#pragma unroll
    for (int k = i + 1; k < NS; ++k) x[i] = fma(-F.at(k, i), x[k], x[i]);
  }
}

// Strain of the nodal velocities u, v as DG coefficients:
// E11 = M^-1 int psi du/dx, E22 = M^-1 int psi dv/dy,
// Esh = M^-1 int psi (du/dy + dv/dx)  (= 2 E12).
template <int NS, typename G, typename T>
__device__ __forceinline__ void strain_general(const G &m, const MassFactor<NS, T> &F,
                                               const T u[9], const T v[9], T E11[NS], T E22[NS],
                                               T Esh[NS]) {
  constexpr int N = DgSpace<NS>::NGP, NG = N * N;
  T D11[NG], D22[NG], Dsh[NG];
  {
    T uxi[NG], ueta[NG], vxi[NG], veta[NG];
    ref_grad_gauss<N>(u, uxi, ueta);
    ref_grad_gauss<N>(v, vxi, veta);
#pragma unroll
    for (int gy = 0; gy < N; ++gy)
#pragma unroll
      for (int gx = 0; gx < N; ++gx) {
        const int g = gx + N * gy;
        T j00, j01, j10, j11;
        jac_at<N>(m, gx, gy, j00, j01, j10, j11);
        D11[g] = fma(j11, uxi[g], -(j10 * ueta[g]));  // detJ du/dx
        D22[g] = fma(j00, veta[g], -(j01 * vxi[g]));  // detJ dv/dy
        const T duy = fma(j00, ueta[g], -(j01 * uxi[g]));
        const T dvx = fma(j11, vxi[g], -(j10 * veta[g]));
        Dsh[g] = duy + dvx;
      }
  }
  gauss_moments<NS>(D11, E11);
  gauss_moments<NS>(D22, E22);
  gauss_moments<NS>(Dsh, Esh);
  mass_solve<NS>(F, E11);
  mass_solve<NS>(F, E22);
  mass_solve<NS>(F, Esh);
}

// Relaxed stress update on a general element from the strain coefficients:
// S <- fac S + M^-1 int psi detJ (X (p +- Q/e), X G/e) - Ph e_0, with
// X = Ph / sqrt(Delta^2), Ph = P/(2 alpha) (invariant form of Listing 1).
// VAR: per-Gauss-point strength Phg (DG1/DG2 H, A), whose -P/2 term is
// projected with the rest; otherwise the element constant Ph.
template <int NS, bool VAR = false, typename T = double, typename G>
__device__ __forceinline__ void relax_general(const G &m, const MassFactor<NS, T> &F,
                                              T S11[NS], T S12[NS], T S22[NS], const T Pc[NS],
                                              const T Qc[NS], const T Gc[NS], T Ph, T dmin2,
                                              T fac, T ie, const T *Phg = nullptr) {
  constexpr int N = DgSpace<NS>::NGP, NG = N * N;
  T RP[NS], RQ[NS], RG[NS];
  {
    T pgv[NG], qgv[NG], ggv[NG];
    gauss_eval<NS>(Pc, pgv);
    gauss_eval<NS>(Qc, qgv);
    gauss_eval<NS>(Gc, ggv);
#pragma unroll
    for (int gy = 0; gy < N; ++gy)
#pragma unroll
      for (int gx = 0; gx < N; ++gx) {
        const int g = gx + N * gy;
        T j00, j01, j10, j11;
        jac_at<N>(m, gx, gy, j00, j01, j10, j11);
        const T det = fma(j00, j11, -(j01 * j10));
        const T d2 = fma(ggv[g], ggv[g], fma(qgv[g], qgv[g], fma(pgv[g], pgv[g], dmin2)));
        const T Pg = VAR ? Phg[g] : Ph;
        const T Xd = Pg * rsqrt_t(d2) * det;
        pgv[g] = VAR ? fma(Xd, pgv[g], -(Pg * det)) : pgv[g] * Xd;
        qgv[g] *= Xd;
        ggv[g] *= Xd;
      }
    gauss_moments<NS>(pgv, RP);
    gauss_moments<NS>(qgv, RQ);
    gauss_moments<NS>(ggv, RG);
  }
  mass_solve<NS>(F, RP);
  mass_solve<NS>(F, RQ);
  mass_solve<NS>(F, RG);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const T base = (!VAR && s == 0) ? RP[s] - Ph : RP[s];
    const T q = ie * RQ[s];
    S11[s] = fma(fac, S11[s], base + q);
    S22[s] = fma(fac, S22[s], base - q);
    S12[s] = fma(fac, S12[s], ie * RG[s]);
  }
}

// Element forces f_j = -int sigma : grad phi_j of a DG stress on a general
// element (fx[j], fy[j] for the 9 local Q2 nodes, j = a + 3b).
template <int NS, typename G, typename T>
__device__ __forceinline__ void forces_general(const G &m, const T S11[NS],
                                               const T S12[NS], const T S22[NS], T fx[9],
                                               T fy[9]) {
  constexpr int N = DgSpace<NS>::NGP, NG = N * N;
  T ax[NG], bx[NG], ay[NG], by[NG];
  {
    T s11[NG], s12[NG], s22[NG];
    gauss_eval<NS>(S11, s11);
    gauss_eval<NS>(S12, s12);
    gauss_eval<NS>(S22, s22);
#pragma unroll
    for (int gy = 0; gy < N; ++gy)
#pragma unroll
      for (int gx = 0; gx < N; ++gx) {
        const int g = gx + N * gy;
        T j00, j01, j10, j11;
        jac_at<N>(m, gx, gy, j00, j01, j10, j11);
        const T w = (T)(Gauss<N>::w(gx) * Gauss<N>::w(gy));
        ax[g] = w * fma(s11[g], j11, -(s12[g] * j01));
        bx[g] = w * fma(s12[g], j00, -(s11[g] * j10));
        ay[g] = w * fma(s12[g], j11, -(s22[g] * j01));
        by[g] = w * fma(s22[g], j00, -(s12[g] * j10));
      }
  }
  // f_ab = -sum_gx [dL_a(gx) sum_gy L_b(gy) a_g + L_a(gx) sum_gy dL_b(gy) b_g]
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    T tax[N], tbx[N], tay[N], tby[N];
#pragma unroll
    for (int gx = 0; gx < N; ++gx) {
      T p = T(-0.0), q = T(-0.0), r = T(-0.0), t = T(-0.0);
#pragma unroll
      for (int gy = 0; gy < N; ++gy) {
        const double c0 = lq<N>(b, gy), cd = dlq<N>(b, gy);
        const int g = gx + N * gy;
        if (c0 != 0.0) {
          p = cmul_acc(c0, ax[g], p);
          r = cmul_acc(c0, ay[g], r);
        }
        if (cd != 0.0) {
          q = cmul_acc(cd, bx[g], q);
          t = cmul_acc(cd, by[g], t);
        }
      }
      tax[gx] = p;
      tbx[gx] = q;
      tay[gx] = r;
      tby[gx] = t;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T x = T(-0.0), y = T(-0.0);
#pragma unroll
      for (int gx = 0; gx < N; ++gx) {
        const double cd = dlq<N>(a, gx), c0 = lq<N>(a, gx);
        if (cd != 0.0) {
          x = cmul_acc(cd, tax[gx], x);
          y = cmul_acc(cd, tay[gx], y);
        }
        if (c0 != 0.0) {
          x = cmul_acc(c0, tbx[gx], x);
          y = cmul_acc(c0, tby[gx], y);
        }
      }
      fx[a + 3 * b] = -x;
      fy[a + 3 * b] = -y;
    }
  }
}

// int_K phi_j for local node (a, b): d0 W_a W_b + d1 X_a W_b + d2 W_a X_b
// with W the Simpson weights and X_a = int xh L_a (exact for the affine det).
__device__ __forceinline__ double node_area_general(const QuadMap &m, int a, int b) {
  return fma(m.d0(), q2w(a) * q2w(b), fma(m.d1(), q2xw(a) * q2w(b), m.d2() * (q2w(a) * q2xw(b))));
}

}  // namespace mevp
