// mevp_ref.cuh -- compile-time reference-element tables of the CUDA path.
//
// Everything the kernels need about the reference square [0,1]^2, derived
// analytically so that every table entry is a compile-time constant the
// compiler can fold (zeros vanish, ones become plain adds):
//
//   * DG stress basis (Sec. 2.1: stress in the gradient space of the CG2
//     velocity, tensor-valued DG): products p_kx(xi) p_ky(eta) of the centred
//     Legendre functions p0 = 1, p1 = t - 1/2, p2 = (t - 1/2)^2 - 1/12, total
//     degree <= 1 (3 dofs) or <= 2 (6 dofs), or degree <= 2 in each
//     variable without the biquadratic product (8 dofs, App. A), in the order
//     (0,0) (1,0) (0,1) (2,0) (1,1) (0,2) (2,1) (1,2).  Orthogonal, so on
//     rectangles the local mass matrix is diagonal: int p_k^2 = 1, 1/12, 1/180.
//   * CG2 velocity basis: Q2 Lagrange L_a(xi) L_b(eta), nodes {0, 1/2, 1},
//     local node j = a + 3b, with L0 = (1-t)(1-2t), L1 = 4t(1-t), L2 = t(2t-1).
//   * Exact 1-D moments  IB[k][b] = int_0^1 p_k L_b,  ID[k][a] = int_0^1 p_k L_a'.
//     With them the L2 projection of a reference derivative of a Q2 field
//     onto the DG space, and the weak divergence of a DG field tested with
//     Q2, are exact rational matrices (no quadrature needed: the Gauss rule
//     of App. A integrates these polynomial products exactly).
//   * Gauss-Legendre rules (App. A: 2x2 points for 3 dofs, 3x3 for 6 and 8) with
//     closed-form points 1/2 -+ 1/(2 sqrt 3) and 1/2, 1/2 -+ sqrt(15)/10.
#pragma once

namespace mevp {

// ---- 1-D moments (exact rationals) -------------------------------------
__host__ __device__ constexpr double ib(int k, int b) {
  // int p_k L_b : k = 0: (1/6, 2/3, 1/6); k = 1: (-1/12, 0, 1/12); k = 2: (1/90, -1/45, 1/90)
  return k == 0 ? (b == 1 ? 2.0 / 3.0 : 1.0 / 6.0)
       : k == 1 ? (b == 0 ? -1.0 / 12.0 : b == 1 ? 0.0 : 1.0 / 12.0)
                : (b == 1 ? -1.0 / 45.0 : 1.0 / 90.0);
}
__host__ __device__ constexpr double idr(int k, int a) {
  // int p_k L_a' : k = 0: (-1, 0, 1); k = 1: (1/3, -2/3, 1/3); k = 2: 0 (L_a' is linear)
  return k == 0 ? (a == 0 ? -1.0 : a == 1 ? 0.0 : 1.0)
       : k == 1 ? (a == 1 ? -2.0 / 3.0 : 1.0 / 3.0)
                : 0.0;
}
__host__ __device__ constexpr double pnorm(int k) {
  return k == 0 ? 1.0 : k == 1 ? 1.0 / 12.0 : 1.0 / 180.0;
}

// ---- DG index -> 1-D degrees --------------------------------------------
__host__ __device__ constexpr int dgx(int s) {
  return s == 1 ? 1 : s == 3 ? 2 : s == 4 ? 1 : s == 6 ? 2 : s == 7 ? 1 : 0;
}
__host__ __device__ constexpr int dgy(int s) {
  return s == 2 ? 1 : s == 4 ? 1 : s == 5 ? 2 : s == 6 ? 1 : s == 7 ? 2 : 0;
}
__host__ __device__ constexpr double dgmass(int s) { return pnorm(dgx(s)) * pnorm(dgy(s)); }

// ---- Gauss rules on [0,1] -----------------------------------------------
// 1/(2 sqrt 3) and sqrt(15)/10 to 21 significant digits.
constexpr double kG2 = 0.288675134594812882254;
constexpr double kG3 = 0.387298334620741688518;

template <int NGP> struct Gauss;
template <> struct Gauss<2> {
  // centred coordinates t - 1/2 and weights
  __host__ __device__ static constexpr double xh(int g) { return g == 0 ? -kG2 : kG2; }
  __host__ __device__ static constexpr double w(int) { return 0.5; }
};
template <> struct Gauss<3> {
  __host__ __device__ static constexpr double xh(int g) { return g == 0 ? -kG3 : g == 1 ? 0.0 : kG3; }
  __host__ __device__ static constexpr double w(int g) { return g == 1 ? 4.0 / 9.0 : 5.0 / 18.0; }
};

// centred Legendre p_k at 1-D Gauss point g (exact where possible: p2 = 1/15, -1/12)
template <int NGP> __host__ __device__ constexpr double pg(int k, int g) {
  return k == 0 ? 1.0
       : k == 1 ? Gauss<NGP>::xh(g)
       : (NGP == 3 ? (g == 1 ? -1.0 / 12.0 : 1.0 / 15.0) : 0.0 /* (1/12 - 1/12) */);
}

// Value at 2-D Gauss point (gx, gy) of the N-point rule of the DG1/DG2 field
// F ([na][ne]) of element K.
template <int N>
__device__ __forceinline__ double dg_at_gauss(const double *F, int na, size_t ne, int K, int gx,
                                              int gy) {
  double v = 0.0;
  for (int i = 0; i < na; ++i) v = fma(F[(size_t)i * ne + K], pg<N>(dgx(i), gx) * pg<N>(dgy(i), gy), v);
  return v;
}

template <int NS> struct DgSpace;
template <> struct DgSpace<3> { static constexpr int NGP = 2; };
template <> struct DgSpace<6> { static constexpr int NGP = 3; };
template <> struct DgSpace<8> { static constexpr int NGP = 3; };

// DG basis function s at 2-D Gauss point g = gx + NGP*gy
template <int NS> __host__ __device__ constexpr double psi(int s, int g) {
  constexpr int N = DgSpace<NS>::NGP;
  return pg<N>(dgx(s), g % N) * pg<N>(dgy(s), g / N);
}
// projection weight: w_g psi_s(g) / mass_s (the reference-square iMJwPSI;
// on a rectangle the Jacobian cancels between M^-1 and w detJ)
template <int NS> __host__ __device__ constexpr double proj(int s, int g) {
  constexpr int N = DgSpace<NS>::NGP;
  return Gauss<N>::w(g % N) * Gauss<N>::w(g / N) * psi<NS>(s, g) / dgmass(s);
}

// L2 projection onto DG of the reference derivatives of Q2 node function j
__host__ __device__ constexpr double dxi(int s, int j) {
  return idr(dgx(s), j % 3) * ib(dgy(s), j / 3) / dgmass(s);
}
__host__ __device__ constexpr double deta(int s, int j) {
  return ib(dgx(s), j % 3) * idr(dgy(s), j / 3) / dgmass(s);
}
// weak-divergence moments: int phi_s d(phi_j)/dxi and int phi_s d(phi_j)/deta
__host__ __device__ constexpr double gxi(int j, int s) {
  return idr(dgx(s), j % 3) * ib(dgy(s), j / 3);
}
__host__ __device__ constexpr double geta(int j, int s) {
  return ib(dgx(s), j % 3) * idr(dgy(s), j / 3);
}
// 1-D integral of the Q2 Lagrange functions: Simpson weights 1/6, 2/3, 1/6
__host__ __device__ constexpr double q2w(int a) { return a == 1 ? 2.0 / 3.0 : 1.0 / 6.0; }

// ---- general (bilinear) element maps -------------------------------------
// In centred coordinates x = t - 1/2 the Q2 Lagrange functions are
// L0 = 2x^2 - x, L1 = 1 - 4x^2, L2 = 2x^2 + x, with derivatives 4x - 1, -8x,
// 4x + 1.  Values at 1-D Gauss point g, using the exact x^2 of the rule
// (1/12 for 2 points; 3/20 and 0 for 3 points).
template <int NGP> __host__ __device__ constexpr double gsq(int g) {
  return NGP == 2 ? 1.0 / 12.0 : (g == 1 ? 0.0 : 3.0 / 20.0);
}
template <int NGP> __host__ __device__ constexpr double lq(int a, int g) {
  return a == 0 ? 2.0 * gsq<NGP>(g) - Gauss<NGP>::xh(g)
       : a == 1 ? 1.0 - 4.0 * gsq<NGP>(g)
                : 2.0 * gsq<NGP>(g) + Gauss<NGP>::xh(g);
}
template <int NGP> __host__ __device__ constexpr double dlq(int a, int g) {
  return a == 0 ? 4.0 * Gauss<NGP>::xh(g) - 1.0
       : a == 1 ? -8.0 * Gauss<NGP>::xh(g)
                : 4.0 * Gauss<NGP>::xh(g) + 1.0;
}
// First moments int x p_i p_j over [-1/2, 1/2]: x p0 = p1 and
// x p1 = p2 + p0/12 give 1/12 for (0,1) and 1/180 for (1,2); all others vanish.
__host__ __device__ constexpr double xmom(int i, int j) {
  return (i + j == 1) ? 1.0 / 12.0 : (i + j == 3 && i != 3 && j != 3) ? 1.0 / 180.0 : 0.0;
}
// int x L_a over [-1/2, 1/2]: -1/12, 0, 1/12
__host__ __device__ constexpr double q2xw(int a) {
  return a == 0 ? -1.0 / 12.0 : a == 1 ? 0.0 : 1.0 / 12.0;
}
// The Jacobian determinant of a bilinear map is affine in the centred
// coordinates, det = d0 + d1 xh + d2 eh, so the local DG mass matrix is
// M = d0 diag(mass_s) + d1 MX + d2 MY with the exact moment matrices
//   MX[s][t] = int xh psi_s psi_t,  MY[s][t] = int eh psi_s psi_t.
__host__ __device__ constexpr double mx(int s, int t) {
  return dgy(s) == dgy(t) ? xmom(dgx(s), dgx(t)) * pnorm(dgy(s)) : 0.0;
}
__host__ __device__ constexpr double my(int s, int t) {
  return dgx(s) == dgx(t) ? pnorm(dgx(s)) * xmom(dgy(s), dgy(t)) : 0.0;
}

}  // namespace mevp
