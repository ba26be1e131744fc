// mevp_adjoint.cu -- hand-written reverse mode of the FP64 mEVP subcycle.
//
// Objective: the kinetic energy after n subcycles, J = 1/2 sum_j m_j |v_j^n|^2,
// as a function of the per-element ice strength parameter P*_K and of the
// nodal wind stress tau_j (the outer step's initial state and the other
// parameters fixed).  The paper's conclusion (Sec. 5) points to automatic
// differentiation for hybrid ML models; this is the adjoint of the subcycle
// of Table 1, written out stage by stage:
//
//   velocity (node j):  (a + i b) v^p = r,  a = m(1+beta)/dt + c,
//                       c = l Cw rho_w |v_o - v^{p-1}|, r = m beta/dt v^{p-1} + q + F + c v_o,
//                       q = (m/dt) v^n + l tau
//     -> rbar = A^-T vbar^p, abar = -rbar.v^p, cbar = abar + rbar.v_o,
//        vbar^{p-1} += m beta/dt rbar - cbar l Cw rho_w (v_o - v)/|v_o - v|  (0 at v = v_o),
//        Fbar_j = rbar, qbar += rbar
//   divergence (element K): f = -int sigma : grad phi  ->  Sbar^p += F^T fbar
//   stress: S^p = (1 - 1/alpha) S^{p-1} + M^-1 int phi s_vp(v^{p-1}, P)/alpha
//     -> Sbar^{p-1} = (1 - 1/alpha) Sbar^p, and the viscous-plastic law
//        reversed at every Gauss point (X = P/(2 alpha Delta), Delta^-1/2 etc.)
//   strain: linear in v^{p-1}  ->  transposed reference operators
//
// On general (bilinear) and curved (isoparametric) elements the same stages
// run through the Gauss-point form of the forward kernels: the transposes of
// the Gauss evaluation, the weighted moments, the Q2 reference gradients and
// the mass solve (M_K is symmetric, so M_K^-T = M_K^-1), with the Jacobians
// and mass factors of the forward kernels.
//
// Since the stress update is affine in S, the reverse sweep needs only the
// velocities v^{p-1}, v^p of each subcycle; the Gauss-point quantities are
// recomputed from them.  Checkpoints (v, S) are kept every k subcycles and
// each segment's velocities are recomputed before it is reversed.  All sums
// over neighbours are gathers in a fixed order (no atomics), so the gradient
// is deterministic.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <vector>

#include "mevp_elem.cuh"
#include "mevp_geom.cuh"
#include "mevp_internal.cuh"
#include "mevp_ref.cuh"

namespace mevp {
namespace {

constexpr int kBlock = 256;

struct AdjBuf {
  double *vbar;    // [2][nn] adjoint of the velocity entering the current reverse step
  double *vdir;    // [2][nn] node-direct part of vbar^{p-1}
  double *Fbar;    // [2][nn] adjoint of the nodal forces
  double *qbar;    // [2][nn] accumulated adjoint of q
  double *Sbar;    // [3][ns][ne] adjoint of the stress (carried)
  double *ubar;    // [18][ne] element contributions to vbar^{p-1}
  double *Pbar;    // [ne] accumulated adjoint of the ice strength P
  double *area;    // [nn] lumped area l_j
  double *partial; // [blocks] reduction partials
  double *J;       // [1]
};

// ---- objective ---------------------------------------------------------------
// vbar^n = m v^n (interior nodes), J partials per block (fixed order)
__global__ void k_adj_seed(DevState d, AdjBuf b, const double *__restrict__ v) {
  __shared__ double red[kBlock];
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (node < d.nn) {
    const size_t nn = d.nn;
    const double m = d.mass[node];
    const double vx = v[node], vy = v[nn + node];
    e = 0.5 * m * (vx * vx + vy * vy);
    b.vbar[node] = m * vx;
    b.vbar[nn + node] = m * vy;
  }
  red[threadIdx.x] = e;
  __syncthreads();
  for (int w = kBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) b.partial[blockIdx.x] = red[0];
}

__global__ void k_adj_sum(AdjBuf b, int nparts) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < nparts; ++i) s += b.partial[i];
  b.J[0] = s;
}

// ---- node stage ----------------------------------------------------------------
// Complete vbar^p of node (ix, iy) = vdir + sum of the element contributions
// ubar (after the first reverse step), then the reverse of its velocity update.
__device__ __forceinline__ void gather_ubar(const DevState &d, const AdjBuf &b, int ix, int iy,
                                            double &gx, double &gy) {
  const int kx1 = (ix & 1) ? (ix >> 1) : (ix >> 1) - 1, kx2 = ix >> 1;
  const int ky1 = (iy & 1) ? (iy >> 1) : (iy >> 1) - 1, ky2 = iy >> 1;
  gx = 0.0;
  gy = 0.0;
  for (int ky = ky1; ky <= ky2; ++ky) {
    if (ky < 0 || ky >= d.ny) continue;
    for (int kx = kx1; kx <= kx2; ++kx) {
      if (kx < 0 || kx >= d.nx) continue;
      const int j = (ix - 2 * kx) + 3 * (iy - 2 * ky);
      const size_t K = (size_t)ky * d.nx + kx;
      gx += b.ubar[(size_t)j * d.ne + K];
      gy += b.ubar[(size_t)(9 + j) * d.ne + K];
    }
  }
}

__global__ void k_adj_node(DevState d, AdjBuf b, const double *__restrict__ vprev,
                           const double *__restrict__ vnext, int has_vo, int gather) {
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= d.nn) return;
  const size_t nn = d.nn;
  const int iy = node / d.nw, ix = node - iy * d.nw;
  if (ix == 0 || iy == 0 || ix == d.nw - 1 || iy == d.nh - 1) {
    b.Fbar[node] = b.Fbar[nn + node] = 0.0;
    b.vdir[node] = b.vdir[nn + node] = 0.0;
    return;
  }
  double vbx = b.vbar[node], vby = b.vbar[nn + node];
  if (gather) {
    double gx, gy;
    gather_ubar(d, b, ix, iy, gx, gy);
    vbx = b.vdir[node] + gx;
    vby = b.vdir[nn + node] + gy;
  }
  const double vx = vprev[node], vy = vprev[nn + node];
  const double cA = d.nodec[0 * nn + node], cB = d.nodec[1 * nn + node];
  const double cK = d.nodec[2 * nn + node], cD = d.nodec[5 * nn + node];
  const double ox = has_vo ? d.vo[node] : 0.0, oy = has_vo ? d.vo[nn + node] : 0.0;
  const double dvx = ox - vx, dvy = oy - vy;
  const double s = sqrt(dvx * dvx + dvy * dvy);
  const double c = cD * s;
  const double a = cA + c;
  const double det = a * a + cB * cB;
  double rbx = 0.0, rby = 0.0, dx = 0.0, dy = 0.0;
  if (det != 0.0) {
    // rbar = A^-T vbar with A = [[a, -b], [b, a]]
    rbx = (a * vbx - cB * vby) / det;
    rby = (cB * vbx + a * vby) / det;
    const double px = vnext[node], py = vnext[nn + node];
    const double abar = -(rbx * px + rby * py);
    const double cbar = abar + rbx * ox + rby * oy;
    dx = cK * rbx;
    dy = cK * rby;
    if (s > 0.0) {
      const double g = cbar * cD / s;  // d c / d v = -cD (v_o - v)/|v_o - v|
      dx -= g * dvx;
      dy -= g * dvy;
    }
  }
  b.Fbar[node] = rbx;
  b.Fbar[nn + node] = rby;
  b.qbar[node] += rbx;
  b.qbar[nn + node] += rby;
  b.vdir[node] = dx;
  b.vdir[nn + node] = dy;
}

// ---- element stage ---------------------------------------------------------------
// VAR: DG1/DG2 ice, the strength P_g = P*_K f_g per Gauss point with
// f_g = max(0, h_g) exp(-C (1 - clamp(a_g))), and the -P/2 term projected
// per Gauss point as in the forward update; Pbar then accumulates
// dJ/dP*_K = sum_g dJ/dP_g f_g directly.
template <int NS, bool VAR>
__device__ __forceinline__ void adj_elem(const DevState &d, const Rheo &r, const AdjBuf &b,
                                         const double *__restrict__ vprev, int K, double C) {
  constexpr int NGP = DgSpace<NS>::NGP;
  constexpr int NG = NGP * NGP;
  const int ky = K / d.nx, kx = K - ky * d.nx;
  const double hx = d.lines[kx], ihx = d.lines[d.nx + kx];
  const double hy = d.lines[2 * d.nx + ky], ihy = d.lines[2 * d.nx + d.ny + ky];
  const size_t nn = d.nn, ne = d.ne;
  // forward recompute: strain invariants and Gauss-point quantities
  double u[9], v[9];
  const size_t base = (size_t)(2 * ky) * d.nw + 2 * kx;
#pragma unroll
  for (int bb = 0; bb < 3; ++bb)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      u[a + 3 * bb] = vprev[base + (size_t)bb * d.nw + a];
      v[a + 3 * bb] = vprev[nn + base + (size_t)bb * d.nw + a];
    }
  double Pc[NS], Qc[NS], Gc[NS];
  strain_invariants<NS>(u, v, ihx, ihy, r.ie, Pc, Qc, Gc);
  double pg_[NG], qg_[NG], gg_[NG];
  gauss_eval<NS>(Pc, pg_);
  gauss_eval<NS>(Qc, qg_);
  gauss_eval<NS>(Gc, gg_);
  const double Ph = VAR ? 0.0 : d.Pe[K] * r.hainv;
  // element-force adjoints from the nodal force adjoints
  double fbx[9], fby[9];
#pragma unroll
  for (int bb = 0; bb < 3; ++bb)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const size_t node = base + (size_t)bb * d.nw + a;
      fbx[a + 3 * bb] = b.Fbar[node];
      fby[a + 3 * bb] = b.Fbar[nn + node];
    }
  // Sbar total = carried Sbar + F^T fbar  (f_x = -hy Gxi S11 - hx Geta S12,
  //                                       f_y = -hy Gxi S12 - hx Geta S22)
  double B11[NS], B12[NS], B22[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double gxx = 0.0, gex = 0.0, gxy = 0.0, gey = 0.0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const double cx = gxi(j, s), ce = geta(j, s);
      if (cx != 0.0) {
        gxx = fma(cx, fbx[j], gxx);
        gxy = fma(cx, fby[j], gxy);
      }
      if (ce != 0.0) {
        gex = fma(ce, fbx[j], gex);
        gey = fma(ce, fby[j], gey);
      }
    }
    B11[s] = b.Sbar[(size_t)(0 * NS + s) * ne + K] - hy * gxx;
    B12[s] = b.Sbar[(size_t)(1 * NS + s) * ne + K] - hx * gex - hy * gxy;
    B22[s] = b.Sbar[(size_t)(2 * NS + s) * ne + K] - hx * gey;
  }
  // carried adjoint of S^{p-1}
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    b.Sbar[(size_t)(0 * NS + s) * ne + K] = r.fac * B11[s];
    b.Sbar[(size_t)(1 * NS + s) * ne + K] = r.fac * B12[s];
    b.Sbar[(size_t)(2 * NS + s) * ne + K] = r.fac * B22[s];
  }
  // S11 = .. + Ap - Ph d_s0 + ie AQ, S22 = .. + Ap - Ph d_s0 - ie AQ, S12 = .. + ie AG
  double Ab[NS], Qb[NS], Gb[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    Ab[s] = B11[s] + B22[s];
    Qb[s] = r.ie * (B11[s] - B22[s]);
    Gb[s] = r.ie * B12[s];
  }
  double Phbar = VAR ? 0.0 : -(B11[0] + B22[0]);
  double pb[NG], qb[NG], gb[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    double xpb = 0.0, xqb = 0.0, xgb = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const double w = proj<NS>(s, g);
      if (w != 0.0) {
        xpb = fma(w, Ab[s], xpb);
        xqb = fma(w, Qb[s], xqb);
        xgb = fma(w, Gb[s], xgb);
      }
    }
    const double d2 = fma(gg_[g], gg_[g], fma(qg_[g], qg_[g], fma(pg_[g], pg_[g], r.dmin2)));
    const double R = rsqrt(d2);
    double Phg = Ph;
    if constexpr (VAR) Phg = d.Pg[(size_t)g * ne + K] * r.hainv;
    const double X = Phg * R;
    const double Xbar = xpb * pg_[g] + xqb * qg_[g] + xgb * gg_[g];
    if constexpr (VAR) {
      const int gx = g % NGP, gy = g / NGP;
      const double h = fmax(0.0, dg_at_gauss<NGP>(d.H, d.na, ne, K, gx, gy));
      const double a = fmin(1.0, fmax(0.0, dg_at_gauss<NGP>(d.A, d.na, ne, K, gx, gy)));
      Phbar = fma(Xbar * R - xpb, h * exp(-C * (1.0 - a)), Phbar);
    } else {
      Phbar += Xbar * R;
    }
    const double d2bar = -0.5 * (Xbar * Phg) * R * R * R;
    pb[g] = X * xpb + 2.0 * pg_[g] * d2bar;
    qb[g] = X * xqb + 2.0 * qg_[g] * d2bar;
    gb[g] = X * xgb + 2.0 * gg_[g] * d2bar;
  }
  b.Pbar[K] += Phbar * r.hainv;
  // Gauss evaluation reversed, then the strain invariants and derivatives
  double Pcb[NS], Qcb[NS], Gcb[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double x = 0.0, y = 0.0, z = 0.0;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const double ps = psi<NS>(s, g);
      if (ps != 0.0) {
        x = fma(ps, pb[g], x);
        y = fma(ps, qb[g], y);
        z = fma(ps, gb[g], z);
      }
    }
    Pcb[s] = x;
    Qcb[s] = y;
    Gcb[s] = z;
  }
  const double cxe = ihx * r.ie, cye = ihy * r.ie;
  double ub[9], vb[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) ub[j] = vb[j] = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const double Uxib = ihx * Pcb[s] + cxe * Qcb[s];
    const double Vetab = ihy * Pcb[s] - cye * Qcb[s];
    const double Uetab = cye * Gcb[s];
    const double Vxib = cxe * Gcb[s];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const double cx = dxi(s, j), ce = deta(s, j);
      if (cx != 0.0) {
        ub[j] = fma(cx, Uxib, ub[j]);
        vb[j] = fma(cx, Vxib, vb[j]);
      }
      if (ce != 0.0) {
        ub[j] = fma(ce, Uetab, ub[j]);
        vb[j] = fma(ce, Vetab, vb[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    b.ubar[(size_t)j * ne + K] = ub[j];
    b.ubar[(size_t)(9 + j) * ne + K] = vb[j];
  }
}

// ---- general and curved elements ---------------------------------------------
// Transpose of gauss_eval: Fbar_s = sum_g psi_s(g) fbar_g.
template <int NS>
__device__ __forceinline__ void psi_T(const double *fbar, double Fbar[NS]) {
  constexpr int NG = DgSpace<NS>::NGP * DgSpace<NS>::NGP;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double acc = 0.0;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const double c = psi<NS>(s, g);
      if (c != 0.0) acc = fma(c, fbar[g], acc);
    }
    Fbar[s] = acc;
  }
}

// Transpose of gauss_moments: Dbar_g = w_g sum_s psi_s(g) Rbar_s.
template <int NS>
__device__ __forceinline__ void moments_T(const double Rbar[NS], double *Dbar) {
  constexpr int N = DgSpace<NS>::NGP;
  gauss_eval<NS>(Rbar, Dbar);
#pragma unroll
  for (int gy = 0; gy < N; ++gy)
#pragma unroll
    for (int gx = 0; gx < N; ++gx) Dbar[gx + N * gy] *= Gauss<N>::w(gx) * Gauss<N>::w(gy);
}

// Transpose of ref_grad_gauss: wbar_j = sum_g (dphi_j/dxi (g) gxib_g +
// dphi_j/deta (g) getab_g), sum-factorised.
template <int N>
__device__ __forceinline__ void ref_grad_T(const double *gxib, const double *getab,
                                           double wbar[9]) {
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    double t1[N], t2[N];
#pragma unroll
    for (int gx = 0; gx < N; ++gx) {
      double p = 0.0, q = 0.0;
#pragma unroll
      for (int gy = 0; gy < N; ++gy) {
        const double c0 = lq<N>(b, gy), cd = dlq<N>(b, gy);
        if (c0 != 0.0) p = fma(c0, gxib[gx + N * gy], p);
        if (cd != 0.0) q = fma(cd, getab[gx + N * gy], q);
      }
      t1[gx] = p;
      t2[gx] = q;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double x = 0.0;
#pragma unroll
      for (int gx = 0; gx < N; ++gx) {
        const double cd = dlq<N>(a, gx), c0 = lq<N>(a, gx);
        if (cd != 0.0) x = fma(cd, t1[gx], x);
        if (c0 != 0.0) x = fma(c0, t2[gx], x);
      }
      wbar[a + 3 * b] = x;
    }
  }
}

// Reverse of one subcycle's element stages on a general or curved element
// (the forward: strain_general, relax_general, forces_general).
template <int NS, bool VAR, typename G>
__device__ __forceinline__ void adj_elem_geo(const DevState &d, const Rheo &r, const AdjBuf &b,
                                             const double *__restrict__ vprev, int K, double C,
                                             const G &m) {
  constexpr int N = DgSpace<NS>::NGP, NG = N * N;
  const int ky = K / d.nx, kx = K - ky * d.nx;
  const size_t nn = d.nn, ne = d.ne;
  MassFactor<NS> F;
  {
    constexpr int NL = NS * (NS - 1) / 2;
#pragma unroll
    for (int i = 0; i < NL; ++i) F.L[i] = d.mfac[(size_t)i * ne + K];
#pragma unroll
    for (int i = 0; i < NS; ++i) F.Dinv[i] = d.mfac[(size_t)(NL + i) * ne + K];
  }
  // forward recompute: strain invariants at the Gauss points
  double pg_[NG], qg_[NG], gg_[NG];
  {
    double u[9], v[9];
    gather9(vprev, d.nw, kx, ky, u, d.flags, d.nn);
    gather9(vprev + nn, d.nw, kx, ky, v, d.flags, d.nn);
    double E11[NS], E22[NS], Esh[NS], Pc[NS], Qc[NS], Gc[NS];
    strain_general<NS>(m, F, u, v, E11, E22, Esh);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Pc[s] = E11[s] + E22[s];
      Qc[s] = r.ie * (E11[s] - E22[s]);
      Gc[s] = r.ie * Esh[s];
    }
    gauss_eval<NS>(Pc, pg_);
    gauss_eval<NS>(Qc, qg_);
    gauss_eval<NS>(Gc, gg_);
  }
  // divergence reversed: f = -(ref_grad)^T (a, b), so (abar, bbar) = -ref_grad(fbar)
  double B11[NS], B12[NS], B22[NS];
  {
    double fb[9], axb[NG], bxb[NG], ayb[NG], byb[NG];
    gather9(b.Fbar, d.nw, kx, ky, fb, d.flags, d.nn);
    ref_grad_gauss<N>(fb, axb, bxb);
    gather9(b.Fbar + nn, d.nw, kx, ky, fb, d.flags, d.nn);
    ref_grad_gauss<N>(fb, ayb, byb);
    double s11b[NG], s12b[NG], s22b[NG];
#pragma unroll
    for (int gy = 0; gy < N; ++gy)
#pragma unroll
      for (int gx = 0; gx < N; ++gx) {
        const int g = gx + N * gy;
        double j00, j01, j10, j11;
        jac_at<N>(m, gx, gy, j00, j01, j10, j11);
        const double w = -(Gauss<N>::w(gx) * Gauss<N>::w(gy));
        s11b[g] = w * fma(axb[g], j11, -(bxb[g] * j10));
        s12b[g] = w * (fma(bxb[g], j00, -(axb[g] * j01)) + fma(ayb[g], j11, -(byb[g] * j10)));
        s22b[g] = w * fma(byb[g], j00, -(ayb[g] * j01));
      }
    psi_T<NS>(s11b, B11);
    psi_T<NS>(s12b, B12);
    psi_T<NS>(s22b, B22);
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    B11[s] += b.Sbar[(size_t)(0 * NS + s) * ne + K];
    B12[s] += b.Sbar[(size_t)(1 * NS + s) * ne + K];
    B22[s] += b.Sbar[(size_t)(2 * NS + s) * ne + K];
    b.Sbar[(size_t)(0 * NS + s) * ne + K] = r.fac * B11[s];
    b.Sbar[(size_t)(1 * NS + s) * ne + K] = r.fac * B12[s];
    b.Sbar[(size_t)(2 * NS + s) * ne + K] = r.fac * B22[s];
  }
  // stress update reversed: S11 = fac S + RP + ie RQ (- Ph on s = 0 with DG0
  // ice), S22 = fac S + RP - ie RQ, S12 = fac S + ie RG, R = M^-1 moments
  double RP[NS], RQ[NS], RG[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    RP[s] = B11[s] + B22[s];
    RQ[s] = r.ie * (B11[s] - B22[s]);
    RG[s] = r.ie * B12[s];
  }
  double Phbar = VAR ? 0.0 : -RP[0];
  mass_solve<NS>(F, RP);
  mass_solve<NS>(F, RQ);
  mass_solve<NS>(F, RG);
  double pb[NG], qb[NG], gb[NG];
  moments_T<NS>(RP, pb);
  moments_T<NS>(RQ, qb);
  moments_T<NS>(RG, gb);
  const double Ph = VAR ? 0.0 : d.Pe[K] * r.hainv;
#pragma unroll
  for (int gy = 0; gy < N; ++gy)
#pragma unroll
    for (int gx = 0; gx < N; ++gx) {
      const int g = gx + N * gy;
      double j00, j01, j10, j11;
      jac_at<N>(m, gx, gy, j00, j01, j10, j11);
      const double det = fma(j00, j11, -(j01 * j10));
      const double d2 = fma(gg_[g], gg_[g], fma(qg_[g], qg_[g], fma(pg_[g], pg_[g], r.dmin2)));
      const double R = rsqrt(d2);
      double Pg = Ph;
      if constexpr (VAR) Pg = d.Pg[(size_t)g * ne + K] * r.hainv;
      const double Xd = Pg * R * det;
      const double Xdbar = pb[g] * pg_[g] + qb[g] * qg_[g] + gb[g] * gg_[g];
      double Pgbar = Xdbar * R * det;
      if constexpr (VAR) {
        Pgbar -= det * pb[g];
        const double h = fmax(0.0, dg_at_gauss<N>(d.H, d.na, ne, K, gx, gy));
        const double a = fmin(1.0, fmax(0.0, dg_at_gauss<N>(d.A, d.na, ne, K, gx, gy)));
        Phbar = fma(Pgbar, h * exp(-C * (1.0 - a)), Phbar);
      } else {
        Phbar += Pgbar;
      }
      const double d2bar = -0.5 * (Xdbar * Pg * det) * R * R * R;
      pb[g] = fma(2.0 * pg_[g], d2bar, Xd * pb[g]);
      qb[g] = fma(2.0 * qg_[g], d2bar, Xd * qb[g]);
      gb[g] = fma(2.0 * gg_[g], d2bar, Xd * gb[g]);
    }
  b.Pbar[K] += Phbar * r.hainv;
  // Gauss evaluation and invariants reversed, then the strain projection
  double E11b[NS], E22b[NS], Eshb[NS];
  {
    double Pcb[NS], Qcb[NS], Gcb[NS];
    psi_T<NS>(pb, Pcb);
    psi_T<NS>(qb, Qcb);
    psi_T<NS>(gb, Gcb);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      E11b[s] = fma(r.ie, Qcb[s], Pcb[s]);
      E22b[s] = fma(-r.ie, Qcb[s], Pcb[s]);
      Eshb[s] = r.ie * Gcb[s];
    }
  }
  mass_solve<NS>(F, E11b);
  mass_solve<NS>(F, E22b);
  mass_solve<NS>(F, Eshb);
  double D11b[NG], D22b[NG], Dshb[NG];
  moments_T<NS>(E11b, D11b);
  moments_T<NS>(E22b, D22b);
  moments_T<NS>(Eshb, Dshb);
  double uxib[NG], uetab[NG], vxib[NG], vetab[NG];
#pragma unroll
  for (int gy = 0; gy < N; ++gy)
#pragma unroll
    for (int gx = 0; gx < N; ++gx) {
      const int g = gx + N * gy;
      double j00, j01, j10, j11;
      jac_at<N>(m, gx, gy, j00, j01, j10, j11);
      uxib[g] = fma(j11, D11b[g], -(j01 * Dshb[g]));
      uetab[g] = fma(j00, Dshb[g], -(j10 * D11b[g]));
      vxib[g] = fma(j11, Dshb[g], -(j01 * D22b[g]));
      vetab[g] = fma(j00, D22b[g], -(j10 * Dshb[g]));
    }
  double ub[9], vb[9];
  ref_grad_T<N>(uxib, uetab, ub);
  ref_grad_T<N>(vxib, vetab, vb);
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    b.ubar[(size_t)j * ne + K] = ub[j];
    b.ubar[(size_t)(9 + j) * ne + K] = vb[j];
  }
}

template <int NS, bool VAR>
__global__ void __launch_bounds__(128) k_adj_elem_geo(DevState d, Rheo r, AdjBuf b,
                                                      const double *__restrict__ vprev, double C) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= d.ne) return;
  if (d.isoJ) {
    const IsoGeoG<DgSpace<NS>::NGP, double> m{d.isoJ + K, (size_t)d.ne};
    adj_elem_geo<NS, VAR>(d, r, b, vprev, K, C, m);
  } else {
    const int ky = K / d.nx, kx = K - ky * d.nx;
    const QuadMap m = quad_map(d.xy, d.nx, kx, ky, d.flags, (long long)(d.nx + 1) * (d.ny + 1));
    adj_elem_geo<NS, VAR>(d, r, b, vprev, K, C, m);
  }
}

// Persistent: the grid is the number of blocks resident on the chip and each
// block takes an equal contiguous share of the element warps (a grid of one
// block per 128 elements ends in a partial wave: 256^2 gives 512 blocks for
// 760 slots, 3 or 4 per SM).
constexpr int kAdjElemBlock = 128;

template <int NS, bool VAR>
__global__ void __launch_bounds__(kAdjElemBlock) k_adj_elem(DevState d, Rheo r, AdjBuf b,
                                                            const double *__restrict__ vprev,
                                                            double C) {
  const int nwarps = (d.ne + 31) >> 5;
  const int w0 = (int)((long long)nwarps * blockIdx.x / gridDim.x);
  const int w1 = (int)((long long)nwarps * (blockIdx.x + 1) / gridDim.x);
  const int lane = threadIdx.x & 31;
  for (int w = w0 + (int)(threadIdx.x >> 5); w < w1; w += kAdjElemBlock / 32) {
    const int K = (w << 5) + lane;
    if (K < d.ne) adj_elem<NS, VAR>(d, r, b, vprev, K, C);
  }
}

// Grid of the persistent reverse element kernel: resident blocks x SMs, at
// most one block per 128 elements.
template <int NS, bool VAR>
int adj_elem_grid(const DevState &d) {
  static int resident = 0;
  if (resident == 0) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_adj_elem<NS, VAR>, kAdjElemBlock, 0) !=
            cudaSuccess ||
        n < 1) {
      cudaGetLastError();
      n = 1;
    }
    resident = n;
  }
  const long long need = (d.ne + kAdjElemBlock - 1) / kAdjElemBlock;
  const long long fit = (long long)resident * d.nsm;
  return (int)(need < fit ? need : fit);
}

// ---- gradients -------------------------------------------------------------------
// dJ/dP*_K = Pbar_K max(0,H) exp(-C(1-clamp A)) (DG0 ice; with DG1/DG2 ice
// Pbar already holds dJ/dP*_K),  dJ/dtau_j = l_j qbar_j
__global__ void k_adj_grads(DevState d, AdjBuf b, double C, double *gP, double *gT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d.ne && gP) {
    if (d.na > 1) {
      gP[i] = b.Pbar[i];
    } else {
      const double h = fmax(0.0, d.H[i]);
      const double a = fmin(1.0, fmax(0.0, d.A[i]));
      gP[i] = b.Pbar[i] * h * exp(-C * (1.0 - a));
    }
  }
  if (i < d.nn && gT) {
    const size_t nn = d.nn;
    gT[i] = b.area[i] * b.qbar[i];
    gT[nn + i] = b.area[i] * b.qbar[nn + i];
  }
}

inline int blocks(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace
}  // namespace mevp

namespace {

int afail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return mevp::api_fail(code, buf);
}

#define ADJ_CUDA(call, what)                                 \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) {                                 \
      rc = mevp::api_cuda_fail(e_, what);                    \
      goto done;                                             \
    }                                                        \
  } while (0)

}  // namespace

extern "C" int mevp_adjoint_kinetic_energy(mevp_state *s, int n, int checkpoint_every,
                                           double *J, double *dJ_dPstar, double *dJ_dtau,
                                           int on_device) {
  using namespace mevp;
  NvtxRange nvtx_range_("mevp_adjoint_kinetic_energy");
  int rc = api_check_state(s);
  if (rc) return rc;
  if (s->prec != MEVP_FP64) return afail(MEVP_ERR_UNSUPPORTED, "adjoint: FP64 states only");
  if (n < 1) return afail(MEVP_ERR_ARG, "adjoint: n=%d < 1", n);
  if (checkpoint_every < 1) return afail(MEVP_ERR_ARG, "adjoint: checkpoint_every < 1");
  if (!s->prepared) return afail(MEVP_ERR_STATE, "adjoint: call mevp_begin_step first");
  const DevState &d = s->d;
  const size_t nn = d.nn, ne = d.ne, ns = s->ns;
  const int k = checkpoint_every < n ? checkpoint_every : n;
  const int nseg = (n + k - 1) / k;
  const size_t vbytes = sizeof(double) * 2 * nn, sbytes = sizeof(double) * 3 * ns * ne;
  const int nparts = blocks((long long)nn, kBlock);
  cudaStream_t st = s->stream;
  // device memory: checkpoints, one segment of velocities, adjoint buffers
  const size_t total = (size_t)nseg * (vbytes + sbytes) + (size_t)(k + 1) * vbytes +
                       4 * vbytes + sbytes + sizeof(double) * (18 * ne + ne + nn + nparts + 1) +
                       vbytes + sbytes;
  char *mem = nullptr;
  double *vfinal = nullptr, *Sfinal = nullptr;
  AdjBuf b{};
  std::vector<double *> ck_v, ck_S;
  double *hist = nullptr;
  int cur0 = s->cur;
  cudaError_t err = cudaMalloc(&mem, total);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return afail(MEVP_ERR_OOM, "adjoint: %zu bytes of device memory unavailable", total);
  }
  {
    char *p = mem;
    auto take = [&](size_t bytes) {
      char *q = p;
      p += bytes;
      return (double *)q;
    };
    for (int g = 0; g < nseg; ++g) {
      ck_v.push_back(take(vbytes));
      ck_S.push_back(take(sbytes));
    }
    hist = take((size_t)(k + 1) * vbytes);
    b.vbar = take(vbytes);
    b.vdir = take(vbytes);
    b.Fbar = take(vbytes);
    b.qbar = take(vbytes);
    b.Sbar = take(sbytes);
    b.ubar = take(sizeof(double) * 18 * ne);
    b.Pbar = take(sizeof(double) * ne);
    b.area = take(sizeof(double) * nn);
    b.partial = take(sizeof(double) * nparts);
    b.J = take(sizeof(double));
    vfinal = take(vbytes);
    Sfinal = take(sbytes);
  }
  {
    // forward sweep with checkpoints (v, S) at the start of every segment
    for (int g = 0; g < nseg; ++g) {
      ADJ_CUDA(cudaMemcpyAsync(ck_v[g], d.vel[s->cur], vbytes, cudaMemcpyDeviceToDevice, st),
               "adjoint checkpoint");
      ADJ_CUDA(cudaMemcpyAsync(ck_S[g], d.S, sbytes, cudaMemcpyDeviceToDevice, st),
               "adjoint checkpoint");
      const int len = (g == nseg - 1) ? n - g * k : k;
      // the last segment's velocities are recorded as they are computed, so
      // the reverse sweep needs no recomputation for it (with
      // checkpoint_every >= n: none at all)
      const bool record = g == nseg - 1;
      if (record)
        ADJ_CUDA(cudaMemcpyAsync(hist, d.vel[s->cur], vbytes, cudaMemcpyDeviceToDevice, st),
                 "adjoint history");
      for (int i = 0; i < len; ++i) {
        ADJ_CUDA(launch_subcycle_f64(d, s->rheo, s->has_vo, s->cur, st, nullptr),
                 "adjoint forward");
        s->cur ^= 1;
        if (record)
          ADJ_CUDA(cudaMemcpyAsync(hist + (size_t)(i + 1) * 2 * nn, d.vel[s->cur], vbytes,
                                   cudaMemcpyDeviceToDevice, st),
                   "adjoint history");
      }
    }
    // final forward state, restored after the reverse sweep
    const int cur_final = s->cur;
    ADJ_CUDA(cudaMemcpyAsync(vfinal, d.vel[cur_final], vbytes, cudaMemcpyDeviceToDevice, st),
             "adjoint save");
    ADJ_CUDA(cudaMemcpyAsync(Sfinal, d.S, sbytes, cudaMemcpyDeviceToDevice, st), "adjoint save");
    // objective and seed
    ADJ_CUDA(cudaMemsetAsync(b.qbar, 0, vbytes, st), "adjoint init");
    ADJ_CUDA(cudaMemsetAsync(b.Sbar, 0, sbytes, st), "adjoint init");
    ADJ_CUDA(cudaMemsetAsync(b.Pbar, 0, sizeof(double) * ne, st), "adjoint init");
    k_adj_seed<<<nparts, kBlock, 0, st>>>(d, b, d.vel[cur_final]);
    k_adj_sum<<<1, 32, 0, st>>>(b, nparts);
    ADJ_CUDA(launch_lumped_area(d, b.area, st), "adjoint area");
    ADJ_CUDA(cudaGetLastError(), "adjoint seed");
    // reverse sweep, segment by segment
    bool first = true;
    for (int g = nseg - 1; g >= 0; --g) {
      const int len = (g == nseg - 1) ? n - g * k : k;
      // recompute the segment's velocities: hist[i] = v after i subcycles of
      // the segment (the last segment's were recorded by the forward sweep)
      const int cur_g = cur0 ^ ((g * k) & 1);
      if (g != nseg - 1) {
        ADJ_CUDA(cudaMemcpyAsync(d.vel[cur_g], ck_v[g], vbytes, cudaMemcpyDeviceToDevice, st),
                 "adjoint restore");
        ADJ_CUDA(cudaMemcpyAsync(d.S, ck_S[g], sbytes, cudaMemcpyDeviceToDevice, st),
                 "adjoint restore");
        ADJ_CUDA(cudaMemcpyAsync(hist, ck_v[g], vbytes, cudaMemcpyDeviceToDevice, st),
                 "adjoint restore");
      }
      int c = cur_g;
      for (int i = 0; i < len && g != nseg - 1; ++i) {
        ADJ_CUDA(launch_subcycle_f64(d, s->rheo, s->has_vo, c, st, nullptr), "adjoint recompute");
        c ^= 1;
        ADJ_CUDA(cudaMemcpyAsync(hist + (size_t)(i + 1) * 2 * nn, d.vel[c], vbytes,
                                 cudaMemcpyDeviceToDevice, st),
                 "adjoint history");
      }
      const bool var = d.na > 1;
      const int eg = ns == 3 ? (var ? adj_elem_grid<3, true>(d) : adj_elem_grid<3, false>(d))
                   : ns == 6 ? (var ? adj_elem_grid<6, true>(d) : adj_elem_grid<6, false>(d))
                             : (var ? adj_elem_grid<8, true>(d) : adj_elem_grid<8, false>(d));
      const double C = s->prm.C;
      for (int i = len - 1; i >= 0; --i) {
        const double *vprev = hist + (size_t)i * 2 * nn;
        const double *vnext = hist + (size_t)(i + 1) * 2 * nn;
        k_adj_node<<<blocks(nn, kBlock), kBlock, 0, st>>>(d, b, vprev, vnext, s->has_vo ? 1 : 0,
                                                           first ? 0 : 1);
        if (d.xy || d.nxy) {
          const int gg = blocks(ne, 128);
          if (ns == 3)
            var ? k_adj_elem_geo<3, true><<<gg, 128, 0, st>>>(d, s->rheo, b, vprev, C)
                : k_adj_elem_geo<3, false><<<gg, 128, 0, st>>>(d, s->rheo, b, vprev, C);
          else if (ns == 6)
            var ? k_adj_elem_geo<6, true><<<gg, 128, 0, st>>>(d, s->rheo, b, vprev, C)
                : k_adj_elem_geo<6, false><<<gg, 128, 0, st>>>(d, s->rheo, b, vprev, C);
          else
            var ? k_adj_elem_geo<8, true><<<gg, 128, 0, st>>>(d, s->rheo, b, vprev, C)
                : k_adj_elem_geo<8, false><<<gg, 128, 0, st>>>(d, s->rheo, b, vprev, C);
        } else if (ns == 3)
          var ? k_adj_elem<3, true><<<eg, kAdjElemBlock, 0, st>>>(d, s->rheo, b, vprev, C)
              : k_adj_elem<3, false><<<eg, kAdjElemBlock, 0, st>>>(d, s->rheo, b, vprev, C);
        else if (ns == 6)
          var ? k_adj_elem<6, true><<<eg, kAdjElemBlock, 0, st>>>(d, s->rheo, b, vprev, C)
              : k_adj_elem<6, false><<<eg, kAdjElemBlock, 0, st>>>(d, s->rheo, b, vprev, C);
        else
          var ? k_adj_elem<8, true><<<eg, kAdjElemBlock, 0, st>>>(d, s->rheo, b, vprev, C)
              : k_adj_elem<8, false><<<eg, kAdjElemBlock, 0, st>>>(d, s->rheo, b, vprev, C);
        ADJ_CUDA(cudaGetLastError(), "adjoint reverse");
        first = false;
      }
    }
    // gradients
    {
      double *gP = dJ_dPstar, *gT = dJ_dtau;
      double *tmp = nullptr;
      if (!on_device && (gP || gT)) {
        err = cudaMalloc(&tmp, sizeof(double) * (ne + 2 * nn));
        if (err != cudaSuccess) {
          cudaGetLastError();
          rc = afail(MEVP_ERR_OOM, "adjoint: gradient staging");
          goto done;
        }
        gP = dJ_dPstar ? tmp : nullptr;
        gT = dJ_dtau ? tmp + ne : nullptr;
      }
      k_adj_grads<<<blocks(ne > 2 * nn ? ne : 2 * nn, kBlock), kBlock, 0, st>>>(d, b, s->prm.C,
                                                                               gP, gT);
      err = cudaGetLastError();
      if (err == cudaSuccess && !on_device) {
        if (dJ_dPstar)
          err = cudaMemcpyAsync(dJ_dPstar, tmp, sizeof(double) * ne, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess && dJ_dtau)
          err = cudaMemcpyAsync(dJ_dtau, tmp + ne, sizeof(double) * 2 * nn,
                                cudaMemcpyDeviceToHost, st);
      }
      if (err == cudaSuccess && J)
        err = cudaMemcpyAsync(J, b.J, sizeof(double),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
      // the state ends where the forward sweep ended
      if (err == cudaSuccess)
        err = cudaMemcpyAsync(d.vel[cur_final], vfinal, vbytes, cudaMemcpyDeviceToDevice, st);
      if (err == cudaSuccess)
        err = cudaMemcpyAsync(d.S, Sfinal, sbytes, cudaMemcpyDeviceToDevice, st);
      if (err == cudaSuccess) err = cudaStreamSynchronize(st);
      s->cur = cur_final;
      if (tmp) cudaFree(tmp);
      if (err != cudaSuccess) {
        rc = api_cuda_fail(err, "adjoint: gradients");
        goto done;
      }
    }
  }
done:
  cudaStreamSynchronize(st);
  cudaFree(mem);
  return rc;
}
