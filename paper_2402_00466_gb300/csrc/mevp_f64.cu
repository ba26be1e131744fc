// mevp_f64.cu -- FP64 kernels of the mEVP momentum subcycle on GB300 (sm_103a).
//
// One subcycle (the four stages of Table 1 of Jendersie, Lessig, Richter,
// PASC'24) runs as two launches:
//
//   k_element_f64  one thread per element: gather the 9 CG2 velocities,
//                  project the symmetric velocity gradient onto the DG stress
//                  space (strain), evaluate it at the Gauss points, apply the
//                  viscous-plastic law and the relaxed stress update of
//                  Listing 1 / App. A (stress), and form the weak divergence
//                  of the new stress tested with the 9 Q2 functions (element
//                  part of "divergence").  Writes S and 18 element forces.
//   k_node_f64     one thread per 2x2 block of CG2 nodes: sum the element
//                  forces of the (up to four) elements around each node in
//                  the fixed order SW, SE, NW, NE -- a gather, no atomics --
//                  and solve the beta-relaxed implicit velocity update with
//                  ocean drag and Coriolis ("velocity").
//
// The element geometry is recomputed on the fly from the mesh lines (the
// paper's "on-the-fly map", Sec. 3.2), so no per-element matrices are read.
// On a rectangle the inverse local mass and the Jacobian cancel, leaving the
// compile-time reference tables of mevp_ref.cuh scaled by 1/hx, 1/hy.
#include "mevp_elem.cuh"
#include "mevp_geom.cuh"
#include "mevp_internal.cuh"
#include "mevp_ref.cuh"

namespace mevp {

namespace {

// The single-state FP64 kernels are persistent: one block per SM, each block
// taking an equal contiguous share of the element warps (node slots), so that
// every SM gets the same work whatever the mesh size -- a plain grid of
// independent blocks leaves part of the chip idle in its last wave.  512
// threads at one block per SM caps the element kernel at 128 registers.
constexpr int kElemBlock = 512;
constexpr int kNodeSlotThreads = 768;
constexpr int kNodeBlock = 256;

// Strain coefficients E11, E12, E22 (for the diagnostic read-back):
// E11 = du/dx, E22 = dv/dy, E12 = (du/dy + dv/dx)/2, projected onto DG.
template <int NS>
__device__ __forceinline__ void strain_dg(const double u[9], const double v[9], double ihx,
                                          double ihy, double E11[NS], double E12[NS],
                                          double E22[NS]) {
  double Uxi[NS], Ueta[NS], Vxi[NS], Veta[NS];
  ref_derivs<NS>(u, Uxi, Ueta);
  ref_derivs<NS>(v, Vxi, Veta);
  const double h2x = 0.5 * ihx, h2y = 0.5 * ihy;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    E11[s] = ihx * Uxi[s];
    E22[s] = ihy * Veta[s];
    E12[s] = fma(h2y, Ueta[s], h2x * Vxi[s]);
  }
}

// One element of the FP64 subcycle (strain, stress update in place, element
// forces into the force buffer).
template <int NS, bool VAR = false>
__device__ __forceinline__ void elem_f64(const DevState &d, const Rheo &r, int cur, int K) {
  const int ky = K / d.nx, kx = K - ky * d.nx;
  const long long nl = 2LL * (d.nx + d.ny);
  const double hx = ck_ldg(d.flags, (const double *)d.lines, kx, nl, 101);
  const double ihx = ck_ldg(d.flags, (const double *)d.lines, d.nx + kx, nl, 101);
  const double hy = ck_ldg(d.flags, (const double *)d.lines, 2 * d.nx + ky, nl, 101);
  const double ihy = ck_ldg(d.flags, (const double *)d.lines, 2 * d.nx + d.ny + ky, nl, 101);
  double u[9], v[9];
  gather9(d.vel[cur], d.nw, kx, ky, u, d.flags, d.nn);
  gather9(d.vel[cur] + d.nn, d.nw, kx, ky, v, d.flags, d.nn);
  double Pc[NS], Qc[NS], Gc[NS];
  strain_invariants<NS>(u, v, ihx, ihy, r.ie, Pc, Qc, Gc);
  double S11[NS], S12[NS], S22[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    S11[s] = ck_ld(d.flags, d.S, (long long)(0 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 103);
    S12[s] = ck_ld(d.flags, d.S, (long long)(1 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 103);
    S22[s] = ck_ld(d.flags, d.S, (long long)(2 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 103);
  }
  if constexpr (VAR) {  // DG1/DG2 H, A: ice strength per Gauss point
    constexpr int NG = DgSpace<NS>::NGP * DgSpace<NS>::NGP;
    double Phg[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) Phg[g] = ck_ldg(d.flags, d.Pg, (long long)g * d.ne + K, (long long)NG * d.ne, 104) * r.hainv;
    relax_stress_p<NS, true>(S11, S12, S22, Pc, Qc, Gc, 0.0, Phg, r.dmin2, r.fac, r.ie);
  } else {
    const double Ph = ck_ldg(d.flags, d.Pe, (long long)K, (long long)d.ne, 104) * r.hainv;
    relax_stress<NS>(S11, S12, S22, Pc, Qc, Gc, Ph, r.dmin2, r.fac, r.ie);
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    ck_st(d.flags, d.S, (long long)(0 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 105, S11[s]);
    ck_st(d.flags, d.S, (long long)(1 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 105, S12[s]);
    ck_st(d.flags, d.S, (long long)(2 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 105, S22[s]);
  }
  double fx[9], fy[9];
  element_forces_t<NS>(S11, S12, S22, hx, hy, fx, fy);
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    ck_st(d.flags, d.fbuf, (long long)j * d.ne + K, 18LL * d.ne, 106, fx[j]);
    ck_st(d.flags, d.fbuf, (long long)(9 + j) * d.ne + K, 18LL * d.ne, 106, fy[j]);
  }
}

template <int NS, bool VAR = false>
__global__ void __launch_bounds__(kElemBlock, 1) k_element_f64(DevState d, Rheo r, int cur) {
  const int nwarps = (d.ne + 31) >> 5;
  const int w0 = (int)((long long)nwarps * blockIdx.x / gridDim.x);
  const int w1 = (int)((long long)nwarps * (blockIdx.x + 1) / gridDim.x);
  const int lane = threadIdx.x & 31;
  for (int w = w0 + (int)(threadIdx.x >> 5); w < w1; w += kElemBlock / 32) {
    const int K = (w << 5) + lane;
    if (K < d.ne) elem_f64<NS, VAR>(d, r, cur, K);
  }
}

// Sum of the element forces at node (ix, iy) over the elements that contain
// it, in ascending element order (SW, SE, NW, NE), starting from the first.
__device__ __forceinline__ void gather_force(const double *__restrict__ fb, int ne, int nx,
                                             int ny, int ix, int iy, double &Fx, double &Fy) {
  const int kx1 = (ix & 1) ? (ix >> 1) : (ix >> 1) - 1;  // first candidate column
  const int kx2 = ix >> 1;                                // last candidate column
  const int ky1 = (iy & 1) ? (iy >> 1) : (iy >> 1) - 1;
  const int ky2 = iy >> 1;
  bool first = true;
  Fx = 0.0;
  Fy = 0.0;
  for (int ky = ky1; ky <= ky2; ++ky) {
    if (ky < 0 || ky >= ny) continue;
    for (int kx = kx1; kx <= kx2; ++kx) {
      if (kx < 0 || kx >= nx) continue;
      const int j = (ix - 2 * kx) + 3 * (iy - 2 * ky);
      const int K = ky * nx + kx;
      const double gx = __ldg(fb + (size_t)j * ne + K);
      const double gy = __ldg(fb + (size_t)(9 + j) * ne + K);
      if (first) {
        Fx = gx;
        Fy = gy;
        first = false;
      } else {
        Fx += gx;
        Fy += gy;
      }
    }
  }
}

// The up-to-four CG2 nodes (2kx + dx, 2ky + dy), dx, dy in {0,1}, of node
// slot (kx, ky): force gather and velocity update.
// VO: an ocean velocity is set (else the ocean is at rest and its terms,
// exact zeros, are left out at compile time).
template <bool VO>
__device__ __forceinline__ void node_slot_f64(const DevState &d, int cur, int kx,
                                              int ky) {
  const double *__restrict__ vp = d.vel[cur];
  double *__restrict__ vq = d.vel[cur ^ 1];
  const size_t nn = d.nn;
  const size_t ne = d.ne;
#pragma unroll
  for (int dy = 0; dy < 2; ++dy) {
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const int ix = 2 * kx + dx, iy = 2 * ky + dy;
      if (ix >= d.nw || iy >= d.nh) continue;
      const size_t node = (size_t)iy * d.nw + ix;
      if (ix == 0 || iy == 0 || ix == d.nw - 1 || iy == d.nh - 1) {
        ck_st(d.flags, vq, (long long)node, 2LL * nn, 115, 0.0);
        ck_st(d.flags, vq, (long long)(nn + node), 2LL * nn, 115, 0.0);
        continue;
      }
      const double *__restrict__ fb = d.fbuf;
      const long long nf = 18LL * ne;
      double Fx, Fy;
      if (dx == 0 && dy == 0) {  // vertex node: 4 elements
        const size_t Ksw = (size_t)(ky - 1) * d.nx + kx - 1, Kse = Ksw + 1;
        const size_t Knw = (size_t)ky * d.nx + kx - 1, Kne = Knw + 1;
        Fx = ck_ldg(d.flags, fb, (long long)(8 * ne + Ksw), nf, 111) + ck_ldg(d.flags, fb, (long long)(6 * ne + Kse), nf, 111);
        Fx = Fx + ck_ldg(d.flags, fb, (long long)(2 * ne + Knw), nf, 111);
        Fx = Fx + ck_ldg(d.flags, fb, (long long)(0 * ne + Kne), nf, 111);
        Fy = ck_ldg(d.flags, fb, (long long)(17 * ne + Ksw), nf, 111) + ck_ldg(d.flags, fb, (long long)(15 * ne + Kse), nf, 111);
        Fy = Fy + ck_ldg(d.flags, fb, (long long)(11 * ne + Knw), nf, 111);
        Fy = Fy + ck_ldg(d.flags, fb, (long long)(9 * ne + Kne), nf, 111);
      } else if (dx == 1 && dy == 0) {  // horizontal edge: S then N element
        const size_t Ks = (size_t)(ky - 1) * d.nx + kx, Kn = (size_t)ky * d.nx + kx;
        Fx = ck_ldg(d.flags, fb, (long long)(7 * ne + Ks), nf, 111) + ck_ldg(d.flags, fb, (long long)(1 * ne + Kn), nf, 111);
        Fy = ck_ldg(d.flags, fb, (long long)(16 * ne + Ks), nf, 111) + ck_ldg(d.flags, fb, (long long)(10 * ne + Kn), nf, 111);
      } else if (dx == 0 && dy == 1) {  // vertical edge: W then E element
        const size_t Kw = (size_t)ky * d.nx + kx - 1, Ke = Kw + 1;
        Fx = ck_ldg(d.flags, fb, (long long)(5 * ne + Kw), nf, 111) + ck_ldg(d.flags, fb, (long long)(3 * ne + Ke), nf, 111);
        Fy = ck_ldg(d.flags, fb, (long long)(14 * ne + Kw), nf, 111) + ck_ldg(d.flags, fb, (long long)(12 * ne + Ke), nf, 111);
      } else {  // element centre
        const size_t K = (size_t)ky * d.nx + kx;
        Fx = ck_ldg(d.flags, fb, (long long)(4 * ne + K), nf, 111);
        Fy = ck_ldg(d.flags, fb, (long long)(13 * ne + K), nf, 111);
      }
      const double vx = ck_ld(d.flags, vp, (long long)node, 2LL * nn, 112);
      const double vy = ck_ld(d.flags, vp, (long long)(nn + node), 2LL * nn, 112);
      const double cA = ck_ldg(d.flags, (const double *)d.nodec, (long long)(0 * nn + node), 6LL * nn, 113), cB = ck_ldg(d.flags, (const double *)d.nodec, (long long)(1 * nn + node), 6LL * nn, 113);
      const double cK = ck_ldg(d.flags, (const double *)d.nodec, (long long)(2 * nn + node), 6LL * nn, 113), qx = ck_ldg(d.flags, (const double *)d.nodec, (long long)(3 * nn + node), 6LL * nn, 113);
      const double qy = ck_ldg(d.flags, (const double *)d.nodec, (long long)(4 * nn + node), 6LL * nn, 113), cD = ck_ldg(d.flags, (const double *)d.nodec, (long long)(5 * nn + node), 6LL * nn, 113);
      double c, rx = fma(cK, vx, qx) + Fx, ry = fma(cK, vy, qy) + Fy;
      if constexpr (VO) {
        const double ox = ck_ldg(d.flags, (const double *)d.vo, (long long)node, 2LL * nn, 114);
        const double oy =
            ck_ldg(d.flags, (const double *)d.vo, (long long)(nn + node), 2LL * nn, 114);
        const double dvx = ox - vx, dvy = oy - vy;
        c = cD * sqrt(dvx * dvx + dvy * dvy);
        rx += c * ox;
        ry += c * oy;
      } else {
        c = cD * sqrt(vx * vx + vy * vy);  // |0 - v|
      }
      const double a = cA + c;
      const double det = fma(a, a, cB * cB);
      double ux = 0.0, uy = 0.0;
      if (det != 0.0) {
        const double inv = 1.0 / det;
        ux = fma(a, rx, cB * ry) * inv;
        uy = fma(a, ry, -cB * rx) * inv;
      }
      ck_st(d.flags, vq, (long long)node, 2LL * nn, 115, ux);
      ck_st(d.flags, vq, (long long)(nn + node), 2LL * nn, 115, uy);
    }
  }
}

// Velocity update at an interior node (Eq. 2 with the mEVP beta relaxation;
// drag coefficient lagged, drag and Coriolis implicit):
//   a = m(1+beta)/dt + c,  b = m f,  c = l Cw rho_w |v_o - v^{p-1}|
//   r = m beta/dt v^{p-1} + (m/dt v^n + l tau) + F + c v_o
//   (a + i b) v^p = r   (complex notation)
template <bool VO>
__global__ void __launch_bounds__(kNodeSlotThreads, 1) k_node_f64(DevState d, int cur) {
  const int sw = d.nx + 1;
  const int nslots = sw * (d.ny + 1);
  const int s0 = (int)((long long)nslots * blockIdx.x / gridDim.x);
  const int s1 = (int)((long long)nslots * (blockIdx.x + 1) / gridDim.x);
  for (int slot = s0 + (int)threadIdx.x; slot < s1; slot += kNodeSlotThreads) {
    const int ky = slot / sw, kx = slot - ky * sw;
    node_slot_f64<VO>(d, cur, kx, ky);
  }
}

// Ensemble kernels: persistent, grid-stride over (member, block) work items.
// One launch per stress space (the members' work lists are kept per n_S), so
// that each runs the element arithmetic of one space alone.  The 3-dof
// kernel fits the single-state budget of 512 resident threads per SM; the
// 6-dof one keeps the member descriptor's pointers in registers besides, and
// capped at 128 registers it spilled 272 B a thread, so it is left uncapped.
template <int B, int NS>
__global__ void __launch_bounds__(B, NS == 3 ? 512 / B : 1)
    k_ens_f64_elem(const EnsMember *__restrict__ mem,
                                                             const EnsWork *__restrict__ work,
                                                             int nwork, int flip) {
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const EnsWork it = work[w];
    const EnsMember &m = mem[it.member];
    const int K = it.tx * B + threadIdx.x;
    if (K >= m.d.ne) continue;
    elem_f64<NS>(m.d, m.r, m.base_cur ^ flip, K);
  }
}

__global__ void __launch_bounds__(kNodeBlock) k_ens_f64_node(const EnsMember *__restrict__ mem,
                                                             const EnsWork *__restrict__ work,
                                                             int nwork, int flip) {
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const EnsWork it = work[w];
    const EnsMember &m = mem[it.member];
    const int slot = it.tx * kNodeBlock + threadIdx.x;
    const int sw = m.d.nx + 1;
    if (slot >= sw * (m.d.ny + 1)) continue;
    const int ky = slot / sw, kx = slot - ky * sw;
    if (m.has_vo)
      node_slot_f64<true>(m.d, m.base_cur ^ flip, kx, ky);
    else
      node_slot_f64<false>(m.d, m.base_cur ^ flip, kx, ky);
  }
}

// ---- outer-step preparation ----------------------------------------------
// Element widths and their inverses per mesh column / row.
__global__ void k_mesh_lines(DevState d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d.nx) {
    const double h = d.xline[i + 1] - d.xline[i];
    d.lines[i] = h;
    d.lines[d.nx + i] = 1.0 / h;
  } else if (i < d.nx + d.ny) {
    const int j = i - d.nx;
    const double h = d.yline[j + 1] - d.yline[j];
    d.lines[2 * d.nx + j] = h;
    d.lines[2 * d.nx + d.ny + j] = 1.0 / h;
  }
}

__global__ void k_strength(DevState d, double Pstar, double C) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= d.ne) return;
  const double h = fmax(0.0, d.H[K]);
  const double a = fmin(1.0, fmax(0.0, d.A[K]));
  d.Pe[K] = (d.pstar ? d.pstar[K] : Pstar) * h * exp(-C * (1.0 - a));
}


// DG1/DG2 H, A: the ice strength P = P* max(0,H) exp(-C(1 - clamp(A,0,1)))
// at each Gauss point of the stress rule (Listing 1 evaluates H, A there).
template <int N>
__global__ void k_strength_gauss(DevState d, double Pstar, double C) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= d.ne) return;
  const double ps = d.pstar ? d.pstar[K] : Pstar;
  for (int gy = 0; gy < N; ++gy)
    for (int gx = 0; gx < N; ++gx) {
      const double h = fmax(0.0, dg_at_gauss<N>(d.H, d.na, d.ne, K, gx, gy));
      const double a = fmin(1.0, fmax(0.0, dg_at_gauss<N>(d.A, d.na, d.ne, K, gx, gy)));
      d.Pg[(size_t)(gx + N * gy) * d.ne + K] = ps * h * exp(-C * (1.0 - a));
    }
}

// det J at the N x N Gauss points of an isoparametric element (reference
// gradients of its 9 node positions).
template <int N>
__device__ __forceinline__ void iso_det_gauss(const DevState &d, int kx, int ky,
                                              double det[N * N]) {
  double X[9], Y[9];
  const long long base = (long long)(2 * ky) * d.nw + 2 * kx;
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) {
      const double2 p = ck_ldg(d.flags, d.nxy, base + (long long)b * d.nw + a, d.nn, 143);
      X[a + 3 * b] = p.x;
      Y[a + 3 * b] = p.y;
    }
  double xxi[N * N], xeta[N * N], yxi[N * N], yeta[N * N];
  ref_grad_gauss<N>(X, xxi, xeta);
  ref_grad_gauss<N>(Y, yxi, yeta);
  for (int g = 0; g < N * N; ++g) det[g] = fma(xxi[g], yeta[g], -(xeta[g] * yxi[g]));
}

// int_K w phi_j (w = 1, or max(0, H) with DG1/DG2 H) on an isoparametric
// element with the N-point rule of the stress space.
template <int N>
__device__ __forceinline__ double iso_integral(const DevState &d, int kx, int ky, int a, int b,
                                               bool with_h) {
  double det[N * N];
  iso_det_gauss<N>(d, kx, ky, det);
  const int K = ky * d.nx + kx;
  double acc = 0.0;
  for (int gy = 0; gy < N; ++gy)
    for (int gx = 0; gx < N; ++gx) {
      double w = Gauss<N>::w(gx) * Gauss<N>::w(gy) * det[gx + N * gy];
      if (with_h) {
        const double hv = d.na == 1 ? d.H[K] : dg_at_gauss<N>(d.H, d.na, d.ne, K, gx, gy);
        w *= fmax(0.0, hv);
      }
      acc = fma(w, lq<N>(a, gx) * lq<N>(b, gy), acc);
    }
  return acc;
}

// int_K max(0, H) phi_j for DG1/DG2 H with the N-point rule of the stress
// space, phi_j the Q2 function of local node (a, b).
template <int N>
__device__ __forceinline__ double mass_integral_gauss(const DevState &d, int kx, int ky, int a,
                                                      int b) {
  if (d.nxy) return iso_integral<N>(d, kx, ky, a, b, true);
  const int K = ky * d.nx + kx;
  QuadMap m;
  if (d.xy) {
    m = quad_map(d.xy, d.nx, kx, ky, d.flags, (long long)(d.nx + 1) * (d.ny + 1));
  } else {
    m.Ax = d.xline[kx + 1] - d.xline[kx];
    m.By = d.yline[ky + 1] - d.yline[ky];
    m.Ay = m.Bx = m.cx = m.cy = 0.0;
  }
  const double d0 = m.d0(), d1 = m.d1(), d2 = m.d2();
  double acc = 0.0;
  for (int gy = 0; gy < N; ++gy)
    for (int gx = 0; gx < N; ++gx) {
      const double det = fma(d1, Gauss<N>::xh(gx), fma(d2, Gauss<N>::xh(gy), d0));
      const double h = fmax(0.0, dg_at_gauss<N>(d.H, d.na, d.ne, K, gx, gy));
      const double w = Gauss<N>::w(gx) * Gauss<N>::w(gy) * det;
      acc = fma(w * h, lq<N>(a, gx) * lq<N>(b, gy), acc);
    }
  return acc;
}

// int_K phi_j of the Q2 function of local node (a, b) on element (kx, ky).
__device__ __forceinline__ double node_area(const DevState &d, int kx, int ky, int a, int b) {
  if (d.nxy)
    return d.ns == 3 ? iso_integral<2>(d, kx, ky, a, b, false)
                     : iso_integral<3>(d, kx, ky, a, b, false);
  if (d.xy)
    return node_area_general(
        quad_map(d.xy, d.nx, kx, ky, d.flags, (long long)(d.nx + 1) * (d.ny + 1)), a, b);
  const double area = (d.xline[kx + 1] - d.xline[kx]) * (d.yline[ky + 1] - d.yline[ky]);
  return area * q2w(a) * q2w(b);
}

// Lumped area l_j = sum_K int_K phi_j (elements in ascending order).
__global__ void k_lumped_area(DevState d, double *__restrict__ out) {
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= d.nn) return;
  const int iy = node / d.nw, ix = node - iy * d.nw;
  const int kx1 = (ix & 1) ? (ix >> 1) : (ix >> 1) - 1, kx2 = ix >> 1;
  const int ky1 = (iy & 1) ? (iy >> 1) : (iy >> 1) - 1, ky2 = iy >> 1;
  double l = 0.0;
  for (int ky = ky1; ky <= ky2; ++ky) {
    if (ky < 0 || ky >= d.ny) continue;
    for (int kx = kx1; kx <= kx2; ++kx) {
      if (kx < 0 || kx >= d.nx) continue;
      l += node_area(d, kx, ky, ix - 2 * kx, iy - 2 * ky);
    }
  }
  out[node] = l;
}

// Lumped mass m_j = rho_ice sum_K max(0,H_K) int_K phi_j and area
// l_j = sum_K int_K phi_j (hx hy w_a w_b on a rectangle, w = 1/6, 2/3, 1/6;
// the exact integral against the affine det J on a general element), then the
// node constants.
__global__ void k_node_constants(DevState d, int cur, mevp_params p, int has_vo) {
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= d.nn) return;
  const int iy = node / d.nw, ix = node - iy * d.nw;
  const int kx1 = (ix & 1) ? (ix >> 1) : (ix >> 1) - 1, kx2 = ix >> 1;
  const int ky1 = (iy & 1) ? (iy >> 1) : (iy >> 1) - 1, ky2 = iy >> 1;
  double l = 0.0, mh = 0.0;
  for (int ky = ky1; ky <= ky2; ++ky) {
    if (ky < 0 || ky >= d.ny) continue;
    for (int kx = kx1; kx <= kx2; ++kx) {
      if (kx < 0 || kx >= d.nx) continue;
      const double w = node_area(d, kx, ky, ix - 2 * kx, iy - 2 * ky);
      l += w;
      if (d.na == 1 && !d.nxy)
        mh += fmax(0.0, d.H[ky * d.nx + kx]) * w;
      else if (d.na == 1)
        mh += d.ns == 3 ? iso_integral<2>(d, kx, ky, ix - 2 * kx, iy - 2 * ky, true)
                        : iso_integral<3>(d, kx, ky, ix - 2 * kx, iy - 2 * ky, true);
      else if (d.ns == 3)
        mh += mass_integral_gauss<2>(d, kx, ky, ix - 2 * kx, iy - 2 * ky);
      else
        mh += mass_integral_gauss<3>(d, kx, ky, ix - 2 * kx, iy - 2 * ky);
    }
  }
  const double m = p.rho_ice * mh;
  const double mdt = m / p.dt;
  const size_t nn = d.nn;
  const double *v = d.vel[cur];
  d.mass[node] = m;
  d.nodec[0 * nn + node] = mdt * (1.0 + p.beta);
  d.nodec[1 * nn + node] = m * p.coriolis_f;
  d.nodec[2 * nn + node] = mdt * p.beta;
  d.nodec[3 * nn + node] = fma(mdt, v[node], l * d.tau[node]);
  d.nodec[4 * nn + node] = fma(mdt, v[nn + node], l * d.tau[nn + node]);
  d.nodec[5 * nn + node] = l * p.Cw * p.rho_water;
  (void)has_vo;
}

// ---- diagnostics ------------------------------------------------------------
template <int NS>
__global__ void k_strain_diag(DevState d, int cur) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= d.ne) return;
  const int ky = K / d.nx, kx = K - ky * d.nx;
  const double ihx = 1.0 / (d.xline[kx + 1] - d.xline[kx]);
  const double ihy = 1.0 / (d.yline[ky + 1] - d.yline[ky]);
  double u[9], v[9];
  gather9(d.vel[cur], d.nw, kx, ky, u, d.flags, d.nn);
  gather9(d.vel[cur] + d.nn, d.nw, kx, ky, v, d.flags, d.nn);
  double E11[NS], E12[NS], E22[NS];
  strain_dg<NS>(u, v, ihx, ihy, E11, E12, E22);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    d.diag[(size_t)(0 * NS + s) * d.ne + K] = E11[s];
    d.diag[(size_t)(1 * NS + s) * d.ne + K] = E12[s];
    d.diag[(size_t)(2 * NS + s) * d.ne + K] = E22[s];
  }
}

template <int NS>
__global__ void k_force_elem(DevState d) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= d.ne) return;
  const int ky = K / d.nx, kx = K - ky * d.nx;
  const double hx = d.xline[kx + 1] - d.xline[kx];
  const double hy = d.yline[ky + 1] - d.yline[ky];
  double S11[NS], S12[NS], S22[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    S11[s] = ck_ld(d.flags, d.S, (long long)(0 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 103);
    S12[s] = ck_ld(d.flags, d.S, (long long)(1 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 103);
    S22[s] = ck_ld(d.flags, d.S, (long long)(2 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 103);
  }
  double fx[9], fy[9];
  element_forces_t<NS>(S11, S12, S22, hx, hy, fx, fy);
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    ck_st(d.flags, d.fbuf, (long long)j * d.ne + K, 18LL * d.ne, 106, fx[j]);
    ck_st(d.flags, d.fbuf, (long long)(9 + j) * d.ne + K, 18LL * d.ne, 106, fy[j]);
  }
}

__global__ void k_force_gather(DevState d) {
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= d.nn) return;
  const int iy = node / d.nw, ix = node - iy * d.nw;
  double Fx, Fy;
  gather_force(d.fbuf, d.ne, d.nx, d.ny, ix, iy, Fx, Fy);
  d.diag[node] = Fx;
  d.diag[(size_t)d.nn + node] = Fy;
}

// Watchdog: any non-finite velocity component raises flags[0] (every writer
// stores the same value, so no atomics are needed).
__global__ void k_nan_check(DevState d, int cur) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)d.nn; i += stride) {
    bool bad;
    if (d.prec == MEVP_MIXED) {
      const float4 v = d.vel4[cur][i];
      bad = !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
    } else {
      bad = !(isfinite(d.vel[cur][i]) && isfinite(d.vel[cur][(size_t)d.nn + i]));
    }
    if (bad) d.flags[0] = 1;
  }
}

inline int blocks(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_nan_check(const DevState &d, int cur, cudaStream_t st) {
  int b = blocks(d.nn, 256);
  if (b > 152 * 8) b = 152 * 8;
  k_nan_check<<<b, 256, 0, st>>>(d, cur);
  return cudaGetLastError();
}

cudaError_t launch_prepare(const DevState &d, const mevp_params &p, bool has_vo, int cur,
                           cudaStream_t st) {
  if (!d.xy && !d.nxy) k_mesh_lines<<<blocks(d.nx + d.ny, 256), 256, 0, st>>>(d);
  if (d.na == 1)
    k_strength<<<blocks(d.ne, 256), 256, 0, st>>>(d, p.Pstar, p.C);
  else if (d.ns == 3)
    k_strength_gauss<2><<<blocks(d.ne, 256), 256, 0, st>>>(d, p.Pstar, p.C);
  else
    k_strength_gauss<3><<<blocks(d.ne, 256), 256, 0, st>>>(d, p.Pstar, p.C);
  k_node_constants<<<blocks(d.nn, 256), 256, 0, st>>>(d, cur, p, has_vo ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_element_f64(const DevState &d, const Rheo &r, int cur, cudaStream_t st) {
  const int eg = d.nsm;  // persistent: one block per SM
  if (d.nxy)
    launch_element_iso(d, r, cur, st);
  else if (d.xy)
    launch_element_general(d, r, cur, st);
  else if (d.na == 1) {
    if (d.ns == 3)
      k_element_f64<3><<<eg, kElemBlock, 0, st>>>(d, r, cur);
    else if (d.ns == 6)
      k_element_f64<6><<<eg, kElemBlock, 0, st>>>(d, r, cur);
    else
      k_element_f64<8><<<eg, kElemBlock, 0, st>>>(d, r, cur);
  } else {
    if (d.ns == 3)
      k_element_f64<3, true><<<eg, kElemBlock, 0, st>>>(d, r, cur);
    else if (d.ns == 6)
      k_element_f64<6, true><<<eg, kElemBlock, 0, st>>>(d, r, cur);
    else
      k_element_f64<8, true><<<eg, kElemBlock, 0, st>>>(d, r, cur);
  }
  return cudaGetLastError();
}

cudaError_t launch_subcycle_f64(const DevState &d, const Rheo &r, bool has_vo, int cur,
                                cudaStream_t st, cudaEvent_t *ev) {
  if (ev) cudaEventRecord(ev[0], st);
  launch_element_f64(d, r, cur, st);
  if (ev) cudaEventRecord(ev[1], st);
  const long long slots = (long long)(d.nx + 1) * (d.ny + 1);
  (void)slots;
  if (has_vo)
    k_node_f64<true><<<d.nsm, kNodeSlotThreads, 0, st>>>(d, cur);
  else
    k_node_f64<false><<<d.nsm, kNodeSlotThreads, 0, st>>>(d, cur);
  if (ev) cudaEventRecord(ev[2], st);
  return cudaGetLastError();
}

// FP64 ensemble element block sizes the autotuner chooses from.
const int kF64Blocks[kF64BlockCount] = {64, 128, 256};

template <int NS>
void launch_ens_elem(const EnsMember *mem, const EnsWork *ework, int nework, int block,
                     int grid, int flip, cudaStream_t st) {
  switch (block) {
    case 0: k_ens_f64_elem<64, NS><<<grid, 64, 0, st>>>(mem, ework, nework, flip); break;
    case 1: k_ens_f64_elem<128, NS><<<grid, 128, 0, st>>>(mem, ework, nework, flip); break;
    default: k_ens_f64_elem<256, NS><<<grid, 256, 0, st>>>(mem, ework, nework, flip); break;
  }
}

cudaError_t launch_ensemble_f64(const EnsMember *mem, const EnsWork *ework, int nework, int ns,
                                int block, int grid, int flip, cudaStream_t st) {
  if (nework <= 0) return cudaSuccess;
  if (ns == 3)
    launch_ens_elem<3>(mem, ework, nework, block, grid, flip, st);
  else
    launch_ens_elem<6>(mem, ework, nework, block, grid, flip, st);
  return cudaGetLastError();
}

cudaError_t launch_ensemble_f64_node(const EnsMember *mem, const EnsWork *nwork_list, int nnwork,
                                     int grid_n, int flip, cudaStream_t st) {
  if (nnwork > 0) k_ens_f64_node<<<grid_n, kNodeBlock, 0, st>>>(mem, nwork_list, nnwork, flip);
  return cudaGetLastError();
}

template <int NS>
int ens_elem_ctas(int block) {
  int n = 0;
  switch (block) {
    case 0: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_f64_elem<64, NS>, 64, 0); break;
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_f64_elem<128, NS>, 128, 0); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_f64_elem<256, NS>, 256, 0); break;
  }
  return n > 0 ? n : 1;
}

int f64_block_ctas_per_sm(int block, int ns) {
  return ns == 3 ? ens_elem_ctas<3>(block) : ens_elem_ctas<6>(block);
}

int f64_node_ctas_per_sm() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_f64_node, kNodeBlock, 0);
  return n > 0 ? n : 1;
}

cudaError_t launch_lumped_area(const DevState &d, double *out, cudaStream_t st) {
  k_lumped_area<<<blocks(d.nn, 256), 256, 0, st>>>(d, out);
  return cudaGetLastError();
}

cudaError_t launch_strain_diag(const DevState &d, int cur, cudaStream_t st) {
  if (d.nxy) return launch_strain_diag_iso(d, cur, st);
  if (d.xy) return launch_strain_diag_general(d, cur, st);
  if (d.ns == 3)
    k_strain_diag<3><<<blocks(d.ne, 128), 128, 0, st>>>(d, cur);
  else if (d.ns == 6)
    k_strain_diag<6><<<blocks(d.ne, 128), 128, 0, st>>>(d, cur);
  else
    k_strain_diag<8><<<blocks(d.ne, 128), 128, 0, st>>>(d, cur);
  return cudaGetLastError();
}

cudaError_t launch_force_diag(const DevState &d, cudaStream_t st) {
  if (d.nxy)
    launch_force_elem_iso(d, st);
  else if (d.xy)
    launch_force_elem_general(d, st);
  else if (d.ns == 3)
    k_force_elem<3><<<blocks(d.ne, 128), 128, 0, st>>>(d);
  else if (d.ns == 6)
    k_force_elem<6><<<blocks(d.ne, 128), 128, 0, st>>>(d);
  else
    k_force_elem<8><<<blocks(d.ne, 128), 128, 0, st>>>(d);
  k_force_gather<<<blocks(d.nn, 256), 256, 0, st>>>(d);
  return cudaGetLastError();
}

}  // namespace mevp
