// mevp_advect.cu -- DG upwind advection of the ice height H and
// concentration A (the transport equations of Sec. 2 with zero sources,
// discretised as Sec. 2.1 states: discontinuous Galerkin in space with the
// standard upwind flux, explicit Runge-Kutta in time).
//
// One thread per element evaluates, for both fields at once (same velocity,
// same upwind decisions),
//   L(U)_K = M_K^-1 [ int_ref U (vt_xi dpsi/dxi + vt_eta dpsi/deta)
//                     - sum_edges int_edge f Uhat psi ],
// where vt = detJ J^-1 v is the contravariant CG2 velocity, f the outward
// flux density per unit reference edge length (+-vt_xi on the east/west
// edges, +-vt_eta on the north/south edges: the edge's tangent rotated and
// dotted with v, which depends only on the edge, so both elements of an edge
// compute the same value and the scheme is conservative to rounding), and
// Uhat the trace of the element the flow leaves (own trace on the domain
// boundary).  NQ x NQ Gauss points in the element and NQ on each edge,
// NQ = 3 for DG0/DG1, 4 for DG2.  The Runge-Kutta stages are Shu-Osher
// combinations U_out = a U0 + b (U_in + dt L(U_in)); one launch per stage.
#include "mevp_geom.cuh"
#include "mevp_internal.cuh"

namespace mevp {

namespace {

constexpr int kAdvBlock = 128;

// 1-D Gauss rules on [0,1] in centred coordinates: 3 points (+-sqrt(15)/10,
// 0) and 4 points (+-sqrt(525 -+ 70 sqrt 30)/70 / 2) with their weights.
template <int NQ> struct Rule;
template <> struct Rule<3> {
  __host__ __device__ static constexpr double xh(int q) { return Gauss<3>::xh(q); }
  __host__ __device__ static constexpr double w(int q) { return Gauss<3>::w(q); }
};
// 4-point Gauss-Legendre on [-1,1]: +-0.339981043584856264803 (weight
// 0.652145154862546142627), +-0.861136311594052575224 (0.347854845137453857373).
template <> struct Rule<4> {
  __host__ __device__ static constexpr double xh(int q) {
    return q == 0 ? -0.430568155797026287612
         : q == 1 ? -0.169990521792428132401
         : q == 2 ? 0.169990521792428132401
                  : 0.430568155797026287612;
  }
  __host__ __device__ static constexpr double w(int q) {
    return (q == 0 || q == 3) ? 0.173927422568726928687 : 0.326072577431273071314;
  }
};

// centred Legendre p_k and its derivative at centred coordinate x
__host__ __device__ constexpr double leg(int k, double x) {
  return k == 0 ? 1.0 : k == 1 ? x : x * x - 1.0 / 12.0;
}
__host__ __device__ constexpr double dleg(int k, double x) {
  return k == 0 ? 0.0 : k == 1 ? 1.0 : 2.0 * x;
}
// Q2 Lagrange function a at centred coordinate x: 2x^2 - x, 1 - 4x^2, 2x^2 + x
__host__ __device__ constexpr double lag2(int a, double x) {
  return a == 0 ? 2.0 * x * x - x : a == 1 ? 1.0 - 4.0 * x * x : 2.0 * x * x + x;
}
// and its derivative: 4x - 1, -8x, 4x + 1
__host__ __device__ constexpr double dlag2(int a, double x) {
  return a == 0 ? 4.0 * x - 1.0 : a == 1 ? -8.0 * x : 4.0 * x + 1.0;
}

// Jacobian of an isoparametric element at centred reference point (xh, eh)
// from its 9 node positions X, Y (local node a + 3b).
__device__ __forceinline__ void iso_jac(const double X[9], const double Y[9], double xh,
                                        double eh, double &j00, double &j01, double &j10,
                                        double &j11) {
  j00 = j01 = j10 = j11 = 0.0;
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double gx = dlag2(a, xh) * lag2(b, eh), ge = lag2(a, xh) * dlag2(b, eh);
      j00 = fma(X[a + 3 * b], gx, j00);
      j01 = fma(X[a + 3 * b], ge, j01);
      j10 = fma(Y[a + 3 * b], gx, j10);
      j11 = fma(Y[a + 3 * b], ge, j11);
    }
}

// Element geometry: the bilinear map from the vertices on a general mesh, or
// the rectangle hx x hy of the mesh lines; and the four edge vectors, each
// the difference of its two vertices (west and east edges oriented along eta,
// south and north edges along xi), so that the two elements sharing an edge
// see the same vector.
struct AdvGeom {
  QuadMap m;
  double ex[4], ey[4];  // 0 west, 1 east, 2 south, 3 north
};

__device__ __forceinline__ AdvGeom adv_geom(const DevState &d, int kx, int ky) {
  AdvGeom G;
  if (d.xy) {
    const size_t vw = (size_t)d.nx + 1;
    const long long nv = (long long)vw * (d.ny + 1);
    const double2 p00 = ck_ld(d.flags, d.xy, (long long)(ky * vw + kx), nv, 175);
    const double2 p10 = ck_ld(d.flags, d.xy, (long long)(ky * vw + kx + 1), nv, 175);
    const double2 p01 = ck_ld(d.flags, d.xy, (long long)((ky + 1) * vw + kx), nv, 175);
    const double2 p11 = ck_ld(d.flags, d.xy, (long long)((ky + 1) * vw + kx + 1), nv, 175);
    G.m = quad_map(d.xy, d.nx, kx, ky, d.flags, (long long)(d.nx + 1) * (d.ny + 1));
    G.ex[0] = p01.x - p00.x; G.ey[0] = p01.y - p00.y;
    G.ex[1] = p11.x - p10.x; G.ey[1] = p11.y - p10.y;
    G.ex[2] = p10.x - p00.x; G.ey[2] = p10.y - p00.y;
    G.ex[3] = p11.x - p01.x; G.ey[3] = p11.y - p01.y;
  } else {
    const double hx = ck_ld(d.flags, d.xline, kx + 1, d.nx + 1, 175) -
                      ck_ld(d.flags, d.xline, kx, d.nx + 1, 175);
    const double hy = ck_ld(d.flags, d.yline, ky + 1, d.ny + 1, 175) -
                      ck_ld(d.flags, d.yline, ky, d.ny + 1, 175);
    G.m.Ax = hx; G.m.Ay = 0.0; G.m.Bx = 0.0; G.m.By = hy; G.m.cx = 0.0; G.m.cy = 0.0;
    G.ex[0] = G.ex[1] = 0.0; G.ey[0] = G.ey[1] = hy;
    G.ex[2] = G.ex[3] = hx; G.ey[2] = G.ey[3] = 0.0;
  }
  return G;
}

struct AdvArgs {
  const double *H0, *A0;    // U0 (start of the step), [n_a][ne]
  const double *Hin, *Ain;  // U_in (stage input)
  double *Hout, *Aout;      // U_out
  const double *vel;        // [2][nn]
  double a, b, dt;          // U_out = a U0 + b (U_in + dt L(U_in))
};

template <int NA, int NQ, bool ISO>
__device__ __forceinline__ void adv_element(const DevState &d, const AdvArgs &g, int K) {
  const int ky = K / d.nx, kx = K - ky * d.nx;
  const size_t ne = d.ne, nn = d.nn;
  // geometry: the bilinear map and edge vectors, or (ISO) the 9 node
  // positions of the isoparametric element
  AdvGeom G{};
  double X[9], Y[9];
  if constexpr (ISO) {
    const long long base = (long long)(2 * ky) * d.nw + 2 * kx;
#pragma unroll
    for (int bb = 0; bb < 3; ++bb)
#pragma unroll
      for (int aa = 0; aa < 3; ++aa) {
        const double2 p = ck_ldg(d.flags, d.nxy, base + (long long)bb * d.nw + aa, d.nn, 176);
        X[aa + 3 * bb] = p.x;
        Y[aa + 3 * bb] = p.y;
      }
  } else {
    G = adv_geom(d, kx, ky);
  }
  const QuadMap &m = G.m;
  double wdet[NQ * NQ];  // ISO: w det J at the volume points (mass matrix)
  const long long nf = (long long)d.na * d.ne;
  double h[NA], a[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) {
    h[i] = ck_ld(d.flags, g.Hin, (long long)i * ne + K, nf, 171);
    a[i] = ck_ld(d.flags, g.Ain, (long long)i * ne + K, nf, 171);
  }
  double vx[9], vy[9];
  gather9(g.vel, d.nw, kx, ky, vx, d.flags, d.nn);
  gather9(g.vel + nn, d.nw, kx, ky, vy, d.flags, d.nn);
  double RH[NA], RA[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) RH[i] = RA[i] = 0.0;

  if constexpr (ISO) {
#pragma unroll
    for (int qy = 0; qy < NQ; ++qy)
#pragma unroll
      for (int qx = 0; qx < NQ; ++qx) {
        double j00, j01, j10, j11;
        iso_jac(X, Y, Rule<NQ>::xh(qx), Rule<NQ>::xh(qy), j00, j01, j10, j11);
        wdet[qx + NQ * qy] = Rule<NQ>::w(qx) * Rule<NQ>::w(qy) * fma(j00, j11, -(j01 * j10));
      }
  }
  // volume terms
  if (NA > 1) {
#pragma unroll
    for (int qy = 0; qy < NQ; ++qy)
#pragma unroll
      for (int qx = 0; qx < NQ; ++qx) {
        const double xh = Rule<NQ>::xh(qx), eh = Rule<NQ>::xh(qy);
        const double w = Rule<NQ>::w(qx) * Rule<NQ>::w(qy);
        double ux = 0.0, uy = 0.0;
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
          double rx = 0.0, ry = 0.0;
#pragma unroll
          for (int aa = 0; aa < 3; ++aa) {
            rx = fma(lag2(aa, xh), vx[aa + 3 * bb], rx);
            ry = fma(lag2(aa, xh), vy[aa + 3 * bb], ry);
          }
          ux = fma(lag2(bb, eh), rx, ux);
          uy = fma(lag2(bb, eh), ry, uy);
        }
        double j00, j01, j10, j11;
        if constexpr (ISO) {
          iso_jac(X, Y, xh, eh, j00, j01, j10, j11);
        } else {
          j00 = fma(m.cx, eh, m.Ax);
          j10 = fma(m.cy, eh, m.Ay);
          j01 = fma(m.cx, xh, m.Bx);
          j11 = fma(m.cy, xh, m.By);
        }
        const double vtx = w * fma(j11, ux, -(j01 * uy));
        const double vte = w * fma(j00, uy, -(j10 * ux));
        double hq = 0.0, aq = 0.0;
#pragma unroll
        for (int i = 0; i < NA; ++i) {
          const double p = leg(dgx(i), xh) * leg(dgy(i), eh);
          hq = fma(h[i], p, hq);
          aq = fma(a[i], p, aq);
        }
#pragma unroll
        for (int i = 1; i < NA; ++i) {
          const double gi = vtx * (dleg(dgx(i), xh) * leg(dgy(i), eh)) +
                            vte * (leg(dgx(i), xh) * dleg(dgy(i), eh));
          RH[i] = fma(hq, gi, RH[i]);
          RA[i] = fma(aq, gi, RA[i]);
        }
      }
  }

  // edges: 0 west (xi=0), 1 east (xi=1), 2 south (eta=0), 3 north (eta=1)
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    int nb;
    if (e == 0) nb = kx > 0 ? K - 1 : -1;
    else if (e == 1) nb = kx < d.nx - 1 ? K + 1 : -1;
    else if (e == 2) nb = ky > 0 ? K - d.nx : -1;
    else nb = ky < d.ny - 1 ? K + d.nx : -1;
    double hn[NA], an[NA];
    if (nb >= 0) {
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        hn[i] = ck_ld(d.flags, g.Hin, (long long)i * ne + nb, nf, 172);
        an[i] = ck_ld(d.flags, g.Ain, (long long)i * ne + nb, nf, 172);
      }
    }
    // edge vector t (along eta on west/east edges, along xi on south/north
    // edges); the outward flux density is f = sgn (t_y v_x - t_x v_y), i.e.
    // +vt_xi on the east, -vt_xi on the west, -vt_eta on the south and
    // +vt_eta on the north edge.
    const bool vert = e < 2;
    const double side = (e == 1 || e == 3) ? 0.5 : -0.5;
    const double sgn = (e == 1 || e == 2) ? 1.0 : -1.0;
    const int n0 = vert ? (e == 0 ? 0 : 2) : (e == 2 ? 0 : 6);
    const int step = vert ? 3 : 1;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const double t = Rule<NQ>::xh(q), w = Rule<NQ>::w(q);
      // the edge tangent (ISO: the derivative of the edge's quadratic through
      // its three nodes, the same seen from both elements)
      double tx = G.ex[e], ty = G.ey[e];
      if constexpr (ISO) {
        tx = 0.0;
        ty = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          tx = fma(dlag2(k, t), X[n0 + step * k], tx);
          ty = fma(dlag2(k, t), Y[n0 + step * k], ty);
        }
      }
      double ux = 0.0, uy = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ux = fma(lag2(k, t), vx[n0 + step * k], ux);
        uy = fma(lag2(k, t), vy[n0 + step * k], uy);
      }
      const double f = sgn * fma(ty, ux, -(tx * uy));
      // reference coordinates of the point on this element's edge
      const double xh = vert ? side : t, eh = vert ? t : side;
      double ho = 0.0, ao = 0.0;
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        const double p = leg(dgx(i), xh) * leg(dgy(i), eh);
        ho = fma(h[i], p, ho);
        ao = fma(a[i], p, ao);
      }
      double hu = ho, au = ao;
      if (nb >= 0 && f < 0.0) {  // inflow: the neighbour's trace at the same point
        const double nxh = vert ? -side : t, neh = vert ? t : -side;
        hu = 0.0;
        au = 0.0;
#pragma unroll
        for (int i = 0; i < NA; ++i) {
          const double p = leg(dgx(i), nxh) * leg(dgy(i), neh);
          hu = fma(hn[i], p, hu);
          au = fma(an[i], p, au);
        }
      }
      const double wf = w * f;
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        const double p = leg(dgx(i), xh) * leg(dgy(i), eh);
        RH[i] = fma(-wf * hu, p, RH[i]);
        RA[i] = fma(-wf * au, p, RA[i]);
      }
    }
  }

  // L = M^-1 R
  bool done = false;
  if constexpr (ISO) {
    if constexpr (NA > 1) {
      MassFactor<NA> F;
      ldl_factor<NA, double>(
          [&](int i, int j) -> double {
            double acc = 0.0;
#pragma unroll
            for (int qy = 0; qy < NQ; ++qy)
#pragma unroll
              for (int qx = 0; qx < NQ; ++qx) {
                const double xh = Rule<NQ>::xh(qx), eh = Rule<NQ>::xh(qy);
                const double pp = leg(dgx(i), xh) * leg(dgy(i), eh) * leg(dgx(j), xh) *
                                  leg(dgy(j), eh);
                acc = fma(wdet[qx + NQ * qy], pp, acc);
              }
            return acc;
          },
          F);
      mass_solve<NA>(F, RH);
      mass_solve<NA>(F, RA);
    } else {
      double area = 0.0;
#pragma unroll
      for (int q = 0; q < NQ * NQ; ++q) area += wdet[q];
      RH[0] /= area;
      RA[0] /= area;
    }
    done = true;
  } else if constexpr (NA > 1) {
    if (d.xy) {
      MassFactor<NA> F;
      mass_factor<NA>(m, F);
      mass_solve<NA>(F, RH);
      mass_solve<NA>(F, RA);
      done = true;
    }
  }
  if (!done) {
    const double idet = 1.0 / m.d0();
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const double s = idet / dgmass(i);
      RH[i] *= s;
      RA[i] *= s;
    }
  }
#pragma unroll
  for (int i = 0; i < NA; ++i) {
    const long long o = (long long)i * ne + K;
    const double hs = fma(g.dt, RH[i], h[i]), as = fma(g.dt, RA[i], a[i]);
    const double h0 = g.a == 0.0 ? 0.0 : ck_ld(d.flags, g.H0, o, nf, 173);
    const double a0 = g.a == 0.0 ? 0.0 : ck_ld(d.flags, g.A0, o, nf, 173);
    ck_st(d.flags, g.Hout, o, nf, 174, g.a == 0.0 ? g.b * hs : fma(g.a, h0, g.b * hs));
    ck_st(d.flags, g.Aout, o, nf, 174, g.a == 0.0 ? g.b * as : fma(g.a, a0, g.b * as));
  }
}

template <int NA, int NQ, bool ISO>
__global__ void __launch_bounds__(kAdvBlock) k_advect(DevState d, AdvArgs g) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K < d.ne) adv_element<NA, NQ, ISO>(d, g, K);
}

inline int blocks(long long n, int b) { return (int)((n + b - 1) / b); }

cudaError_t stage(const DevState &d, const AdvArgs &g, cudaStream_t st) {
  const int gr = blocks(d.ne, kAdvBlock);
  if (d.nxy) {
    switch (d.na) {
      case 1: k_advect<1, 3, true><<<gr, kAdvBlock, 0, st>>>(d, g); break;
      case 3: k_advect<3, 3, true><<<gr, kAdvBlock, 0, st>>>(d, g); break;
      default: k_advect<6, 4, true><<<gr, kAdvBlock, 0, st>>>(d, g); break;
    }
  } else {
    switch (d.na) {
      case 1: k_advect<1, 3, false><<<gr, kAdvBlock, 0, st>>>(d, g); break;
      case 3: k_advect<3, 3, false><<<gr, kAdvBlock, 0, st>>>(d, g); break;
      default: k_advect<6, 4, false><<<gr, kAdvBlock, 0, st>>>(d, g); break;
    }
  }
  return cudaGetLastError();
}

}  // namespace

// One advection step of length dt with the FP64 velocity vel: Euler (DG0),
// Heun (DG1) or the Shu-Osher three-stage scheme (DG2).  T1, T2: scratch
// [2][n_a][ne] each (H part, then A part).
cudaError_t launch_advect_step(const DevState &d, const double *vel, double dt, double *T1,
                               double *T2, cudaStream_t st) {
  const size_t n = (size_t)d.na * d.ne;
  AdvArgs g;
  g.vel = vel;
  g.dt = dt;
  g.H0 = d.H;
  g.A0 = d.A;
  // stage 1: T1 = U0 + dt L(U0)
  g.Hin = d.H;
  g.Ain = d.A;
  g.Hout = T1;
  g.Aout = T1 + n;
  g.a = 0.0;
  g.b = 1.0;
  cudaError_t e = stage(d, g, st);
  if (e != cudaSuccess) return e;
  if (d.na == 1) {
    e = cudaMemcpyAsync(d.H, T1, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d.A, T1 + n, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    return e;
  }
  if (d.na == 3) {
    // U = U0/2 + (T1 + dt L(T1))/2, written in place (each thread reads only
    // its own U0 entries)
    g.Hin = T1;
    g.Ain = T1 + n;
    g.Hout = d.H;
    g.Aout = d.A;
    g.a = 0.5;
    g.b = 0.5;
    return stage(d, g, st);
  }
  // T2 = 3 U0/4 + (T1 + dt L(T1))/4
  g.Hin = T1;
  g.Ain = T1 + n;
  g.Hout = T2;
  g.Aout = T2 + n;
  g.a = 0.75;
  g.b = 0.25;
  e = stage(d, g, st);
  if (e != cudaSuccess) return e;
  // U = U0/3 + 2 (T2 + dt L(T2))/3, in place
  g.Hin = T2;
  g.Ain = T2 + n;
  g.Hout = d.H;
  g.Aout = d.A;
  g.a = 1.0 / 3.0;
  g.b = 2.0 / 3.0;
  return stage(d, g, st);
}

}  // namespace mevp
