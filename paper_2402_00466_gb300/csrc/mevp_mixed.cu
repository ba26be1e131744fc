// mevp_mixed.cu -- mixed-precision kernels of the mEVP momentum subcycle.
//
// Strain, viscosities and the stress relaxation run in FP32 (the paper's
// Sec. 4 FP32 experiment, taken to every element stage), while the state
// that accumulates over subcycles keeps FP64-level accuracy without any FP64
// instruction in the loop (GB300 issues FP64 at 1/58 of the FP32 rate):
//
//   * velocity is stored as compensated FP32 pairs (hi, lo), v = hi + lo;
//   * the element kernel forms nodal velocity differences against the
//     element-centre node from the pairs, (hi_j - hi_c) + (lo_j - lo_c), so
//     rigid-body motion cancels before the FP32 strain (the cancellation the
//     paper's FP32 run is exposed to);
//   * the node kernel sums the element forces with TwoSum (compensated FP32)
//     and updates the velocity in residual form: with A v^p = r the
//     implicit system of the velocity update, it solves A d = r - A v^{p-1}
//     in FP32 and adds v^p = v^{p-1} + d in compensated FP32, so the FP32
//     rounding only touches the small increment d.
//
// The stress state is FP32.  Boundary handling, the force gather order and
// the per-element algorithm are the same as in the FP64 kernels.
#include "mevp_elem.cuh"
#include "mevp_internal.cuh"
#include "mevp_ref.cuh"

namespace mevp {

namespace {

constexpr int kElemBlock = 128;
constexpr int kNodeBlock = 256;

// Error-free transformations (Knuth TwoSum, Dekker FastTwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

struct MixArgs {
  float ie, hainv, dmin2, fac;  // stress update
  float opb, fdt;               // 1 + beta, f dt (velocity update)
  int has_vo;
};

// Full element step of element (kx, ky) in FP32: strain from the velocity
// pairs, relaxed stress update (S32[cur] -> out), element forces.
template <int NS>
__device__ __forceinline__ void element_mix(const DevState &d, const MixArgs &a, int kx, int ky,
                                            int cur, bool write_S, float fx[9], float fy[9]) {
  const size_t K = (size_t)ky * d.nx + kx;
  const float hx = (float)__ldg(d.lines + kx), ihx = (float)__ldg(d.lines + d.nx + kx);
  const float hy = (float)__ldg(d.lines + 2 * d.nx + ky);
  const float ihy = (float)__ldg(d.lines + 2 * d.nx + d.ny + ky);
  const float2 *__restrict__ vu = d.vel2[cur];
  const float2 *__restrict__ vv = d.vel2[cur] + d.nn;
  const size_t base = (size_t)(2 * ky) * d.nw + 2 * kx;
  float2 pu[9], pv[9];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pu[c + 3 * b] = __ldg(vu + base + (size_t)b * d.nw + c);
      pv[c + 3 * b] = __ldg(vv + base + (size_t)b * d.nw + c);
    }
  float du[9], dv[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    du[j] = __fsub_rn(pu[j].x, pu[4].x) + __fsub_rn(pu[j].y, pu[4].y);
    dv[j] = __fsub_rn(pv[j].x, pv[4].x) + __fsub_rn(pv[j].y, pv[4].y);
  }
  float Pc[NS], Qc[NS], Gc[NS];
  strain_invariants<NS>(du, dv, ihx, ihy, a.ie, Pc, Qc, Gc);
  const float *__restrict__ Sin = d.S32[cur];
  float S11[NS], S12[NS], S22[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    S11[s] = __ldg(Sin + (size_t)(0 * NS + s) * d.ne + K);
    S12[s] = __ldg(Sin + (size_t)(1 * NS + s) * d.ne + K);
    S22[s] = __ldg(Sin + (size_t)(2 * NS + s) * d.ne + K);
  }
  const float Ph = __ldg(d.Pe32 + K) * a.hainv;
  relax_stress<NS>(S11, S12, S22, Pc, Qc, Gc, Ph, a.dmin2, a.fac, a.ie);
  if (write_S) {
    float *__restrict__ Sout = d.S32[cur ^ 1];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Sout[(size_t)(0 * NS + s) * d.ne + K] = S11[s];
      Sout[(size_t)(1 * NS + s) * d.ne + K] = S12[s];
      Sout[(size_t)(2 * NS + s) * d.ne + K] = S22[s];
    }
  }
  element_forces_t<NS>(S11, S12, S22, hx, hy, fx, fy);
}

template <int NS>
__global__ void __launch_bounds__(kElemBlock) k_element_mix(DevState d, MixArgs a, int cur) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= d.ne) return;
  const int ky = K / d.nx, kx = K - ky * d.nx;
  float fx[9], fy[9];
  element_mix<NS>(d, a, kx, ky, cur, true, fx, fy);
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    d.fbuf32[(size_t)j * d.ne + K] = fx[j];
    d.fbuf32[(size_t)(9 + j) * d.ne + K] = fy[j];
  }
}

// Compensated sum of up to four FP32 element contributions in the fixed
// order SW, SE, NW, NE: returns hi + lo.
__device__ __forceinline__ void csum(const float *t, int n, float &hi, float &lo) {
  hi = t[0];
  lo = 0.0f;
#pragma unroll
  for (int i = 1; i < 4; ++i) {
    if (i < n) {
      float e;
      two_sum(hi, t[i], hi, e);
      lo = __fadd_rn(lo, e);
    }
  }
}

// Mixed velocity update at an interior node, residual form (see file header):
//   a = m(1+beta)/dt + c, b = m f, c = l Cw rho_w |v_o - v|,
//   r' = (q - (m/dt) v) + F + c (v_o - v) + b (v_y, -v_x),  q = (m/dt) v^n + l tau,
//   (a + i b) d = r',  v <- v + d (compensated).
__device__ __forceinline__ void node_update_mix(const DevState &d, const MixArgs &ma, int cur,
                                                size_t node, const float tx[4],
                                                const float ty[4], int n) {
  const size_t nn = d.nn;
  const float2 *__restrict__ vp = d.vel2[cur];
  float2 *__restrict__ vq = d.vel2[cur ^ 1];
  float Fxh, Fxl, Fyh, Fyl;
  csum(tx, n, Fxh, Fxl);
  csum(ty, n, Fyh, Fyl);
  const float2 ux = vp[node], uy = vp[nn + node];
  const float mdt = __ldg(d.nodec32 + 0 * nn + node);
  const float qx = __ldg(d.nodec32 + 1 * nn + node), qy = __ldg(d.nodec32 + 2 * nn + node);
  const float cD = __ldg(d.nodec32 + 3 * nn + node);
  float ox = 0.f, oy = 0.f;
  if (ma.has_vo) {
    const float2 o = __ldg(d.vo2 + node);
    ox = o.x;
    oy = o.y;
  }
  const float rx0 = (ox - ux.x) - ux.y, ry0 = (oy - uy.x) - uy.y;
  const float c = cD * sqrtf(fmaf(rx0, rx0, ry0 * ry0));
  const float a = fmaf(mdt, ma.opb, c);
  const float b = mdt * ma.fdt;
  float rx = (qx - fmaf(mdt, ux.x, mdt * ux.y)) + Fxh;
  rx = fmaf(c, rx0, rx + Fxl);
  rx = fmaf(b, uy.x, rx);
  float ry = (qy - fmaf(mdt, uy.x, mdt * uy.y)) + Fyh;
  ry = fmaf(c, ry0, ry + Fyl);
  ry = fmaf(-b, ux.x, ry);
  const float det = fmaf(a, a, b * b);
  float2 nx, ny;
  if (det > 0.f) {
    const float inv = 1.0f / det;
    const float ddx = fmaf(a, rx, b * ry) * inv;
    const float ddy = fmaf(a, ry, -b * rx) * inv;
    float s, e;
    two_sum(ux.x, ddx, s, e);
    fast_two_sum(s, __fadd_rn(ux.y, e), nx.x, nx.y);
    two_sum(uy.x, ddy, s, e);
    fast_two_sum(s, __fadd_rn(uy.y, e), ny.x, ny.y);
  } else {
    nx = make_float2(0.f, 0.f);
    ny = make_float2(0.f, 0.f);
  }
  vq[node] = nx;
  vq[nn + node] = ny;
}

__global__ void __launch_bounds__(kNodeBlock) k_node_mix(DevState d, MixArgs ma, int cur) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  const int sw = d.nx + 1;
  if (slot >= sw * (d.ny + 1)) return;
  const int ky = slot / sw, kx = slot - ky * sw;
  float2 *__restrict__ vq = d.vel2[cur ^ 1];
  const size_t nn = d.nn;
  const size_t ne = d.ne;
  const float *__restrict__ fb = d.fbuf32;
#pragma unroll
  for (int dy = 0; dy < 2; ++dy) {
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const int ix = 2 * kx + dx, iy = 2 * ky + dy;
      if (ix >= d.nw || iy >= d.nh) continue;
      const size_t node = (size_t)iy * d.nw + ix;
      if (ix == 0 || iy == 0 || ix == d.nw - 1 || iy == d.nh - 1) {
        vq[node] = make_float2(0.f, 0.f);
        vq[nn + node] = make_float2(0.f, 0.f);
        continue;
      }
      float tx[4] = {0.f, 0.f, 0.f, 0.f}, ty[4] = {0.f, 0.f, 0.f, 0.f};
      int n;
      if (dx == 0 && dy == 0) {
        const size_t Ksw = (size_t)(ky - 1) * d.nx + kx - 1, Kse = Ksw + 1;
        const size_t Knw = (size_t)ky * d.nx + kx - 1, Kne = Knw + 1;
        tx[0] = __ldg(fb + 8 * ne + Ksw); tx[1] = __ldg(fb + 6 * ne + Kse);
        tx[2] = __ldg(fb + 2 * ne + Knw); tx[3] = __ldg(fb + 0 * ne + Kne);
        ty[0] = __ldg(fb + 17 * ne + Ksw); ty[1] = __ldg(fb + 15 * ne + Kse);
        ty[2] = __ldg(fb + 11 * ne + Knw); ty[3] = __ldg(fb + 9 * ne + Kne);
        n = 4;
      } else if (dx == 1 && dy == 0) {
        const size_t Ks = (size_t)(ky - 1) * d.nx + kx, Kn = (size_t)ky * d.nx + kx;
        tx[0] = __ldg(fb + 7 * ne + Ks); tx[1] = __ldg(fb + 1 * ne + Kn);
        ty[0] = __ldg(fb + 16 * ne + Ks); ty[1] = __ldg(fb + 10 * ne + Kn);
        n = 2;
      } else if (dx == 0 && dy == 1) {
        const size_t Kw = (size_t)ky * d.nx + kx - 1, Ke = Kw + 1;
        tx[0] = __ldg(fb + 5 * ne + Kw); tx[1] = __ldg(fb + 3 * ne + Ke);
        ty[0] = __ldg(fb + 14 * ne + Kw); ty[1] = __ldg(fb + 12 * ne + Ke);
        n = 2;
      } else {
        const size_t K = (size_t)ky * d.nx + kx;
        tx[0] = __ldg(fb + 4 * ne + K);
        ty[0] = __ldg(fb + 13 * ne + K);
        n = 1;
      }
      node_update_mix(d, ma, cur, node, tx, ty, n);
    }
  }
}

// One fused subcycle.  A CTA takes a FTX x FTY block of elements: the
// (FTX-1) x (FTY-1) elements it owns plus one halo column to the west and one
// halo row to the south, recomputed from S^{p-1} and v^{p-1} so that every
// node the CTA owns -- ix in [2 x0, 2 x0 + 2(FTX-1)), iy likewise, plus the
// last boundary row/column of the domain -- sees all of its element forces
// without any exchange.  Forces go through shared memory; the stress is
// ping-ponged (halo readers need S^{p-1}).  Arithmetic is identical to the
// two-kernel path, element for element and node for node.
constexpr int FTX = 32, FTY = 16;

template <int NS>
__global__ void __launch_bounds__(FTX *FTY) k_subcycle_mix(DevState d, MixArgs ma, int cur) {
  __shared__ float fs[18][FTY][FTX];
  const int lx = threadIdx.x, ly = threadIdx.y;
  const int x0 = blockIdx.x * (FTX - 1), y0 = blockIdx.y * (FTY - 1);
  const int kx = x0 - 1 + lx, ky = y0 - 1 + ly;
  const bool active = kx >= 0 && ky >= 0 && kx < d.nx && ky < d.ny;
  float fx[9], fy[9];
  if (active) {
    element_mix<NS>(d, ma, kx, ky, cur, lx >= 1 && ly >= 1, fx, fy);
  } else {
#pragma unroll
    for (int j = 0; j < 9; ++j) fx[j] = fy[j] = 0.f;
  }
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    fs[j][ly][lx] = fx[j];
    fs[9 + j][ly][lx] = fy[j];
  }
  __syncthreads();
  const int ixs = 2 * x0, iys = 2 * y0;
  const int ixe = (x0 + FTX - 1 >= d.nx) ? d.nw : ixs + 2 * (FTX - 1);
  const int iye = (y0 + FTY - 1 >= d.ny) ? d.nh : iys + 2 * (FTY - 1);
  const int wx = ixe - ixs, wy = iye - iys;
  float2 *__restrict__ vq = d.vel2[cur ^ 1];
  const size_t nn = d.nn;
  for (int t = ly * FTX + lx; t < wx * wy; t += FTX * FTY) {
    const int ty_ = t / wx;
    const int ix = ixs + (t - ty_ * wx), iy = iys + ty_;
    const size_t node = (size_t)iy * d.nw + ix;
    if (ix == 0 || iy == 0 || ix == d.nw - 1 || iy == d.nh - 1) {
      vq[node] = make_float2(0.f, 0.f);
      vq[nn + node] = make_float2(0.f, 0.f);
      continue;
    }
    // local tile coordinates of the element whose lower-left node is (ix, iy)
    const int ex = (ix >> 1) - x0 + 1, ey = (iy >> 1) - y0 + 1;
    float tx[4] = {0.f, 0.f, 0.f, 0.f}, tyv[4] = {0.f, 0.f, 0.f, 0.f};
    int n;
    const bool odd_x = ix & 1, odd_y = iy & 1;
    if (!odd_x && !odd_y) {  // vertex: SW, SE, NW, NE
      tx[0] = fs[8][ey - 1][ex - 1]; tx[1] = fs[6][ey - 1][ex];
      tx[2] = fs[2][ey][ex - 1];     tx[3] = fs[0][ey][ex];
      tyv[0] = fs[17][ey - 1][ex - 1]; tyv[1] = fs[15][ey - 1][ex];
      tyv[2] = fs[11][ey][ex - 1];     tyv[3] = fs[9][ey][ex];
      n = 4;
    } else if (odd_x && !odd_y) {  // horizontal edge: S, N
      tx[0] = fs[7][ey - 1][ex]; tx[1] = fs[1][ey][ex];
      tyv[0] = fs[16][ey - 1][ex]; tyv[1] = fs[10][ey][ex];
      n = 2;
    } else if (!odd_x && odd_y) {  // vertical edge: W, E
      tx[0] = fs[5][ey][ex - 1]; tx[1] = fs[3][ey][ex];
      tyv[0] = fs[14][ey][ex - 1]; tyv[1] = fs[12][ey][ex];
      n = 2;
    } else {  // centre
      tx[0] = fs[4][ey][ex];
      tyv[0] = fs[13][ey][ex];
      n = 1;
    }
    node_update_mix(d, ma, cur, node, tx, tyv, n);
  }
}

// ---- conversions between the FP64 staging buffers and the FP32 state ----
// v (FP64) -> (hi, lo) with hi = fl32(v), lo = fl32(v - hi).
__global__ void k_vel_split(DevState d, int cur) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * (size_t)d.nn) return;
  const double v = d.vel[cur][i];
  const float hi = __double2float_rn(v);
  const float lo = __double2float_rn(v - (double)hi);
  d.vel2[cur][i] = make_float2(hi, lo);
}

__global__ void k_vel_join(DevState d, int cur) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * (size_t)d.nn) return;
  const float2 p = d.vel2[cur][i];
  d.vel[cur][i] = (double)p.x + (double)p.y;
}

__global__ void k_stress_to_f32(DevState d, int cur) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * (size_t)d.ns * d.ne) return;
  d.S32[cur][i] = __double2float_rn(d.S[i]);
}

__global__ void k_stress_to_f64(DevState d, int cur) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * (size_t)d.ns * d.ne) return;
  d.S[i] = (double)d.S32[cur][i];
}

// FP32 copies of the per-outer-step constants (computed in FP64 by the
// shared preparation kernels): m/dt, q = (m/dt) v^n + l tau, l Cw rho_w,
// ice strength, ocean velocity.
__global__ void k_consts_to_f32(DevState d, double dt, int has_vo) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nn = d.nn;
  if (i < nn) {
    d.nodec32[0 * nn + i] = __double2float_rn(d.mass[i] / dt);
    d.nodec32[1 * nn + i] = __double2float_rn(d.nodec[3 * nn + i]);
    d.nodec32[2 * nn + i] = __double2float_rn(d.nodec[4 * nn + i]);
    d.nodec32[3 * nn + i] = __double2float_rn(d.nodec[5 * nn + i]);
    if (has_vo)
      d.vo2[i] = make_float2(__double2float_rn(d.vo[i]), __double2float_rn(d.vo[nn + i]));
  }
  if (i < (size_t)d.ne) d.Pe32[i] = __double2float_rn(d.Pe[i]);
}

inline int blocks(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_vel_split(const DevState &d, int cur, cudaStream_t st) {
  k_vel_split<<<blocks(2LL * d.nn, 256), 256, 0, st>>>(d, cur);
  return cudaGetLastError();
}

cudaError_t launch_vel_join(const DevState &d, int cur, cudaStream_t st) {
  k_vel_join<<<blocks(2LL * d.nn, 256), 256, 0, st>>>(d, cur);
  return cudaGetLastError();
}

cudaError_t launch_stress_to_f32(const DevState &d, int cur, cudaStream_t st) {
  k_stress_to_f32<<<blocks(3LL * d.ns * d.ne, 256), 256, 0, st>>>(d, cur);
  return cudaGetLastError();
}

cudaError_t launch_stress_to_f64(const DevState &d, int cur, cudaStream_t st) {
  k_stress_to_f64<<<blocks(3LL * d.ns * d.ne, 256), 256, 0, st>>>(d, cur);
  return cudaGetLastError();
}

cudaError_t launch_prepare_mixed(const DevState &d, const mevp_params &p, bool has_vo, int cur,
                                 cudaStream_t st) {
  k_vel_join<<<blocks(2LL * d.nn, 256), 256, 0, st>>>(d, cur);
  cudaError_t e = launch_prepare(d, p, has_vo, cur, st);
  if (e != cudaSuccess) return e;
  const long long n = d.nn > d.ne ? d.nn : d.ne;
  k_consts_to_f32<<<blocks(n, 256), 256, 0, st>>>(d, p.dt, has_vo ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_subcycle_mixed(const DevState &d, const Rheo &r, const mevp_params &p,
                                  bool has_vo, int cur, cudaStream_t st, cudaEvent_t *ev,
                                  bool fused) {
  MixArgs a;
  a.ie = (float)r.ie;
  a.hainv = (float)r.hainv;
  a.dmin2 = (float)r.dmin2;
  a.fac = (float)r.fac;
  a.opb = (float)(1.0 + p.beta);
  a.fdt = (float)(p.coriolis_f * p.dt);
  a.has_vo = has_vo ? 1 : 0;
  if (ev) cudaEventRecord(ev[0], st);
  if (fused) {
    const dim3 grid((d.nx + FTX - 2) / (FTX - 1), (d.ny + FTY - 2) / (FTY - 1));
    const dim3 block(FTX, FTY);
    if (d.ns == 3)
      k_subcycle_mix<3><<<grid, block, 0, st>>>(d, a, cur);
    else
      k_subcycle_mix<6><<<grid, block, 0, st>>>(d, a, cur);
    if (ev) cudaEventRecord(ev[1], st);
    if (ev) cudaEventRecord(ev[2], st);
    return cudaGetLastError();
  }
  if (d.ns == 3)
    k_element_mix<3><<<blocks(d.ne, kElemBlock), kElemBlock, 0, st>>>(d, a, cur);
  else
    k_element_mix<6><<<blocks(d.ne, kElemBlock), kElemBlock, 0, st>>>(d, a, cur);
  if (ev) cudaEventRecord(ev[1], st);
  const long long slots = (long long)(d.nx + 1) * (d.ny + 1);
  k_node_mix<<<blocks(slots, kNodeBlock), kNodeBlock, 0, st>>>(d, a, cur);
  if (ev) cudaEventRecord(ev[2], st);
  return cudaGetLastError();
}

}  // namespace mevp
