// mevp_mixed.cu -- mixed-precision kernels of the mEVP momentum subcycle.
//
// Strain, viscosities and the stress relaxation run in FP32 (the paper's
// Sec. 4 FP32 experiment, taken to every element stage), while the state
// that accumulates over subcycles keeps FP64-level accuracy without any FP64
// instruction in the loop (GB300 issues FP64 at 1/58 of the FP32 rate):
//
//   * velocity is stored as compensated FP32 pairs (hi, lo), v = hi + lo,
//     one 16-byte record (u_hi, u_lo, v_hi, v_lo) per node;
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
//
// Default launch: one fused kernel per subcycle (k_subcycle_mix).  A CTA
// computes the element stage for its tile plus a one-element halo,
// exchanges forces through shared memory and updates the nodes it owns.  The
// two-kernel variant (k_element_mix + k_node_mix) does the same arithmetic
// through a global force buffer.
#include "mevp_elem.cuh"
#include "mevp_geom.cuh"
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

// Asynchronous global -> shared copies (16 bytes, L2 only).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Tensor-memory-accelerator (TMA) copies of 3-D boxes into shared memory,
// completed on an mbarrier (transaction count in bytes).
__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  // make the initialised barrier visible to the copy engine
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return done != 0;
}
// Bounded wait for phase `parity`: false once `limit_ns` of the global timer
// have passed (or after 2^22 attempts, whichever comes first), so a copy that
// never completes cannot hang the kernel.  A staging copy normally lands in
// microseconds.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < (1 << 22); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
  return false;
}



// Element step in FP32 from the 9 nodal velocity records (u_hi, u_lo, v_hi,
// v_lo) and the element's stress (in/out): strain from pair differences
// against the centre node, relaxed stress update, element forces.
// The element's ice strength: P (DG0 H, A) or, with VAR, P at each Gauss
// point (DG1/DG2 H, A), both scaled by 1/(2 alpha).
template <int NS, bool VAR> struct Strength {
  float Ph;
  float Phg[VAR ? DgSpace<NS>::NGP * DgSpace<NS>::NGP : 1];
};

template <int NS, bool VAR>
__device__ __forceinline__ Strength<NS, VAR> load_strength(const DevState &d, const MixArgs &a,
                                                           size_t K) {
  Strength<NS, VAR> p;
  if constexpr (VAR) {
    constexpr int NG = DgSpace<NS>::NGP * DgSpace<NS>::NGP;
    p.Ph = 0.f;
#pragma unroll
    for (int g = 0; g < NG; ++g)
      p.Phg[g] = ck_ldg(d.flags, (const float *)d.Pg32, (long long)g * d.ne + (long long)K,
                        (long long)NG * d.ne, 154) * a.hainv;
  } else {
    p.Ph = ck_ldg(d.flags, (const float *)d.Pe32, (long long)K, d.ne, 154) * a.hainv;
    p.Phg[0] = 0.f;
  }
  return p;
}

// Element geometry of the mixed kernels: mesh lines (rectangles), bilinear
// map records, or isoparametric node records.
constexpr int kGeoRect = 0, kGeoQuad = 1, kGeoIso = 2;

// The same element step on a general element: the map in FP32 from the
// per-element record of the preparation (bilinear QuadMapT, or the Jacobians
// at the Gauss points of an isoparametric element, IsoGeo), the local mass
// matrix factored per element (the FP64 general path's arithmetic in FP32).
template <int NS, bool VAR, typename G>
__device__ __forceinline__ void element_core_general(const float4 pv[9], float S11[NS],
                                                     float S12[NS], float S22[NS],
                                                     const Strength<NS, VAR> &P, const G &m,
                                                     const MassFactor<NS, float> &F,
                                                     const MixArgs &a, float fx[9], float fy[9]) {
  float du[9], dv[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    du[j] = __fsub_rn(pv[j].x, pv[4].x) + __fsub_rn(pv[j].y, pv[4].y);
    dv[j] = __fsub_rn(pv[j].z, pv[4].z) + __fsub_rn(pv[j].w, pv[4].w);
  }
  float Pc[NS], Qc[NS], Gc[NS];
  {
    float E11[NS], E22[NS], Esh[NS];
    strain_general<NS>(m, F, du, dv, E11, E22, Esh);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Pc[s] = E11[s] + E22[s];
      Qc[s] = a.ie * (E11[s] - E22[s]);
      Gc[s] = a.ie * Esh[s];
    }
  }
  relax_general<NS, VAR, float>(m, F, S11, S12, S22, Pc, Qc, Gc, P.Ph, a.dmin2, a.fac, a.ie,
                                P.Phg);
  forces_general<NS>(m, S11, S12, S22, fx, fy);
}

// FP32 map record of a general element: (Ax, Ay, Bx, By) and (cx, cy).
__device__ __forceinline__ QuadMapT<float> map_record(const DevState &d, size_t K) {
  const float4 ab = ck_ldg(d.flags, (const float4 *)d.map32ab, (long long)K, d.ne, 162);
  const float2 c = ck_ldg(d.flags, (const float2 *)d.map32c, (long long)K, d.ne, 162);
  QuadMapT<float> m;
  m.Ax = ab.x;
  m.Ay = ab.y;
  m.Bx = ab.z;
  m.By = ab.w;
  m.cx = c.x;
  m.cy = c.y;
  return m;
}

// FP32 node record of an isoparametric element: its 8 non-centre node
// positions minus the centre node's, as four float4 planes holding the node
// pairs (0,1), (2,3), (5,6), (7,8).  The centre node drops out of J because
// the Q2 reference gradients sum to zero, and the offsets (about h) keep FP32's
// relative precision where absolute coordinates (~5e5 m) would lose it.  The
// Jacobian at the N x N Gauss points goes to this thread's shared-memory
// column col[(q * N * N + g) * stride], as in the FP64 isoparametric kernel.
template <int N>
__device__ __forceinline__ IsoGeo<N, float> iso_record(const DevState &d, size_t K, float *col,
                                                       int stride) {
  constexpr int NG = N * N;
  float X[9], Y[9];
  const long long ne = d.ne, n4 = 4LL * d.ne;
  const float4 r0 = ck_ldg(d.flags, (const float4 *)d.iso32, (long long)K, n4, 163);
  const float4 r1 = ck_ldg(d.flags, (const float4 *)d.iso32, ne + (long long)K, n4, 163);
  const float4 r2 = ck_ldg(d.flags, (const float4 *)d.iso32, 2 * ne + (long long)K, n4, 163);
  const float4 r3 = ck_ldg(d.flags, (const float4 *)d.iso32, 3 * ne + (long long)K, n4, 163);
  X[0] = r0.x; Y[0] = r0.y; X[1] = r0.z; Y[1] = r0.w;
  X[2] = r1.x; Y[2] = r1.y; X[3] = r1.z; Y[3] = r1.w;
  X[4] = 0.f;  Y[4] = 0.f;
  X[5] = r2.x; Y[5] = r2.y; X[6] = r2.z; Y[6] = r2.w;
  X[7] = r3.x; Y[7] = r3.y; X[8] = r3.z; Y[8] = r3.w;
  {  // one coordinate at a time, to keep the live registers down
    float gxi[NG], geta[NG];
    ref_grad_gauss<N>(X, gxi, geta);
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      col[(0 * NG + g) * stride] = gxi[g];
      col[(1 * NG + g) * stride] = geta[g];
    }
  }
  float gxi[NG], geta[NG];
  ref_grad_gauss<N>(Y, gxi, geta);
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    col[(2 * NG + g) * stride] = gxi[g];
    col[(3 * NG + g) * stride] = geta[g];
  }
  return IsoGeo<N, float>{col, stride};
}

// FP32 L D L^T factor of the element's mass matrix from the records written
// once per outer step (the FP32 arithmetic of the element, done once).
template <int NS>
__device__ __forceinline__ MassFactor<NS, float> mass_record(const DevState &d, size_t K) {
  constexpr int NL = NS * (NS - 1) / 2;
  const long long ne = d.ne, n = (long long)mass_factor_words<NS>() * ne;
  MassFactor<NS, float> F;
#pragma unroll
  for (int i = 0; i < NL; ++i) F.L[i] = ck_ldg(d.flags, (const float *)d.mfac32, i * ne + (long long)K, n, 165);
#pragma unroll
  for (int i = 0; i < NS; ++i)
    F.Dinv[i] = ck_ldg(d.flags, (const float *)d.mfac32, (NL + i) * ne + (long long)K, n, 165);
  return F;
}

// Shared memory of the isoparametric Jacobian columns: 4 N^2 floats a thread.
template <int NS>
constexpr size_t iso_cols_bytes(int threads) {
  return sizeof(float) * 4 * DgSpace<NS>::NGP * DgSpace<NS>::NGP * threads;
}

template <int NS, bool VAR>
__device__ __forceinline__ void element_core(const float4 pv[9], float S11[NS], float S12[NS],
                                             float S22[NS], const Strength<NS, VAR> &P, float hx,
                                             float ihx, float hy, float ihy, const MixArgs &a,
                                             float fx[9], float fy[9]) {
  float du[9], dv[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    du[j] = __fsub_rn(pv[j].x, pv[4].x) + __fsub_rn(pv[j].y, pv[4].y);
    dv[j] = __fsub_rn(pv[j].z, pv[4].z) + __fsub_rn(pv[j].w, pv[4].w);
  }
  float Pc[NS], Qc[NS], Gc[NS];
  strain_invariants<NS>(du, dv, ihx, ihy, a.ie, Pc, Qc, Gc);
  relax_stress_p<NS, VAR, float>(S11, S12, S22, Pc, Qc, Gc, P.Ph, P.Phg, a.dmin2, a.fac, a.ie);
  element_forces_t<NS>(S11, S12, S22, hx, hy, fx, fy);
}

template <int NS>
__device__ __forceinline__ void load_stress(const DevState &d, int cur, size_t K, float S11[NS],
                                            float S12[NS], float S22[NS]) {
  const float *__restrict__ Sin = d.S32[cur];
  const long long n = 3LL * d.ns * d.ne;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    S11[s] = ck_ldg(d.flags, Sin, (long long)(0 * NS + s) * d.ne + (long long)K, n, 152);
    S12[s] = ck_ldg(d.flags, Sin, (long long)(1 * NS + s) * d.ne + (long long)K, n, 152);
    S22[s] = ck_ldg(d.flags, Sin, (long long)(2 * NS + s) * d.ne + (long long)K, n, 152);
  }
}

template <int NS>
__device__ __forceinline__ void store_stress(const DevState &d, int cur, size_t K,
                                             const float S11[NS], const float S12[NS],
                                             const float S22[NS]) {
  float *__restrict__ Sout = d.S32[cur ^ 1];
  const long long n = 3LL * d.ns * d.ne;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    ck_st(d.flags, Sout, (long long)(0 * NS + s) * d.ne + (long long)K, n, 153, S11[s]);
    ck_st(d.flags, Sout, (long long)(1 * NS + s) * d.ne + (long long)K, n, 153, S12[s]);
    ck_st(d.flags, Sout, (long long)(2 * NS + s) * d.ne + (long long)K, n, 153, S22[s]);
  }
}

__device__ __forceinline__ void line_geometry(const DevState &d, int kx, int ky, float &hx,
                                              float &ihx, float &hy, float &ihy) {
  const long long nl = (long long)d.nx + d.ny;
  const float2 gx = ck_ldg(d.flags, (const float2 *)d.lines32, kx, nl, 155);
  const float2 gy = ck_ldg(d.flags, (const float2 *)d.lines32, (long long)d.nx + ky, nl, 155);
  hx = gx.x;
  ihx = gx.y;
  hy = gy.x;
  ihy = gy.y;
}

template <int NS, bool VAR, int GEO>
__global__ void __launch_bounds__(kElemBlock) k_element_mix(DevState d, MixArgs a, int cur) {
  extern __shared__ float jcols[];  // isoparametric elements only
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= d.ne) return;
  const int ky = K / d.nx, kx = K - ky * d.nx;
  const float4 *__restrict__ vel = d.vel4[cur];
  const size_t base = (size_t)(2 * ky) * d.nw + 2 * kx;
  float4 pv[9];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      pv[c + 3 * b] = ck_ldg(d.flags, vel, (long long)(base + (size_t)b * d.nw + c), d.nn, 151);
  float S11[NS], S12[NS], S22[NS];
  load_stress<NS>(d, cur, K, S11, S12, S22);
  float fx[9], fy[9];
  if constexpr (GEO == kGeoIso) {
    const auto m = iso_record<DgSpace<NS>::NGP>(d, K, jcols + threadIdx.x, blockDim.x);
    element_core_general<NS, VAR>(pv, S11, S12, S22, load_strength<NS, VAR>(d, a, K), m,
                                  mass_record<NS>(d, K), a, fx, fy);
  } else if constexpr (GEO == kGeoQuad) {
    element_core_general<NS, VAR>(pv, S11, S12, S22, load_strength<NS, VAR>(d, a, K),
                                  map_record(d, K), mass_record<NS>(d, K), a, fx, fy);
  } else {
    float hx, ihx, hy, ihy;
    line_geometry(d, kx, ky, hx, ihx, hy, ihy);
    element_core<NS, VAR>(pv, S11, S12, S22, load_strength<NS, VAR>(d, a, K), hx, ihx, hy, ihy,
                          a, fx, fy);
  }
  store_stress<NS>(d, cur, K, S11, S12, S22);
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    ck_st(d.flags, d.fbuf32, (long long)j * d.ne + K, 18LL * d.ne, 158, fx[j]);
    ck_st(d.flags, d.fbuf32, (long long)(9 + j) * d.ne + K, 18LL * d.ne, 158, fy[j]);
  }
}

// Compensated sum of up to four FP32 element contributions in the fixed
// order SW, SE, NW, NE: returns hi + lo.
__device__ __forceinline__ void csum(const float2 *t, int n, float2 &hi, float2 &lo) {
  hi = t[0];
  lo = make_float2(0.f, 0.f);
#pragma unroll
  for (int i = 1; i < 4; ++i) {
    if (i < n) {
      float e;
      two_sum(hi.x, t[i].x, hi.x, e);
      lo.x = __fadd_rn(lo.x, e);
      two_sum(hi.y, t[i].y, hi.y, e);
      lo.y = __fadd_rn(lo.y, e);
    }
  }
}

// Mixed velocity update at an interior node, residual form (see file header):
//   a = m(1+beta)/dt + c, b = m f, c = l Cw rho_w |v_o - v|,
//   r' = (q - (m/dt) v) + F + c (v_o - v) + b (v_y, -v_x),  q = (m/dt) v^n + l tau,
//   (a + i b) d = r',  v <- v + d (compensated).
// v = (u_hi, u_lo, v_hi, v_lo), k = (m/dt, qx, qy, l Cw rho_w), t[n] = element
// force contributions (f_x, f_y).
__device__ __forceinline__ float4 node_update_mix(const MixArgs &ma, float4 v, float4 k,
                                                  float2 o, const float2 *t, int n) {
  float2 Fh, Fl;
  csum(t, n, Fh, Fl);
  const float mdt = k.x, qx = k.y, qy = k.z, cD = k.w;
  const float rx0 = (o.x - v.x) - v.y, ry0 = (o.y - v.z) - v.w;
  const float c = cD * sqrtf(fmaf(rx0, rx0, ry0 * ry0));
  const float a = fmaf(mdt, ma.opb, c);
  const float b = mdt * ma.fdt;
  float rx = (qx - fmaf(mdt, v.x, mdt * v.y)) + Fh.x;
  rx = fmaf(c, rx0, rx + Fl.x);
  rx = fmaf(b, v.z, rx);
  float ry = (qy - fmaf(mdt, v.z, mdt * v.w)) + Fh.y;
  ry = fmaf(c, ry0, ry + Fl.y);
  ry = fmaf(-b, v.x, ry);
  const float det = fmaf(a, a, b * b);
  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
  if (det > 0.f) {
    const float inv = 1.0f / det;
    const float ddx = fmaf(a, rx, b * ry) * inv;
    const float ddy = fmaf(a, ry, -b * rx) * inv;
    float s, e;
    two_sum(v.x, ddx, s, e);
    fast_two_sum(s, __fadd_rn(v.y, e), out.x, out.y);
    two_sum(v.z, ddy, s, e);
    fast_two_sum(s, __fadd_rn(v.w, e), out.z, out.w);
  }
  return out;
}

__device__ __forceinline__ float2 ocean(const DevState &d, const MixArgs &ma, size_t node) {
  return ma.has_vo ? ck_ldg(d.flags, (const float2 *)d.vo2, (long long)node, d.nn, 157)
                   : make_float2(0.f, 0.f);
}

__global__ void __launch_bounds__(kNodeBlock) k_node_mix(DevState d, MixArgs ma, int cur) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  const int sw = d.nx + 1;
  if (slot >= sw * (d.ny + 1)) return;
  const int ky = slot / sw, kx = slot - ky * sw;
  const float4 *__restrict__ vp = d.vel4[cur];
  float4 *__restrict__ vq = d.vel4[cur ^ 1];
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
        ck_st(d.flags, vq, (long long)node, d.nn, 161, make_float4(0.f, 0.f, 0.f, 0.f));
        continue;
      }
      float2 t[4];
      int n;
      auto F = [&](int j, size_t K) {
        return make_float2(ck_ldg(d.flags, fb, (long long)(j * ne + K), 18LL * ne, 158),
                           ck_ldg(d.flags, fb, (long long)((9 + j) * ne + K), 18LL * ne, 158));
      };
      if (dx == 0 && dy == 0) {
        const size_t Ksw = (size_t)(ky - 1) * d.nx + kx - 1, Kse = Ksw + 1;
        const size_t Knw = (size_t)ky * d.nx + kx - 1, Kne = Knw + 1;
        t[0] = F(8, Ksw); t[1] = F(6, Kse); t[2] = F(2, Knw); t[3] = F(0, Kne);
        n = 4;
      } else if (dx == 1 && dy == 0) {
        t[0] = F(7, (size_t)(ky - 1) * d.nx + kx); t[1] = F(1, (size_t)ky * d.nx + kx);
        n = 2;
      } else if (dx == 0 && dy == 1) {
        const size_t Kw = (size_t)ky * d.nx + kx - 1;
        t[0] = F(5, Kw); t[1] = F(3, Kw + 1);
        n = 2;
      } else {
        t[0] = F(4, (size_t)ky * d.nx + kx);
        n = 1;
      }
      ck_st(d.flags, vq, (long long)node, d.nn, 161,
            node_update_mix(ma, ck_ld(d.flags, vp, (long long)node, d.nn, 151),
                            ck_ldg(d.flags, (const float4 *)d.nodec4, (long long)node, d.nn, 156),
                            ocean(d, ma, node), t, n));
    }
  }
}

// ---- fused subcycle ---------------------------------------------------------
// A CTA takes a TX x TY block of elements: the (TX-1) x (TY-1) elements it
// owns plus one halo column to the west and one halo row to the south,
// recomputed from S^{p-1} and v^{p-1} so that every node the CTA owns -- ix in
// [2 x0, 2 x0 + 2(TX-1)), iy likewise, plus the last boundary row/column of
// the domain -- sees all of its element forces without an exchange.  The
// stress is ping-ponged (halo readers need S^{p-1}).
//
// The element stage loads straight from global memory, so each warp proceeds
// as soon as its own loads arrive (staging the whole tile into shared memory
// first, behind a barrier, measured slower: 106 vs 91 us per subcycle at
// 1024^2).  The owned nodes' velocity and constant records, needed only by
// the node stage, are copied into shared memory asynchronously from the start.
template <int TX, int TY> struct Tile {
  static constexpr int NW = 2 * (TX - 1), NH = 2 * (TY - 1);  // owned-node window
  // records per window, rounded up to 8 (128 bytes: a TMA destination)
  static constexpr int NWH = (NW * NH + 7) / 8 * 8;
  static constexpr size_t smem = sizeof(float4) * 2 * NWH + sizeof(float2) * 9 * TX * TY;
};

// Staging of the owned nodes' records.  TMA: one thread issues two tensor
// copies of the (NW x NH) window (velocity records of buffer cur, constant
// records) at the tile's first owned node; nodes past the domain read as
// zeros and are not used.  Otherwise (ensemble tiles, whose members each
// have their own buffers) every thread issues 16-byte cp.async copies.
struct TileMaps {
  const CUtensorMap *vel;   // velocity records of the current buffer, box {4, NW, NH}
  const CUtensorMap *cons;  // node-constant records, same box
};

template <int NS, int TX, int TY, bool VAR = false, int GEO = kGeoRect, bool TMA = false>
__device__ __forceinline__ void mix_tile(const DevState &d, const MixArgs &ma, int cur, int bx,
                                         int by, float4 *smem, TileMaps maps = {nullptr, nullptr},
                                         unsigned long long *bar = nullptr) {
  constexpr int TNW = Tile<TX, TY>::NW, TNH = Tile<TX, TY>::NH, NWH = Tile<TX, TY>::NWH;
  float4 *sv = smem;              // [TNH][TNW] velocity records of the owned nodes
  float4 *sk = sv + NWH;          // [TNH][TNW] constant records of the owned nodes
  float2(*fs)[TY][TX] = (float2(*)[TY][TX])(sk + NWH);  // [9][TY][TX] forces
  const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * TX + lx;
  const int x0 = bx * (TX - 1), y0 = by * (TY - 1);
  const int ixs = 2 * x0, iys = 2 * y0;
  const float4 *__restrict__ vel = d.vel4[cur];
  // The node stage's inputs do not depend on the element stage: start their
  // copies now, so that they arrive while the elements are computed.
  if constexpr (TMA) {
    if (tid == 0) {
      mbar_init(bar, 1);
      mbar_expect_tx(bar, 2u * (unsigned)(sizeof(float4) * TNW * TNH) + 16u * ma.stall);
      tma_load_3d(sv, maps.vel, 0, ixs, iys, bar);
      tma_load_3d(sk, maps.cons, 0, ixs, iys, bar);
    }
  } else {
    for (int i = tid; i < TNW * TNH; i += TX * TY) {
      const int r = i / TNW, c = i - r * TNW;
      const int gx = ixs + c, gy = iys + r;
      if (gx < d.nw && gy < d.nh) {
        const size_t node = (size_t)gy * d.nw + gx;
        cp_async16(sv + i, vel + node);
        cp_async16(sk + i, d.nodec4 + node);
      }
    }
    cp_async_commit();
  }
  const int kx = x0 - 1 + lx, ky = y0 - 1 + ly;
  const bool active = kx >= 0 && ky >= 0 && kx < d.nx && ky < d.ny;
  float2 f[9];
  if (active) {
    const size_t K = (size_t)ky * d.nx + kx;
    float S11[NS], S12[NS], S22[NS];
    load_stress<NS>(d, cur, K, S11, S12, S22);
    const Strength<NS, VAR> P = load_strength<NS, VAR>(d, ma, K);
    const size_t base = (size_t)(2 * ky) * d.nw + 2 * kx;
    float4 pv[9];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        pv[c + 3 * b] = ck_ldg(d.flags, vel, (long long)(base + (size_t)b * d.nw + c), d.nn, 151);
    float fx[9], fy[9];
    if constexpr (GEO == kGeoIso) {
      // Jacobian columns after the tile's own shared memory
      float *jc = (float *)((char *)smem + Tile<TX, TY>::smem) + tid;
      const auto m = iso_record<DgSpace<NS>::NGP>(d, K, jc, TX * TY);
      element_core_general<NS, VAR>(pv, S11, S12, S22, P, m, mass_record<NS>(d, K), ma, fx, fy);
    } else if constexpr (GEO == kGeoQuad) {
      element_core_general<NS, VAR>(pv, S11, S12, S22, P, map_record(d, K), mass_record<NS>(d, K),
                                    ma, fx, fy);
    } else {
      float hx, ihx, hy, ihy;
      line_geometry(d, kx, ky, hx, ihx, hy, ihy);
      element_core<NS, VAR>(pv, S11, S12, S22, P, hx, ihx, hy, ihy, ma, fx, fy);
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) f[j] = make_float2(fx[j], fy[j]);
    if (lx >= 1 && ly >= 1) store_stress<NS>(d, cur, K, S11, S12, S22);
  } else {
#pragma unroll
    for (int j = 0; j < 9; ++j) f[j] = make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int j = 0; j < 9; ++j) fs[j][ly][lx] = f[j];
  if constexpr (!TMA) cp_async_wait_all();
  __syncthreads();  // forces written; with TMA also: the barrier is initialised
  if constexpr (TMA) {
    if (!mbar_wait(bar, 0, 1000000000ull)) {
      // the copies did not complete within a second: report it, give them a
      // last bounded chance to land (they target this CTA's shared memory),
      // and skip the node stage; mevp_sync returns MEVP_ERR_TIMEOUT
      if (tid == 0) atomicExch(d.flags + 2, 1);
      mbar_wait(bar, 0, 100000000ull);
      return;
    }
  }
  const int ixe = (x0 + TX - 1 >= d.nx) ? d.nw : ixs + TNW;
  const int iye = (y0 + TY - 1 >= d.ny) ? d.nh : iys + TNH;
  float4 *__restrict__ vq = d.vel4[cur ^ 1];
  // interior window first (constant width: cheap index arithmetic) ...
  for (int t = tid; t < TNW * TNH; t += TX * TY) {
    const int r = t / TNW;
    const int ix = ixs + (t - r * TNW), iy = iys + r;
    if (ix >= ixe || iy >= iye) continue;
    const size_t node = (size_t)iy * d.nw + ix;
    if (ix == 0 || iy == 0 || ix == d.nw - 1 || iy == d.nh - 1) {
      ck_st(d.flags, vq, (long long)node, d.nn, 161, make_float4(0.f, 0.f, 0.f, 0.f));
      continue;
    }
    // local tile coordinates of the element whose lower-left node is (ix, iy)
    const int ex = (ix >> 1) - x0 + 1, ey = (iy >> 1) - y0 + 1;
    if (!ck_ok(d.flags, ex - 1, TX - 1, 159) || !ck_ok(d.flags, ey - 1, TY - 1, 159)) continue;
    float2 tf[4];
    int n;
    const bool odd_x = ix & 1, odd_y = iy & 1;
    if (!odd_x && !odd_y) {  // vertex: SW, SE, NW, NE
      tf[0] = fs[8][ey - 1][ex - 1]; tf[1] = fs[6][ey - 1][ex];
      tf[2] = fs[2][ey][ex - 1];     tf[3] = fs[0][ey][ex];
      n = 4;
    } else if (odd_x && !odd_y) {  // horizontal edge: S, N
      tf[0] = fs[7][ey - 1][ex]; tf[1] = fs[1][ey][ex];
      n = 2;
    } else if (!odd_x && odd_y) {  // vertical edge: W, E
      tf[0] = fs[5][ey][ex - 1]; tf[1] = fs[3][ey][ex];
      n = 2;
    } else {  // centre
      tf[0] = fs[4][ey][ex];
      n = 1;
    }
    ck_st(d.flags, vq, (long long)node, d.nn, 161,
          node_update_mix(ma, sv[t], sk[t], ocean(d, ma, node), tf, n));
  }
  // ... then the domain's last boundary column / row, owned by the last tiles
  if (ixe == d.nw)
    for (int iy = iys + tid; iy < iye; iy += TX * TY)
      ck_st(d.flags, vq, (long long)iy * d.nw + d.nw - 1, d.nn, 161,
            make_float4(0.f, 0.f, 0.f, 0.f));
  if (iye == d.nh)
    for (int ix = ixs + tid; ix < ixe; ix += TX * TY)
      ck_st(d.flags, vq, (long long)(d.nh - 1) * d.nw + ix, d.nn, 161,
            make_float4(0.f, 0.f, 0.f, 0.f));
}

// Single-domain tiles (elements per CTA, halo included), with 1024 threads
// per SM resident (64 registers a thread).  Measured at 1024^2 DG2 (us per
// subcycle): 32x8 82.7, 64x4 83.6, 32x4 84.0, 16x8 84.1, 32x16 87.8,
// 64x8 90.5, 32x32 100; at 256^2 the smaller 32x4 tiles win (12.4 vs 12.7 us)
// because 32x8 tiles no longer fill four rounds of CTAs per SM.
template <int NS, int TX, int TY, bool VAR>
__global__ void __launch_bounds__(TX *TY, 1024 / (TX * TY))
    k_subcycle_mix(DevState d, MixArgs ma, int cur, const __grid_constant__ CUtensorMap tmv,
                   const __grid_constant__ CUtensorMap tmk) {
  extern __shared__ __align__(128) float4 smem[];
  __shared__ unsigned long long bar;
  mix_tile<NS, TX, TY, VAR, kGeoRect, true>(d, ma, cur, blockIdx.x, blockIdx.y, smem,
                                            TileMaps{&tmv, &tmk}, &bar);
}

// General (bilinear) elements: the mass solves need more registers, so 768
// threads per SM (80 registers a thread).  Measured with the stored FP32 mass
// factors (element-subcycles/s, 1024^2 / 256^2 wavy DG2): 768 threads
// 9.22e9 / 5.59e9, 1024 threads 9.22e9 / 5.23e9; factorising per element
// instead: 512 threads 8.14e9 / 4.81e9, 768 threads 8.65e9 / 5.17e9.
template <int NS, int TX, int TY, bool VAR>
__global__ void __launch_bounds__(TX *TY, 768 / (TX * TY))
    k_subcycle_mix_gen(DevState d, MixArgs ma, int cur, const __grid_constant__ CUtensorMap tmv,
                       const __grid_constant__ CUtensorMap tmk) {
  extern __shared__ __align__(128) float4 smem[];
  __shared__ unsigned long long bar;
  mix_tile<NS, TX, TY, VAR, kGeoQuad, true>(d, ma, cur, blockIdx.x, blockIdx.y, smem,
                                            TileMaps{&tmv, &tmk}, &bar);
}

// Isoparametric elements: as the bilinear kernel, with the Jacobians at the
// Gauss points in shared memory after the tile's buffers, at 512 threads per
// SM (128 registers): with 768 or 1024 threads the spills cost more than the
// occupancy gains (1024^2: 6.07e9 -> 5.35e9 / 4.29e9 element-subcycles/s).
template <int NS, int TX, int TY, bool VAR>
__global__ void __launch_bounds__(TX *TY, 512 / (TX * TY))
    k_subcycle_mix_iso(DevState d, MixArgs ma, int cur, const __grid_constant__ CUtensorMap tmv,
                       const __grid_constant__ CUtensorMap tmk) {
  extern __shared__ __align__(128) float4 smem[];
  __shared__ unsigned long long bar;
  mix_tile<NS, TX, TY, VAR, kGeoIso, true>(d, ma, cur, blockIdx.x, blockIdx.y, smem,
                                           TileMaps{&tmv, &tmk}, &bar);
}

template <int NS, int TX, int TY>
cudaError_t launch_fused(const DevState &d, const MixArgs &a, int cur, const MixMaps &mm,
                         cudaStream_t st) {
  if (mm.rows != TY) return cudaErrorInvalidValue;  // maps built for another tile shape
  const dim3 grid((d.nx + TX - 2) / (TX - 1), (d.ny + TY - 2) / (TY - 1));
  const size_t sm = Tile<TX, TY>::smem;
  const CUtensorMap &tv = mm.vel[cur], &tk = mm.cons;
  if (d.nxy) {
    const size_t smi = sm + iso_cols_bytes<NS>(TX * TY);
    if (d.na > 1)
      k_subcycle_mix_iso<NS, TX, TY, true><<<grid, dim3(TX, TY), smi, st>>>(d, a, cur, tv, tk);
    else
      k_subcycle_mix_iso<NS, TX, TY, false><<<grid, dim3(TX, TY), smi, st>>>(d, a, cur, tv, tk);
  } else if (d.xy) {
    if (d.na > 1)
      k_subcycle_mix_gen<NS, TX, TY, true><<<grid, dim3(TX, TY), sm, st>>>(d, a, cur, tv, tk);
    else
      k_subcycle_mix_gen<NS, TX, TY, false><<<grid, dim3(TX, TY), sm, st>>>(d, a, cur, tv, tk);
  } else if (d.na > 1) {
    k_subcycle_mix<NS, TX, TY, true><<<grid, dim3(TX, TY), sm, st>>>(d, a, cur, tv, tk);
  } else {
    k_subcycle_mix<NS, TX, TY, false><<<grid, dim3(TX, TY), sm, st>>>(d, a, cur, tv, tk);
  }
  return cudaGetLastError();
}

template <int NS, int TX, int TY>
cudaError_t fused_attribute() {
  const int sm = (int)Tile<TX, TY>::smem;
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_subcycle_mix<NS, TX, TY, false>, at, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_subcycle_mix<NS, TX, TY, true>, at, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_subcycle_mix_gen<NS, TX, TY, false>, at, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_subcycle_mix_gen<NS, TX, TY, true>, at, sm);
  const int smi = sm + (int)iso_cols_bytes<NS>(TX * TY);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_subcycle_mix_iso<NS, TX, TY, false>, at, smi);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_subcycle_mix_iso<NS, TX, TY, true>, at, smi);
  return e;
}

template <int TX, int TY>
cudaError_t fused_attributes() {
  cudaError_t e = fused_attribute<3, TX, TY>();
  if (e == cudaSuccess) e = fused_attribute<6, TX, TY>();
  if (e == cudaSuccess) e = fused_attribute<8, TX, TY>();
  return e;
}

// Ensemble: one persistent launch per subcycle over the (member, tile) work
// list of all members (largest work first).  Member m runs on velocity /
// stress buffer base_cur(m) ^ flip.
template <int TX, int TY>
__global__ void __launch_bounds__(TX *TY, 1024 / (TX * TY)) k_ens_mix(const EnsMember *__restrict__ mem,
                                                    const EnsWork *__restrict__ work, int nwork,
                                                    int flip) {
  extern __shared__ float4 smem[];
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const EnsWork it = work[w];
    const EnsMember &m = mem[it.member];
    const int cur = m.base_cur ^ flip;
    if (m.d.ns == 3)
      mix_tile<3, TX, TY>(m.d, m.ma, cur, it.tx, it.ty, smem);
    else
      mix_tile<6, TX, TY>(m.d, m.ma, cur, it.tx, it.ty, smem);
    __syncthreads();  // the next tile reuses the shared memory
  }
}

// ---- conversions between the FP64 staging buffers and the FP32 state ----
// v (FP64) -> (hi, lo) with hi = fl32(v), lo = fl32(v - hi).
__global__ void k_vel_split(DevState d, int cur) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)d.nn) return;
  const double u = d.vel[cur][i], v = d.vel[cur][(size_t)d.nn + i];
  const float uh = __double2float_rn(u), vh = __double2float_rn(v);
  d.vel4[cur][i] = make_float4(uh, __double2float_rn(u - (double)uh), vh,
                               __double2float_rn(v - (double)vh));
}

__global__ void k_vel_join(DevState d, int cur) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)d.nn) return;
  const float4 p = d.vel4[cur][i];
  d.vel[cur][i] = (double)p.x + (double)p.y;
  d.vel[cur][(size_t)d.nn + i] = (double)p.z + (double)p.w;
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
    d.nodec4[i] = make_float4(__double2float_rn(d.mass[i] / dt),
                              __double2float_rn(d.nodec[3 * nn + i]),
                              __double2float_rn(d.nodec[4 * nn + i]),
                              __double2float_rn(d.nodec[5 * nn + i]));
    if (has_vo)
      d.vo2[i] = make_float2(__double2float_rn(d.vo[i]), __double2float_rn(d.vo[nn + i]));
  }
  if (i < (size_t)d.ne) {
    d.Pe32[i] = __double2float_rn(d.Pe[i]);
    if (d.na > 1) {
      const int ng = d.ns == 3 ? 4 : 9;
      for (int g = 0; g < ng; ++g)
        d.Pg32[(size_t)g * d.ne + i] = __double2float_rn(d.Pg[(size_t)g * d.ne + i]);
    }
  }
  if (d.nxy && d.iso32 && i < (size_t)d.ne) {  // curved mesh: FP32 node offsets
    const int ky = (int)(i / d.nx), kx = (int)(i - (size_t)ky * d.nx);
    const long long base = (long long)(2 * ky) * d.nw + 2 * kx;
    double2 p[9];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a)
        p[a + 3 * b] = ck_ldg(d.flags, d.nxy, base + (long long)b * d.nw + a, d.nn, 164);
    float o[18];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      o[2 * q] = __double2float_rn(p[q].x - p[4].x);
      o[2 * q + 1] = __double2float_rn(p[q].y - p[4].y);
    }
    d.iso32[i] = make_float4(o[0], o[1], o[2], o[3]);
    d.iso32[(size_t)d.ne + i] = make_float4(o[4], o[5], o[6], o[7]);
    d.iso32[2 * (size_t)d.ne + i] = make_float4(o[10], o[11], o[12], o[13]);
    d.iso32[3 * (size_t)d.ne + i] = make_float4(o[14], o[15], o[16], o[17]);
  }
  if (d.xy && i < (size_t)d.ne) {  // general mesh: FP32 map record per element
    const int ky = (int)(i / d.nx), kx = (int)(i - (size_t)ky * d.nx);
    const QuadMap m = quad_map(d.xy, d.nx, kx, ky, d.flags, (long long)(d.nx + 1) * (d.ny + 1));
    d.map32ab[i] = make_float4(__double2float_rn(m.Ax), __double2float_rn(m.Ay),
                               __double2float_rn(m.Bx), __double2float_rn(m.By));
    d.map32c[i] = make_float2(__double2float_rn(m.cx), __double2float_rn(m.cy));
  }
  if (i < (size_t)d.nx)
    d.lines32[i] = make_float2(__double2float_rn(d.lines[i]), __double2float_rn(d.lines[d.nx + i]));
  if (i < (size_t)d.ny)
    d.lines32[d.nx + i] = make_float2(__double2float_rn(d.lines[2 * d.nx + i]),
                                      __double2float_rn(d.lines[2 * d.nx + d.ny + i]));
}

inline int blocks(long long n, int b) { return (int)((n + b - 1) / b); }

// FP32 mass-factor records of a general or curved mixed state, once per outer
// step after the geometry records: the element's own FP32 factorisation
// (bilinear map record, or the Jacobians of the curved record in a local
// column), so the tile kernels read what they would have computed.
template <int NS>
__global__ void k_mass_records(DevState d) {
  constexpr int N = DgSpace<NS>::NGP;
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= d.ne) return;
  MassFactor<NS, float> F;
  if (d.nxy) {
    float col[4 * N * N];
    mass_factor<NS>(iso_record<N>(d, (size_t)K, col, 1), F);
  } else {
    mass_factor<NS>(map_record(d, (size_t)K), F);
  }
  constexpr int NL = NS * (NS - 1) / 2;
  const long long n = (long long)mass_factor_words<NS>() * d.ne;
  for (int i = 0; i < NL; ++i) ck_st(d.flags, d.mfac32, (long long)i * d.ne + K, n, 166, F.L[i]);
  for (int i = 0; i < NS; ++i)
    ck_st(d.flags, d.mfac32, (long long)(NL + i) * d.ne + K, n, 166, F.Dinv[i]);
}

}  // namespace

cudaError_t setup_mixed_kernels() {
  cudaError_t e = fused_attributes<32, 8>();
  if (e == cudaSuccess) e = fused_attributes<32, 4>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ens_mix<32, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Tile<32, 8>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ens_mix<32, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Tile<32, 4>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ens_mix<64, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Tile<64, 4>::smem);
  return e;
}

// Mixed ensemble tile shapes (TX, TY) the autotuner chooses from.
const int kMixTiles[kMixTileCount][2] = {{32, 8}, {32, 4}, {64, 4}};

int mixed_tile_count(int tile, int nx, int ny, int *tiles_x, int *tiles_y) {
  const int tx = kMixTiles[tile][0], ty = kMixTiles[tile][1];
  *tiles_x = (nx + tx - 2) / (tx - 1);
  *tiles_y = (ny + ty - 2) / (ty - 1);
  return *tiles_x * *tiles_y;
}

cudaError_t launch_ensemble_mixed(const EnsMember *mem, const EnsWork *work, int nwork, int tile,
                                  int grid, int flip, cudaStream_t st) {
  switch (tile) {
    case 0:
      k_ens_mix<32, 8><<<grid, dim3(32, 8), Tile<32, 8>::smem, st>>>(mem, work, nwork, flip);
      break;
    case 1:
      k_ens_mix<32, 4><<<grid, dim3(32, 4), Tile<32, 4>::smem, st>>>(mem, work, nwork, flip);
      break;
    default:
      k_ens_mix<64, 4><<<grid, dim3(64, 4), Tile<64, 4>::smem, st>>>(mem, work, nwork, flip);
      break;
  }
  return cudaGetLastError();
}

int mixed_tile_ctas_per_sm(int tile) {
  int n = 0;
  switch (tile) {
    case 0:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_mix<32, 8>, 256, Tile<32, 8>::smem);
      break;
    case 1:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_mix<32, 4>, 128, Tile<32, 4>::smem);
      break;
    default:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_mix<64, 4>, 256, Tile<64, 4>::smem);
      break;
  }
  return n > 0 ? n : 1;
}

cudaError_t launch_vel_split(const DevState &d, int cur, cudaStream_t st) {
  k_vel_split<<<blocks(d.nn, 256), 256, 0, st>>>(d, cur);
  return cudaGetLastError();
}

cudaError_t launch_vel_join(const DevState &d, int cur, cudaStream_t st) {
  k_vel_join<<<blocks(d.nn, 256), 256, 0, st>>>(d, cur);
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
  k_vel_join<<<blocks(d.nn, 256), 256, 0, st>>>(d, cur);
  cudaError_t e = launch_prepare(d, p, has_vo, cur, st);
  if (e != cudaSuccess) return e;
  long long n = d.nn > d.ne ? d.nn : d.ne;
  if (n < d.nx) n = d.nx;
  if (n < d.ny) n = d.ny;
  k_consts_to_f32<<<blocks(n, 256), 256, 0, st>>>(d, p.dt, has_vo ? 1 : 0);
  if (d.mfac32) {
    if (d.ns == 3)
      k_mass_records<3><<<blocks(d.ne, 128), 128, 0, st>>>(d);
    else if (d.ns == 6)
      k_mass_records<6><<<blocks(d.ne, 128), 128, 0, st>>>(d);
    else
      k_mass_records<8><<<blocks(d.ne, 128), 128, 0, st>>>(d);
  }
  return cudaGetLastError();
}

MixArgs make_mixargs(const Rheo &r, const mevp_params &p, bool has_vo) {
  MixArgs a;
  a.ie = (float)r.ie;
  a.hainv = (float)r.hainv;
  a.dmin2 = (float)r.dmin2;
  a.fac = (float)r.fac;
  a.opb = (float)(1.0 + p.beta);
  a.fdt = (float)(p.coriolis_f * p.dt);
  a.has_vo = has_vo ? 1 : 0;
  a.stall = 0;
  return a;
}

template <int NS, bool VAR>
void launch_element_mix_ns(const DevState &d, const MixArgs &a, int cur, cudaStream_t st) {
  const int eg = blocks(d.ne, kElemBlock);
  if (d.nxy)
    k_element_mix<NS, VAR, kGeoIso>
        <<<eg, kElemBlock, iso_cols_bytes<NS>(kElemBlock), st>>>(d, a, cur);
  else if (d.xy)
    k_element_mix<NS, VAR, kGeoQuad><<<eg, kElemBlock, 0, st>>>(d, a, cur);
  else
    k_element_mix<NS, VAR, kGeoRect><<<eg, kElemBlock, 0, st>>>(d, a, cur);
}

void launch_element_mix(const DevState &d, const MixArgs &a, int cur, cudaStream_t st) {
  const bool var = d.na > 1;
  if (d.ns == 3)
    var ? launch_element_mix_ns<3, true>(d, a, cur, st) : launch_element_mix_ns<3, false>(d, a, cur, st);
  else if (d.ns == 6)
    var ? launch_element_mix_ns<6, true>(d, a, cur, st) : launch_element_mix_ns<6, false>(d, a, cur, st);
  else
    var ? launch_element_mix_ns<8, true>(d, a, cur, st) : launch_element_mix_ns<8, false>(d, a, cur, st);
}

// Rows of the single-state fused tiles: 32x8 tiles once they fill four rounds
// of CTAs on every SM, else 32x4.
int mixed_tile_rows(const DevState &d) {
  const long long big = (long long)((d.nx + 29) / 31) * ((d.ny + 5) / 7);
  return big < 4LL * 4 * d.nsm ? 4 : 8;
}

cudaError_t make_mix_maps(const DevState &d, MixMaps *mm) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  // a node record is 4 floats; the window of a tile's owned nodes is
  // 2 (TX - 1) x 2 (TY - 1) records, TX = 32
  const int rows = mixed_tile_rows(d);
  const cuuint64_t dims[3] = {4, (cuuint64_t)d.nw, (cuuint64_t)d.nh};
  const cuuint64_t strides[2] = {sizeof(float4), sizeof(float4) * (cuuint64_t)d.nw};
  const cuuint32_t box[3] = {4, 2 * (32 - 1), (cuuint32_t)(2 * (rows - 1))};
  const cuuint32_t estr[3] = {1, 1, 1};
  void *bases[3] = {d.vel4[0], d.vel4[1], d.nodec4};
  CUtensorMap *maps[3] = {&mm->vel[0], &mm->vel[1], &mm->cons};
  for (int i = 0; i < 3; ++i) {
    const CUresult r = encode(maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, bases[i], dims,
                              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  mm->rows = rows;
  return cudaSuccess;
}

cudaError_t launch_subcycle_mixed(const DevState &d, const Rheo &r, const mevp_params &p,
                                  bool has_vo, int cur, cudaStream_t st, cudaEvent_t *ev,
                                  bool fused, const MixMaps &mm, int stall) {
  MixArgs a = make_mixargs(r, p, has_vo);
  a.stall = stall ? 1 : 0;
  if (ev) cudaEventRecord(ev[0], st);
  if (fused) {
    const bool small = mixed_tile_rows(d) == 4;
    cudaError_t e;
    if (d.ns == 3)
      e = small ? launch_fused<3, 32, 4>(d, a, cur, mm, st) : launch_fused<3, 32, 8>(d, a, cur, mm, st);
    else if (d.ns == 6)
      e = small ? launch_fused<6, 32, 4>(d, a, cur, mm, st) : launch_fused<6, 32, 8>(d, a, cur, mm, st);
    else
      e = small ? launch_fused<8, 32, 4>(d, a, cur, mm, st) : launch_fused<8, 32, 8>(d, a, cur, mm, st);
    if (ev) cudaEventRecord(ev[1], st);
    if (ev) cudaEventRecord(ev[2], st);
    return e;
  }
  launch_element_mix(d, a, cur, st);
  if (ev) cudaEventRecord(ev[1], st);
  const long long slots = (long long)(d.nx + 1) * (d.ny + 1);
  k_node_mix<<<blocks(slots, kNodeBlock), kNodeBlock, 0, st>>>(d, a, cur);
  if (ev) cudaEventRecord(ev[2], st);
  return cudaGetLastError();
}

}  // namespace mevp
