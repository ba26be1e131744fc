// mevp_general.cu -- FP64 element kernels of the mEVP subcycle on general
// (non-affine) quadrilateral meshes.
//
// k_element_gen does what k_element_f64 does on a rectilinear mesh (strain,
// stress update of Listing 1 / App. A, element forces of the weak
// divergence), with the bilinear element map evaluated on the fly from the
// four vertices (Sec. 3.2) and the local DG mass matrix factored per element
// (mevp_geom.cuh).  The node kernel (force gather in the fixed SW, SE, NW, NE
// order and the velocity update) is shared with the rectilinear path.
#include "mevp_geom.cuh"
#include "mevp_internal.cuh"

namespace mevp {

namespace {

constexpr int kGenBlock = 128;

// The element kernels of this file are persistent: the grid is the number of
// blocks that fit on the chip at once (queried at state creation), and each
// block takes an equal contiguous share of the element warps, which its warps
// walk in turn.  A grid of one block per 128 elements ends in a partial wave
// that leaves part of the chip idle (256x256: 512 blocks on 304 slots).
__device__ __forceinline__ void warp_share(int ne, int &w0, int &w1) {
  const int nwarps = (ne + 31) >> 5;
  w0 = (int)((long long)nwarps * blockIdx.x / gridDim.x);
  w1 = (int)((long long)nwarps * (blockIdx.x + 1) / gridDim.x);
}

// The element's mass factor from the records written at state creation.
template <int NS>
__device__ __forceinline__ void load_mass_factor(const DevState &d, int K, MassFactor<NS> &F) {
  constexpr int NL = NS * (NS - 1) / 2;
  const long long ne = d.ne, n = (long long)mass_factor_words<NS>() * ne;
#pragma unroll
  for (int i = 0; i < NL; ++i) F.L[i] = ck_ldg(d.flags, (const double *)d.mfac, i * ne + K, n, 145);
#pragma unroll
  for (int i = 0; i < NS; ++i)
    F.Dinv[i] = ck_ldg(d.flags, (const double *)d.mfac, (NL + i) * ne + K, n, 145);
}

// FP64 general and curved elements read the L D L^T factor of M_K (and a
// curved element its Jacobians) from records computed once per state: on
// this chip an FP64 operation costs about as much as 5 bytes of memory
// traffic, so the factorisation (with its divisions) and the curved map's
// 252-flop Jacobians are cheaper read than recomputed every subcycle.
template <int NS, bool VAR>
__device__ __forceinline__ void elem_gen(const DevState &d, const Rheo &r, int cur, int K) {
  const int ky = K / d.nx, kx = K - ky * d.nx;
  const QuadMap m = quad_map(d.xy, d.nx, kx, ky, d.flags, (long long)(d.nx + 1) * (d.ny + 1));
  MassFactor<NS> F;
  load_mass_factor<NS>(d, K, F);
  double Pc[NS], Qc[NS], Gc[NS];
  {
    double u[9], v[9];
    gather9(d.vel[cur], d.nw, kx, ky, u, d.flags, d.nn);
    gather9(d.vel[cur] + d.nn, d.nw, kx, ky, v, d.flags, d.nn);
    double E11[NS], E22[NS], Esh[NS];
    strain_general<NS>(m, F, u, v, E11, E22, Esh);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Pc[s] = E11[s] + E22[s];
      Qc[s] = r.ie * (E11[s] - E22[s]);
      Gc[s] = r.ie * Esh[s];
    }
  }
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
    relax_general<NS, true>(m, F, S11, S12, S22, Pc, Qc, Gc, 0.0, r.dmin2, r.fac, r.ie, Phg);
  } else {
    const double Ph = ck_ldg(d.flags, d.Pe, (long long)K, (long long)d.ne, 104) * r.hainv;
    relax_general<NS>(m, F, S11, S12, S22, Pc, Qc, Gc, Ph, r.dmin2, r.fac, r.ie);
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    ck_st(d.flags, d.S, (long long)(0 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 105, S11[s]);
    ck_st(d.flags, d.S, (long long)(1 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 105, S12[s]);
    ck_st(d.flags, d.S, (long long)(2 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 105, S22[s]);
  }
  double fx[9], fy[9];
  forces_general<NS>(m, S11, S12, S22, fx, fy);
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    ck_st(d.flags, d.fbuf, (long long)j * d.ne + K, 18LL * d.ne, 106, fx[j]);
    ck_st(d.flags, d.fbuf, (long long)(9 + j) * d.ne + K, 18LL * d.ne, 106, fy[j]);
  }
}

template <int NS, bool VAR>
__global__ void __launch_bounds__(kGenBlock) k_element_gen(DevState d, Rheo r, int cur) {
  int w0, w1;
  warp_share(d.ne, w0, w1);
  const int lane = threadIdx.x & 31;
  for (int w = w0 + (int)(threadIdx.x >> 5); w < w1; w += kGenBlock / 32) {
    const int K = (w << 5) + lane;
    if (K < d.ne) elem_gen<NS, VAR>(d, r, cur, K);
  }
}

// Strain coefficients E11, E12, E22 of the current velocity (read-back).
template <int NS>
__global__ void k_strain_diag_gen(DevState d, int cur) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= d.ne) return;
  const int ky = K / d.nx, kx = K - ky * d.nx;
  const QuadMap m = quad_map(d.xy, d.nx, kx, ky, d.flags, (long long)(d.nx + 1) * (d.ny + 1));
  MassFactor<NS> F;
  mass_factor<NS>(m, F);
  double u[9], v[9];
  gather9(d.vel[cur], d.nw, kx, ky, u, d.flags, d.nn);
  gather9(d.vel[cur] + d.nn, d.nw, kx, ky, v, d.flags, d.nn);
  double E11[NS], E22[NS], Esh[NS];
  strain_general<NS>(m, F, u, v, E11, E22, Esh);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    d.diag[(size_t)(0 * NS + s) * d.ne + K] = E11[s];
    d.diag[(size_t)(1 * NS + s) * d.ne + K] = 0.5 * Esh[s];
    d.diag[(size_t)(2 * NS + s) * d.ne + K] = E22[s];
  }
}

// Element forces of the current stress into the force buffer (read-back).
template <int NS>
__global__ void k_force_elem_gen(DevState d) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= d.ne) return;
  const int ky = K / d.nx, kx = K - ky * d.nx;
  const QuadMap m = quad_map(d.xy, d.nx, kx, ky, d.flags, (long long)(d.nx + 1) * (d.ny + 1));
  double S11[NS], S12[NS], S22[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    S11[s] = ck_ld(d.flags, d.S, (long long)(0 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 103);
    S12[s] = ck_ld(d.flags, d.S, (long long)(1 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 103);
    S22[s] = ck_ld(d.flags, d.S, (long long)(2 * NS + s) * d.ne + K, 3LL * d.ns * d.ne, 103);
  }
  double fx[9], fy[9];
  forces_general<NS>(m, S11, S12, S22, fx, fy);
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    ck_st(d.flags, d.fbuf, (long long)j * d.ne + K, 18LL * d.ne, 106, fx[j]);
    ck_st(d.flags, d.fbuf, (long long)(9 + j) * d.ne + K, 18LL * d.ne, 106, fy[j]);
  }
}

// ---- isoparametric (Q2) elements ------------------------------------------
constexpr int kIsoBlock = 128;

// The 9 CG2 node positions of element (kx, ky).
__device__ __forceinline__ void gather_nodes9(const DevState &d, int kx, int ky, double X[9],
                                              double Y[9]) {
  const long long base = (long long)(2 * ky) * d.nw + 2 * kx;
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 p = ck_ldg(d.flags, d.nxy, base + (long long)b * d.nw + a, d.nn, 143);
      X[a + 3 * b] = p.x;
      Y[a + 3 * b] = p.y;
    }
}

// Jacobian of the isoparametric map at the N x N Gauss points (reference
// gradients of the node positions), into this thread's shared-memory column.
template <int N>
__device__ __forceinline__ IsoGeo<N, double> iso_geometry(const DevState &d, int kx, int ky,
                                                          double *sm) {
  constexpr int NG = N * N;
  double X[9], Y[9];
  gather_nodes9(d, kx, ky, X, Y);
  double xxi[NG], xeta[NG], yxi[NG], yeta[NG];
  ref_grad_gauss<N>(X, xxi, xeta);
  ref_grad_gauss<N>(Y, yxi, yeta);
  const int stride = blockDim.x;
  double *col = sm + threadIdx.x;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    col[(0 * NG + g) * stride] = xxi[g];   // dx/dxi
    col[(1 * NG + g) * stride] = xeta[g];  // dx/deta
    col[(2 * NG + g) * stride] = yxi[g];   // dy/dxi
    col[(3 * NG + g) * stride] = yeta[g];  // dy/deta
  }
  return IsoGeo<N, double>{col, stride};
}

// The element's Jacobians at the Gauss points are read where they are used,
// from the records written at state creation (the [4 N^2][ne] array is sized
// for every K < ne, so these reads stay in bounds by construction).
template <int NS, bool VAR>
__device__ __forceinline__ void elem_iso(const DevState &d, const Rheo &r, int cur, int K) {
  constexpr int N = DgSpace<NS>::NGP;
  const int ky = K / d.nx, kx = K - ky * d.nx;
  const IsoGeoG<N, double> m{d.isoJ + K, (size_t)d.ne};
  MassFactor<NS> F;
  load_mass_factor<NS>(d, K, F);
  double Pc[NS], Qc[NS], Gc[NS];
  {
    double u[9], v[9];
    gather9(d.vel[cur], d.nw, kx, ky, u, d.flags, d.nn);
    gather9(d.vel[cur] + d.nn, d.nw, kx, ky, v, d.flags, d.nn);
    double E11[NS], E22[NS], Esh[NS];
    strain_general<NS>(m, F, u, v, E11, E22, Esh);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Pc[s] = E11[s] + E22[s];
      Qc[s] = r.ie * (E11[s] - E22[s]);
      Gc[s] = r.ie * Esh[s];
    }
  }
  double S11[NS], S12[NS], S22[NS];
  const long long nsd = 3LL * d.ns * d.ne;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    S11[s] = ck_ld(d.flags, d.S, (long long)(0 * NS + s) * d.ne + K, nsd, 103);
    S12[s] = ck_ld(d.flags, d.S, (long long)(1 * NS + s) * d.ne + K, nsd, 103);
    S22[s] = ck_ld(d.flags, d.S, (long long)(2 * NS + s) * d.ne + K, nsd, 103);
  }
  if constexpr (VAR) {
    constexpr int NG = N * N;
    double Phg[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g)
      Phg[g] = ck_ldg(d.flags, d.Pg, (long long)g * d.ne + K, (long long)NG * d.ne, 104) * r.hainv;
    relax_general<NS, true>(m, F, S11, S12, S22, Pc, Qc, Gc, 0.0, r.dmin2, r.fac, r.ie, Phg);
  } else {
    const double Ph = ck_ldg(d.flags, d.Pe, (long long)K, (long long)d.ne, 104) * r.hainv;
    relax_general<NS>(m, F, S11, S12, S22, Pc, Qc, Gc, Ph, r.dmin2, r.fac, r.ie);
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    ck_st(d.flags, d.S, (long long)(0 * NS + s) * d.ne + K, nsd, 105, S11[s]);
    ck_st(d.flags, d.S, (long long)(1 * NS + s) * d.ne + K, nsd, 105, S12[s]);
    ck_st(d.flags, d.S, (long long)(2 * NS + s) * d.ne + K, nsd, 105, S22[s]);
  }
  double fx[9], fy[9];
  forces_general<NS>(m, S11, S12, S22, fx, fy);
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    ck_st(d.flags, d.fbuf, (long long)j * d.ne + K, 18LL * d.ne, 106, fx[j]);
    ck_st(d.flags, d.fbuf, (long long)(9 + j) * d.ne + K, 18LL * d.ne, 106, fy[j]);
  }
}

template <int NS>
constexpr size_t iso_smem() {
  return sizeof(double) * 4 * DgSpace<NS>::NGP * DgSpace<NS>::NGP * kIsoBlock;
}

template <int NS, bool VAR>
__global__ void __launch_bounds__(kIsoBlock) k_element_iso(DevState d, Rheo r, int cur) {
  int w0, w1;
  warp_share(d.ne, w0, w1);
  const int lane = threadIdx.x & 31;
  for (int w = w0 + (int)(threadIdx.x >> 5); w < w1; w += kIsoBlock / 32) {
    const int K = (w << 5) + lane;
    if (K < d.ne) elem_iso<NS, VAR>(d, r, cur, K);
  }
}

template <int NS>
__global__ void __launch_bounds__(kIsoBlock) k_strain_diag_iso(DevState d, int cur) {
  extern __shared__ double iso_sm[];
  constexpr int N = DgSpace<NS>::NGP;
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= d.ne) return;
  const int ky = K / d.nx, kx = K - ky * d.nx;
  const IsoGeo<N, double> m = iso_geometry<N>(d, kx, ky, iso_sm);
  MassFactor<NS> F;
  mass_factor<NS>(m, F);
  double u[9], v[9];
  gather9(d.vel[cur], d.nw, kx, ky, u, d.flags, d.nn);
  gather9(d.vel[cur] + d.nn, d.nw, kx, ky, v, d.flags, d.nn);
  double E11[NS], E22[NS], Esh[NS];
  strain_general<NS>(m, F, u, v, E11, E22, Esh);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    d.diag[(size_t)(0 * NS + s) * d.ne + K] = E11[s];
    d.diag[(size_t)(1 * NS + s) * d.ne + K] = 0.5 * Esh[s];
    d.diag[(size_t)(2 * NS + s) * d.ne + K] = E22[s];
  }
}

template <int NS>
__global__ void __launch_bounds__(kIsoBlock) k_force_elem_iso(DevState d) {
  extern __shared__ double iso_sm[];
  constexpr int N = DgSpace<NS>::NGP;
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= d.ne) return;
  const int ky = K / d.nx, kx = K - ky * d.nx;
  const IsoGeo<N, double> m = iso_geometry<N>(d, kx, ky, iso_sm);
  double S11[NS], S12[NS], S22[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    S11[s] = d.S[(size_t)(0 * NS + s) * d.ne + K];
    S12[s] = d.S[(size_t)(1 * NS + s) * d.ne + K];
    S22[s] = d.S[(size_t)(2 * NS + s) * d.ne + K];
  }
  double fx[9], fy[9];
  forces_general<NS>(m, S11, S12, S22, fx, fy);
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    d.fbuf[(size_t)j * d.ne + K] = fx[j];
    d.fbuf[(size_t)(9 + j) * d.ne + K] = fy[j];
  }
}

inline int blocks(long long n, int b) { return (int)((n + b - 1) / b); }

// Per-element geometry records of an FP64 general (ISO = false) or curved
// mesh: the L D L^T factor of M_K, and for a curved element its Jacobians at
// the Gauss points, by the same functions the on-the-fly diagnostics use.
template <int NS, bool ISO>
__global__ void __launch_bounds__(kIsoBlock) k_geom_factors(DevState d) {
  extern __shared__ double iso_sm[];
  constexpr int N = DgSpace<NS>::NGP, NG = N * N;
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= d.ne) return;
  const int ky = K / d.nx, kx = K - ky * d.nx;
  MassFactor<NS> F;
  if constexpr (ISO) {
    const IsoGeo<N, double> m = iso_geometry<N>(d, kx, ky, iso_sm);
    mass_factor<NS>(m, F);
    for (int i = 0; i < 4 * NG; ++i)
      ck_st(d.flags, d.isoJ, (long long)i * d.ne + K, 4LL * NG * d.ne, 147, m.sJ[i * m.stride]);
  } else {
    const QuadMap m = quad_map(d.xy, d.nx, kx, ky, d.flags, (long long)(d.nx + 1) * (d.ny + 1));
    mass_factor<NS>(m, F);
  }
  constexpr int NL = NS * (NS - 1) / 2;
  const long long n = (long long)mass_factor_words<NS>() * d.ne;
  for (int i = 0; i < NL; ++i) ck_st(d.flags, d.mfac, (long long)i * d.ne + K, n, 148, F.L[i]);
  for (int i = 0; i < NS; ++i)
    ck_st(d.flags, d.mfac, (long long)(NL + i) * d.ne + K, n, 148, F.Dinv[i]);
}

template <int NS>
void launch_geom_factors_ns(const DevState &d, cudaStream_t st) {
  const int g = blocks(d.ne, kIsoBlock);
  if (d.nxy)
    k_geom_factors<NS, true><<<g, kIsoBlock, iso_smem<NS>(), st>>>(d);
  else
    k_geom_factors<NS, false><<<g, kIsoBlock, 0, st>>>(d);
}

// Resident blocks per SM of the persistent element kernels, [NS index][VAR];
// filled at state creation, 2 until then (the grid size only affects speed).
int g_gen_resident[3][2] = {{2, 2}, {2, 2}, {2, 2}};
int g_iso_resident[3][2] = {{2, 2}, {2, 2}, {2, 2}};

constexpr int ns_index(int ns) { return ns == 3 ? 0 : ns == 6 ? 1 : 2; }

inline int persistent_grid(const DevState &d, int resident, int block) {
  const int need = blocks(d.ne, block);
  const int fit = (resident > 0 ? resident : 1) * d.nsm;
  return need < fit ? need : fit;
}

template <class Kernel>
cudaError_t resident_blocks(Kernel k, int block, size_t smem, int &out) {
  int n = 0;
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, smem);
  if (e == cudaSuccess && n > 0) out = n;
  return e;
}

template <int NS, bool VAR>
void launch_iso_ns(const DevState &d, const Rheo &r, int cur, cudaStream_t st) {
  const int g = persistent_grid(d, g_iso_resident[ns_index(NS)][VAR], kIsoBlock);
  k_element_iso<NS, VAR><<<g, kIsoBlock, 0, st>>>(d, r, cur);
}

template <int NS, bool VAR>
void launch_gen_ns(const DevState &d, const Rheo &r, int cur, cudaStream_t st) {
  const int g = persistent_grid(d, g_gen_resident[ns_index(NS)][VAR], kGenBlock);
  k_element_gen<NS, VAR><<<g, kGenBlock, 0, st>>>(d, r, cur);
}

template <int NS, bool VAR>
cudaError_t setup_iso_ns() {
  return resident_blocks(k_element_iso<NS, VAR>, kIsoBlock, 0, g_iso_resident[ns_index(NS)][VAR]);
}

template <int NS, bool VAR>
cudaError_t setup_gen_ns() {
  return resident_blocks(k_element_gen<NS, VAR>, kGenBlock, 0, g_gen_resident[ns_index(NS)][VAR]);
}

}  // namespace

cudaError_t setup_iso_kernels() {
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = setup_iso_ns<3, false>();
  if (e == cudaSuccess) e = setup_iso_ns<3, true>();
  if (e == cudaSuccess) e = setup_iso_ns<6, false>();
  if (e == cudaSuccess) e = setup_iso_ns<6, true>();
  if (e == cudaSuccess) e = setup_iso_ns<8, false>();
  if (e == cudaSuccess) e = setup_iso_ns<8, true>();
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_strain_diag_iso<3>, at, (int)iso_smem<3>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_strain_diag_iso<6>, at, (int)iso_smem<6>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_strain_diag_iso<8>, at, (int)iso_smem<8>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_force_elem_iso<3>, at, (int)iso_smem<3>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_force_elem_iso<6>, at, (int)iso_smem<6>());
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_force_elem_iso<8>, at, (int)iso_smem<8>());
  return e;
}

cudaError_t launch_element_iso(const DevState &d, const Rheo &r, int cur, cudaStream_t st) {
  const bool var = d.na > 1;
  if (d.ns == 3)
    var ? launch_iso_ns<3, true>(d, r, cur, st) : launch_iso_ns<3, false>(d, r, cur, st);
  else if (d.ns == 6)
    var ? launch_iso_ns<6, true>(d, r, cur, st) : launch_iso_ns<6, false>(d, r, cur, st);
  else
    var ? launch_iso_ns<8, true>(d, r, cur, st) : launch_iso_ns<8, false>(d, r, cur, st);
  return cudaGetLastError();
}

cudaError_t launch_strain_diag_iso(const DevState &d, int cur, cudaStream_t st) {
  const int g = blocks(d.ne, kIsoBlock);
  if (d.ns == 3)
    k_strain_diag_iso<3><<<g, kIsoBlock, iso_smem<3>(), st>>>(d, cur);
  else if (d.ns == 6)
    k_strain_diag_iso<6><<<g, kIsoBlock, iso_smem<6>(), st>>>(d, cur);
  else
    k_strain_diag_iso<8><<<g, kIsoBlock, iso_smem<8>(), st>>>(d, cur);
  return cudaGetLastError();
}

cudaError_t launch_force_elem_iso(const DevState &d, cudaStream_t st) {
  const int g = blocks(d.ne, kIsoBlock);
  if (d.ns == 3)
    k_force_elem_iso<3><<<g, kIsoBlock, iso_smem<3>(), st>>>(d);
  else if (d.ns == 6)
    k_force_elem_iso<6><<<g, kIsoBlock, iso_smem<6>(), st>>>(d);
  else
    k_force_elem_iso<8><<<g, kIsoBlock, iso_smem<8>(), st>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_geom_factors(const DevState &d, cudaStream_t st) {
  if (d.ns == 3)
    launch_geom_factors_ns<3>(d, st);
  else if (d.ns == 6)
    launch_geom_factors_ns<6>(d, st);
  else
    launch_geom_factors_ns<8>(d, st);
  return cudaGetLastError();
}

cudaError_t setup_general_kernels() {
  cudaError_t e = setup_gen_ns<3, false>();
  if (e == cudaSuccess) e = setup_gen_ns<3, true>();
  if (e == cudaSuccess) e = setup_gen_ns<6, false>();
  if (e == cudaSuccess) e = setup_gen_ns<6, true>();
  if (e == cudaSuccess) e = setup_gen_ns<8, false>();
  if (e == cudaSuccess) e = setup_gen_ns<8, true>();
  return e;
}

cudaError_t launch_element_general(const DevState &d, const Rheo &r, int cur, cudaStream_t st) {
  const bool var = d.na > 1;
  if (d.ns == 3)
    var ? launch_gen_ns<3, true>(d, r, cur, st) : launch_gen_ns<3, false>(d, r, cur, st);
  else if (d.ns == 6)
    var ? launch_gen_ns<6, true>(d, r, cur, st) : launch_gen_ns<6, false>(d, r, cur, st);
  else
    var ? launch_gen_ns<8, true>(d, r, cur, st) : launch_gen_ns<8, false>(d, r, cur, st);
  return cudaGetLastError();
}

cudaError_t launch_strain_diag_general(const DevState &d, int cur, cudaStream_t st) {
  const int g = blocks(d.ne, 128);
  if (d.ns == 3)
    k_strain_diag_gen<3><<<g, 128, 0, st>>>(d, cur);
  else if (d.ns == 6)
    k_strain_diag_gen<6><<<g, 128, 0, st>>>(d, cur);
  else
    k_strain_diag_gen<8><<<g, 128, 0, st>>>(d, cur);
  return cudaGetLastError();
}

cudaError_t launch_force_elem_general(const DevState &d, cudaStream_t st) {
  const int g = blocks(d.ne, 128);
  if (d.ns == 3)
    k_force_elem_gen<3><<<g, 128, 0, st>>>(d);
  else if (d.ns == 6)
    k_force_elem_gen<6><<<g, 128, 0, st>>>(d);
  else
    k_force_elem_gen<8><<<g, 128, 0, st>>>(d);
  return cudaGetLastError();
}

}  // namespace mevp
