// mevp_internal.cuh -- internal data structures and kernel launchers.
#pragma once

#include <cuda.h>  // CUtensorMap (types only; the encoder is reached through the runtime)
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mevp.h"

namespace mevp {
// NVTX range over one C-ABI call (host side; shows the call in a profiler's
// timeline, free otherwise).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace mevp

struct mevp_mesh {
  int nx = 0, ny = 0;
  std::vector<double> xline;  // nx+1 vertex x coordinates (rectilinear mesh)
  std::vector<double> yline;  // ny+1 vertex y coordinates
  bool general = false;       // vertices not on a rectilinear grid
  std::vector<double> xy;     // general mesh: [(nx+1)(ny+1)][2] vertex coordinates
  bool iso = false;           // isoparametric: geometry from the CG2 node positions
  std::vector<double> nxy;    // isoparametric mesh: [(2nx+1)(2ny+1)][2] node positions
};

namespace mevp {

// Scalar constants of the stress update, derived once from mevp_params.
struct Rheo {
  double dmin2;  // Delta_min^2
  double k_sq;   // 1 + 1/e^2        (5/4 at e = 2)
  double k_mix;  // 2 (1 - 1/e^2)    (3/2)
  double k_sh;   // 4/e^2            (1)
  double c_a;    // (1 + 1/e^2)/2    (5/8)
  double c_b;    // (1 - 1/e^2)/2    (3/8)
  double c_s;    // 1/e^2            (1/4)
  double ainv;   // 1/alpha
  double fac;    // 1 - 1/alpha
  double ie;     // 1/e
  double hainv;  // 1/(2 alpha)
};

// Derive the stress-update constants from the parameters.
inline Rheo make_rheo(const mevp_params &p) {
  Rheo r{};
  const double ie2 = 1.0 / (p.e * p.e);
  r.dmin2 = p.DeltaMin * p.DeltaMin;
  r.k_sq = 1.0 + ie2;
  r.k_mix = 2.0 * (1.0 - ie2);
  r.k_sh = 4.0 * ie2;
  r.c_a = 0.5 * (1.0 + ie2);
  r.c_b = 0.5 * (1.0 - ie2);
  r.c_s = ie2;
  r.ainv = 1.0 / p.alpha;
  r.fac = 1.0 - r.ainv;
  r.ie = 1.0 / p.e;
  r.hainv = 0.5 / p.alpha;
  return r;
}

// Device view of a state (all pointers into the workspace).
struct DevState {
  int nx, ny, ne, nw, nh, nn, ns, prec;
  int na;              // DG dofs of H and A per element (1, 3 or 6)
  int nsm;             // SMs of the device (grid of the persistent kernels)
  const double *xline, *yline;
  const double2 *xy;   // general mesh: [(nx+1)(ny+1)] vertices; NULL on rectilinear meshes
  const double2 *nxy;  // isoparametric mesh: [nn] CG2 node positions; NULL otherwise
  double *lines;       // [hx: nx][1/hx: nx][hy: ny][1/hy: ny], from the mesh lines
  double *vel[2];      // [2][nn] ping-pong
  double *S;           // FP64: [3][ns][ne]
  float *S32[2];       // mixed: [3][ns][ne], ping-pong with the velocity
  double *H, *A;       // [ne]
  double *tau;         // [2][nn]
  double *vo;          // [2][nn]
  double *Pe;          // [ne] ice strength per element (DG0 H, A)
  double *Pg;          // [NGP^2][ne] ice strength per Gauss point (DG1/DG2 H, A)
  const double *pstar; // [ne] per-element P* field, or NULL (params.Pstar everywhere)
  double *nodec;       // [6][nn] cA, cB, cK, qx, qy, cD
  double *mass;        // [nn]
  double *fbuf;        // FP64: [18][ne] per-element nodal forces (scratch)
  float *fbuf32;       // mixed: [18][ne]
  double *diag;        // [3][ns][ne] or [2][nn] diagnostic output
  int *flags;          // [4] device status words: [0] non-finite velocity seen
  // mixed precision only (FP64 buffers above stage inputs and outputs)
  float4 *vel4[2];     // [nn] (u_hi, u_lo, v_hi, v_lo) records, ping-pong
  float *Pe32;         // [ne]
  float *Pg32;         // [NGP^2][ne] (DG1/DG2 H, A)
  float4 *map32ab;     // general mesh: [ne] (Ax, Ay, Bx, By) of the element map
  float2 *map32c;      // general mesh: [ne] (cx, cy)
  float4 *iso32;       // curved mesh: [4][ne] node offsets from the centre node
  double *mfac;        // FP64, general or curved mesh: [ns(ns+1)/2][ne] L D L^T of M_K
  double *isoJ;        // FP64, curved mesh: [4 NGP^2][ne] J at the Gauss points
  float *mfac32;       // mixed, general or curved mesh: [ns(ns+1)/2][ne] FP32 factor of M_K
  float4 *nodec4;      // [nn] (m/dt, qx, qy, l Cw rho_w) records
  float2 *vo2;         // [nn] ocean velocity
  float2 *lines32;     // [nx + ny] (h, 1/h) per mesh column, then per row
};

// ---- bounds-checked accesses (builds with -DMEVP_CHECKED) -----------------
// In a checked build every global access of the subcycle, transport and
// preparation kernels goes through these: an index outside [0, n) records
// its site number in flags[1] (the first one wins), and the access is
// skipped (a load returns 0).  mevp_sync reports it as MEVP_ERR_BOUNDS.  In
// a normal build they are the plain access.
__device__ __forceinline__ bool ck_ok(int *flags, long long i, long long n, int site) {
#ifdef MEVP_CHECKED
  if (i >= 0 && i < n) return true;
  if (flags) atomicCAS(flags + 1, 0, site);
  return false;
#else
  (void)flags; (void)i; (void)n; (void)site;
  return true;
#endif
}
template <typename T>
__device__ __forceinline__ T ck_ld(int *flags, const T *p, long long i, long long n, int site) {
  return ck_ok(flags, i, n, site) ? p[i] : T{};
}
template <typename T>
__device__ __forceinline__ T ck_ldg(int *flags, const T *p, long long i, long long n, int site) {
  return ck_ok(flags, i, n, site) ? __ldg(p + i) : T{};
}
template <typename T>
__device__ __forceinline__ void ck_st(int *flags, T *p, long long i, long long n, int site, T v) {
  if (ck_ok(flags, i, n, site)) p[i] = v;
}

// Scalar constants of the mixed-precision kernels (FP32).
struct MixArgs {
  float ie, hainv, dmin2, fac;  // stress update
  float opb, fdt;               // 1 + beta, f dt (velocity update)
  int has_vo;
  int stall;                    // test hook: extra bytes the staging barrier waits for
};

// Ensemble member as the persistent kernels see it.
struct EnsMember {
  DevState d;
  MixArgs ma;    // mixed precision
  Rheo r;        // FP64
  int has_vo;
  int base_cur;  // velocity/stress buffer at flip = 0
};
struct EnsWork {
  int member;
  int tx, ty;  // tile (mixed) or block index (FP64, in tx)
};

// Launchers (return cudaGetLastError of the launch).
cudaError_t launch_prepare(const DevState &d, const mevp_params &p, bool has_vo, int cur,
                           cudaStream_t st);
// ev: NULL, or 3 events recorded before the element kernel, between the
// two kernels and after the node kernel.
cudaError_t launch_subcycle_f64(const DevState &d, const Rheo &r, bool has_vo, int cur,
                                cudaStream_t st, cudaEvent_t *ev);
// the element part alone (any geometry, stress dofs and ice degree)
cudaError_t launch_element_f64(const DevState &d, const Rheo &r, int cur, cudaStream_t st);
cudaError_t launch_strain_diag(const DevState &d, int cur, cudaStream_t st);
// l_j = sum_K int_K phi_j into out[nn] (the area weights of the wind stress)
cudaError_t launch_lumped_area(const DevState &d, double *out, cudaStream_t st);
// general (non-affine) meshes: element kernel and read-back diagnostics
cudaError_t launch_element_general(const DevState &d, const Rheo &r, int cur, cudaStream_t st);
cudaError_t launch_strain_diag_general(const DevState &d, int cur, cudaStream_t st);
cudaError_t launch_force_elem_general(const DevState &d, cudaStream_t st);
// isoparametric (Q2) meshes
cudaError_t setup_iso_kernels();
cudaError_t setup_general_kernels();  // once per device, before any capture
// FP64 general / curved meshes: the per-element mass factors (and curved
// Jacobians) the element kernels read, once at state creation
cudaError_t launch_geom_factors(const DevState &d, cudaStream_t st);
cudaError_t launch_element_iso(const DevState &d, const Rheo &r, int cur, cudaStream_t st);
cudaError_t launch_strain_diag_iso(const DevState &d, int cur, cudaStream_t st);
cudaError_t launch_force_elem_iso(const DevState &d, cudaStream_t st);

// FP64 ensemble: persistent element kernel (block size chosen from
// kF64Blocks) + persistent node kernel (256 threads), over their work lists
constexpr int kF64BlockCount = 3;
extern const int kF64Blocks[kF64BlockCount];
constexpr int kNodeSlotBlock = 256;
// element launch over the work items of the members with n_S = ns
cudaError_t launch_ensemble_f64(const EnsMember *mem, const EnsWork *ework, int nework, int ns,
                                int block, int grid, int flip, cudaStream_t st);
cudaError_t launch_ensemble_f64_node(const EnsMember *mem, const EnsWork *nwork_list, int nnwork,
                                     int grid_n, int flip, cudaStream_t st);
int f64_block_ctas_per_sm(int block, int ns);
int f64_node_ctas_per_sm();

// mixed precision
constexpr int kMixTileCount = 3;
extern const int kMixTiles[kMixTileCount][2];
MixArgs make_mixargs(const Rheo &r, const mevp_params &p, bool has_vo);
int mixed_tile_count(int tile, int nx, int ny, int *tiles_x, int *tiles_y);
cudaError_t launch_ensemble_mixed(const EnsMember *mem, const EnsWork *work, int nwork, int tile,
                                  int grid, int flip, cudaStream_t st);
int mixed_tile_ctas_per_sm(int tile);
cudaError_t setup_mixed_kernels();  // once per device, before any capture
cudaError_t launch_prepare_mixed(const DevState &d, const mevp_params &p, bool has_vo, int cur,
                                 cudaStream_t st);
// Tensor maps of a mixed state's node records for the fused kernels' TMA
// staging: both velocity buffers and the node constants, boxes of one tile's
// owned-node window (rows: the tile height they were built for)
struct MixMaps {
  CUtensorMap vel[2];
  CUtensorMap cons;
  int rows = 0;
};
cudaError_t make_mix_maps(const DevState &d, MixMaps *mm);
cudaError_t launch_subcycle_mixed(const DevState &d, const Rheo &r, const mevp_params &p,
                                  bool has_vo, int cur, cudaStream_t st, cudaEvent_t *ev,
                                  bool fused, const MixMaps &mm, int stall = 0);
cudaError_t launch_vel_split(const DevState &d, int cur, cudaStream_t st);
cudaError_t launch_vel_join(const DevState &d, int cur, cudaStream_t st);
cudaError_t launch_stress_to_f32(const DevState &d, int cur, cudaStream_t st);
cudaError_t launch_stress_to_f64(const DevState &d, int cur, cudaStream_t st);
cudaError_t launch_force_diag(const DevState &d, cudaStream_t st);
// One advection step of H and A (in place) with the FP64 velocity vel;
// T1, T2: scratch of 2 n_a N_e doubles each (T2 used for n_a = 6 only).
cudaError_t launch_advect_step(const DevState &d, const double *vel, double dt, double *T1,
                               double *T2, cudaStream_t st);
// sets flags[0] when the current velocity holds a non-finite value
cudaError_t launch_nan_check(const DevState &d, int cur, cudaStream_t st);

// Error reporting shared by the C-ABI translation units (sets the thread-local
// message returned by mevp_last_error and returns the code).
int api_fail(int code, const char *msg);
int api_cuda_fail(cudaError_t e, const char *what);

}  // namespace mevp

// Host-side state behind the opaque mevp_state handle.
struct mevp_state {
  const mevp_mesh *mesh = nullptr;
  int ns = 0, na = 0, prec = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  bool owns_ws = false;
  mevp::DevState d{};
  int cur = 0;
  mevp_params prm{};
  mevp::Rheo rheo{};
  bool have_params = false;
  bool prepared = false;
  bool has_vo = false;
  bool has_pstar = false;  // per-element P* field set (mevp_set_strength_field)
  double *pstar_buf = nullptr;
  bool fused = true;  // mixed precision: one fused launch per subcycle
  int stall_test = 0;  // MEVP_OPT_STALL_TEST
  mevp::MixMaps maps;  // mixed precision: tensor maps of the fused kernels' TMA staging
  double *adv1 = nullptr, *adv2 = nullptr;  // advection stage buffers [2][na][ne]
  int nan_every = 0;         // watchdog interval in subcycles (0 = off)
  long long since_check = 0; // subcycles since the last watchdog scan
  bool use_graphs = true;  // replay captured subcycle chunks (non-default streams)
  struct Graph {
    int parity, len;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;  // instantiated chunks, dropped when kernel arguments change
  // event timing (benchmarks)
  int timing = 0;                   // sampling stride (0 = off)
  long long timed_calls = 0;        // subcycles launched since timing was enabled
  std::vector<cudaEvent_t> events;  // pool, 3 per timed subcycle
  size_t ev_used = 0;
};

namespace mevp {
int api_check_state(const mevp_state *s);
}  // namespace mevp
