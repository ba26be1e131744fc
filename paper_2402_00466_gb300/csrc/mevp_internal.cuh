// mevp_internal.cuh -- internal data structures and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/mevp.h"

struct mevp_mesh {
  int nx = 0, ny = 0;
  std::vector<double> xline;  // nx+1 vertex x coordinates (rectilinear mesh)
  std::vector<double> yline;  // ny+1 vertex y coordinates
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
  const double *xline, *yline;
  double *lines;       // [hx: nx][1/hx: nx][hy: ny][1/hy: ny], from the mesh lines
  double *vel[2];      // [2][nn] ping-pong
  double *S;           // FP64: [3][ns][ne]
  float *S32[2];       // mixed: [3][ns][ne], ping-pong with the velocity
  double *H, *A;       // [ne]
  double *tau;         // [2][nn]
  double *vo;          // [2][nn]
  double *Pe;          // [ne] ice strength per element
  double *nodec;       // [6][nn] cA, cB, cK, qx, qy, cD
  double *mass;        // [nn]
  double *fbuf;        // FP64: [18][ne] per-element nodal forces (scratch)
  float *fbuf32;       // mixed: [18][ne]
  double *diag;        // [3][ns][ne] or [2][nn] diagnostic output
  // mixed precision only (FP64 buffers above stage inputs and outputs)
  float4 *vel4[2];     // [nn] (u_hi, u_lo, v_hi, v_lo) records, ping-pong
  float *Pe32;         // [ne]
  float4 *nodec4;      // [nn] (m/dt, qx, qy, l Cw rho_w) records
  float2 *vo2;         // [nn] ocean velocity
  float2 *lines32;     // [nx + ny] (h, 1/h) per mesh column, then per row
};

// Launchers (return cudaGetLastError of the launch).
cudaError_t launch_prepare(const DevState &d, const mevp_params &p, bool has_vo, int cur,
                           cudaStream_t st);
// ev: NULL, or 3 events recorded before the element kernel, between the
// two kernels and after the node kernel.
cudaError_t launch_subcycle_f64(const DevState &d, const Rheo &r, bool has_vo, int cur,
                                cudaStream_t st, cudaEvent_t *ev);
cudaError_t launch_strain_diag(const DevState &d, int cur, cudaStream_t st);

// mixed precision
cudaError_t setup_mixed_kernels();  // once per device, before any capture
cudaError_t launch_prepare_mixed(const DevState &d, const mevp_params &p, bool has_vo, int cur,
                                 cudaStream_t st);
cudaError_t launch_subcycle_mixed(const DevState &d, const Rheo &r, const mevp_params &p,
                                  bool has_vo, int cur, cudaStream_t st, cudaEvent_t *ev,
                                  bool fused);
cudaError_t launch_vel_split(const DevState &d, int cur, cudaStream_t st);
cudaError_t launch_vel_join(const DevState &d, int cur, cudaStream_t st);
cudaError_t launch_stress_to_f32(const DevState &d, int cur, cudaStream_t st);
cudaError_t launch_stress_to_f64(const DevState &d, int cur, cudaStream_t st);
cudaError_t launch_force_diag(const DevState &d, cudaStream_t st);

}  // namespace mevp
