// mevp_capi.cu -- the C ABI declared in include/mevp.h.
//
// Host-side bookkeeping only: argument checks, the workspace layout, copies
// on the state's stream, and the launch sequence of a subcycle.  Every
// arithmetic step of the method runs in the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <new>
#include <string>

#include "mevp_internal.cuh"

using mevp::DevState;
using mevp::Rheo;


namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(MEVP_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

}  // namespace

namespace mevp {
int api_fail(int code, const char *msg) { return fail(code, "%s", msg); }
int api_cuda_fail(cudaError_t e, const char *what) { return cuda_fail(e, what); }
}  // namespace mevp

namespace {

#define MEVP_CUDA(call, what)                    \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Subcycle runs of at least kMinGraphChunk are replayed as CUDA graphs of up
// to kMaxGraphChunk subcycles: an outer step of up to 512 subcycles is one
// graph launch.
constexpr int kMinGraphChunk = 4;
constexpr int kMaxGraphChunk = 512;

struct Layout {
  size_t xline, yline, xy, nxy, lines, pstar, flags, adv1, adv2, Pg, Pg32, map32ab, map32c, iso32, mfac, isoJ, mfac32, vel0, vel1, S, S32a, S32b, H, A, tau, vo, Pe, nodec, mass, fbuf, fbuf32, diag,
      vel2a, vel2b, Pe32, nodec32, vo2, lines32, total;
};

Layout make_layout(const mevp_mesh *m, int ns, int na, int prec) {
  Layout L{};
  const size_t ne = (size_t)m->nx * m->ny;
  const size_t nn = (size_t)(2 * m->nx + 1) * (2 * m->ny + 1);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  L.xline = take(sizeof(double) * (m->nx + 1));
  L.yline = take(sizeof(double) * (m->ny + 1));
  L.xy = take(m->general ? m->xy.size() * sizeof(double) : 0);
  L.nxy = take(m->iso ? m->nxy.size() * sizeof(double) : 0);
  L.lines = take(sizeof(double) * 2 * (m->nx + m->ny));
  L.pstar = take(sizeof(double) * ne);
  L.flags = take(sizeof(int) * 4);
  L.adv1 = take(sizeof(double) * 2 * na * ne);
  L.adv2 = take(na == 6 ? sizeof(double) * 2 * na * ne : 0);
  L.Pg = take(na > 1 ? sizeof(double) * (ns == 3 ? 4 : 9) * ne : 0);
  L.Pg32 = take(na > 1 && prec == MEVP_MIXED ? sizeof(float) * (ns == 3 ? 4 : 9) * ne : 0);
  L.map32ab = take(m->general && prec == MEVP_MIXED ? sizeof(float4) * ne : 0);
  L.map32c = take(m->general && prec == MEVP_MIXED ? sizeof(float2) * ne : 0);
  L.iso32 = take(m->iso && prec == MEVP_MIXED ? 4 * sizeof(float4) * ne : 0);
  const bool geo64 = (m->general || m->iso) && prec == MEVP_FP64;
  L.mfac = take(geo64 ? sizeof(double) * (ns * (ns + 1) / 2) * ne : 0);
  L.isoJ = take(m->iso && prec == MEVP_FP64 ? sizeof(double) * 4 * (ns == 3 ? 4 : 9) * ne : 0);
  const bool geo32 = (m->general || m->iso) && prec == MEVP_MIXED;
  L.mfac32 = take(geo32 ? sizeof(float) * (ns * (ns + 1) / 2) * ne : 0);
  L.vel0 = take(sizeof(double) * 2 * nn);
  L.vel1 = take(sizeof(double) * 2 * nn);
  L.S = take(sizeof(double) * 3 * ns * ne);
  L.S32a = take(prec == MEVP_MIXED ? sizeof(float) * 3 * ns * ne : 0);
  L.S32b = take(prec == MEVP_MIXED ? sizeof(float) * 3 * ns * ne : 0);
  L.H = take(sizeof(double) * na * ne);
  L.A = take(sizeof(double) * na * ne);
  L.tau = take(sizeof(double) * 2 * nn);
  L.vo = take(sizeof(double) * 2 * nn);
  L.Pe = take(sizeof(double) * ne);
  L.nodec = take(sizeof(double) * 6 * nn);
  L.mass = take(sizeof(double) * nn);
  L.fbuf = take(sizeof(double) * 18 * ne);
  L.fbuf32 = take(prec == MEVP_MIXED ? sizeof(float) * 18 * ne : 0);
  const size_t dg = sizeof(double) * 3 * ns * ne, nd = sizeof(double) * 2 * nn;
  L.diag = take(dg > nd ? dg : nd);
  const bool mx = prec == MEVP_MIXED;
  L.vel2a = take(mx ? sizeof(float4) * nn : 0);
  L.vel2b = take(mx ? sizeof(float4) * nn : 0);
  L.Pe32 = take(mx ? sizeof(float) * ne : 0);
  L.nodec32 = take(mx ? sizeof(float4) * nn : 0);
  L.vo2 = take(mx ? sizeof(float2) * nn : 0);
  L.lines32 = take(mx ? sizeof(float2) * (m->nx + m->ny) : 0);
  L.total = off;
  return L;
}

// Sets *bad when any of x[0, n) is not finite (exponent field all ones).
__global__ void k_finite_check(const double *__restrict__ x, size_t n, int *bad) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  bool found = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x[i]);
    found |= ((bits >> 52) & 0x7ffull) == 0x7ffull;
  }
  if (found) *bad = 1;  // every writer stores the same value
}

}  // namespace

int mevp::api_check_state(const mevp_state *s) {
  if (!s) return fail(MEVP_ERR_ARG, "state is NULL");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != s->device)
    return fail(MEVP_ERR_STATE, "current device %d is not the state's device %d", dev, s->device);
  return MEVP_OK;
}

namespace {

int check_state(const mevp_state *s) { return mevp::api_check_state(s); }

// Copy n doubles into device buffer dst on the state's stream.  A host input
// is copied into the diagnostic buffer first (it holds max(3 n_stress N_e,
// 2 N_n) doubles, as much as the largest input), checked there for
// non-finite values by a kernel, and moved into dst only when it passed, so
// that a refused input leaves the state unchanged.  The call returns once
// the host buffer has been read and checked.
int copy_in(mevp_state *s, double *dst, const double *src, size_t n, int on_device,
            const char *what) {
  if (!src) return fail(MEVP_ERR_ARG, "%s: NULL pointer", what);
  if (on_device) {
    MEVP_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream),
              what);
    return MEVP_OK;
  }
  double *stage = s->d.diag;
  int *flag = s->d.flags + 3;
  MEVP_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s->stream), what);
  MEVP_CUDA(cudaMemcpyAsync(stage, src, n * sizeof(double), cudaMemcpyHostToDevice, s->stream),
            what);
  const size_t blocks = std::min<size_t>((n + 255) / 256, (size_t)s->d.nsm * 8);
  k_finite_check<<<(unsigned)std::max<size_t>(blocks, 1), 256, 0, s->stream>>>(stage, n, flag);
  MEVP_CUDA(cudaGetLastError(), what);
  int bad = 0;
  MEVP_CUDA(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream), what);
  MEVP_CUDA(cudaStreamSynchronize(s->stream), what);
  if (bad) return fail(MEVP_ERR_NAN, "%s: non-finite value in host input", what);
  MEVP_CUDA(cudaMemcpyAsync(dst, stage, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream),
            what);
  return MEVP_OK;
}

void drop_graphs(mevp_state *s) {
  for (auto &g : s->graphs) cudaGraphExecDestroy(g.exec);
  s->graphs.clear();
}

cudaError_t launch_one(mevp_state *s, int cur, cudaEvent_t *ev) {
  return s->prec == MEVP_MIXED
             ? mevp::launch_subcycle_mixed(s->d, s->rheo, s->prm, s->has_vo, cur, s->stream, ev,
                                           s->fused, s->maps, s->stall_test)
             : mevp::launch_subcycle_f64(s->d, s->rheo, s->has_vo, cur, s->stream, ev);
}

// Instantiated graph of `len` subcycles starting from velocity buffer
// `parity`, captured on the state's stream and cached.
int chunk_graph(mevp_state *s, int parity, int len, cudaGraphExec_t *out) {
  for (auto &g : s->graphs)
    if (g.parity == parity && g.len == len) {
      *out = g.exec;
      return MEVP_OK;
    }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "run_subcycles: begin capture");
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < len && le == cudaSuccess; ++k) le = launch_one(s, parity ^ (k & 1), nullptr);
  e = cudaStreamEndCapture(s->stream, &graph);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return cuda_fail(le != cudaSuccess ? le : e, "run_subcycles: capture");
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "run_subcycles: instantiate");
  s->graphs.push_back({parity, len, exec});
  *out = exec;
  return MEVP_OK;
}

}  // namespace

extern "C" {

const char *mevp_last_error(void) { return g_err.c_str(); }

const char *mevp_version(void) {
#ifdef MEVP_CHECKED
  return "mevp-gb300 0.1 (sm_103a, bounds-checked)";
#else
  return "mevp-gb300 0.1 (sm_103a)";
#endif
}

int mevp_mesh_create(int nx, int ny, double Lx, double Ly, const double *vertex_xy,
                     mevp_mesh **out) {
  if (!out) return fail(MEVP_ERR_ARG, "mesh_create: out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1) return fail(MEVP_ERR_ARG, "mesh_create: nx=%d ny=%d must be >= 1", nx, ny);
  const long long nn = (long long)(2 * (long long)nx + 1) * (2 * (long long)ny + 1);
  if (nn >= (1LL << 31) - 1) return fail(MEVP_ERR_ARG, "mesh_create: too many nodes (%lld)", nn);
  mevp_mesh *m = new (std::nothrow) mevp_mesh;
  if (!m) return fail(MEVP_ERR_OOM, "mesh_create: host allocation failed");
  m->nx = nx;
  m->ny = ny;
  m->xline.resize(nx + 1);
  m->yline.resize(ny + 1);
  if (!vertex_xy) {
    if (!(std::isfinite(Lx) && std::isfinite(Ly) && Lx > 0 && Ly > 0)) {
      delete m;
      return fail(MEVP_ERR_ARG, "mesh_create: Lx, Ly must be finite and > 0");
    }
    for (int i = 0; i <= nx; ++i) m->xline[i] = Lx * i / nx;
    for (int j = 0; j <= ny; ++j) m->yline[j] = Ly * j / ny;
  } else {
    const int vw = nx + 1;
    for (int i = 0; i <= nx; ++i) m->xline[i] = vertex_xy[2 * i];
    for (int j = 0; j <= ny; ++j) m->yline[j] = vertex_xy[2 * (j * vw) + 1];
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        const double x = vertex_xy[2 * (j * vw + i)], y = vertex_xy[2 * (j * vw + i) + 1];
        if (!std::isfinite(x) || !std::isfinite(y)) {
          delete m;
          return fail(MEVP_ERR_ARG, "mesh_create: non-finite vertex %d", j * vw + i);
        }
        if (x != m->xline[i] || y != m->yline[j]) m->general = true;
      }
    if (m->general) {
      // Every element must be a convex, counter-clockwise quadrilateral: the
      // Jacobian determinant of the bilinear map is affine in the reference
      // coordinates, so it is positive everywhere iff it is at the corners,
      // where it is the cross product of the two edges meeting there.
      m->xy.assign(vertex_xy, vertex_xy + 2 * (size_t)vw * (ny + 1));
      const double *v = m->xy.data();
      for (int ky = 0; ky < ny; ++ky)
        for (int kx = 0; kx < nx; ++kx) {
          const double *p00 = v + 2 * ((size_t)ky * vw + kx), *p10 = p00 + 2;
          const double *p01 = v + 2 * ((size_t)(ky + 1) * vw + kx), *p11 = p01 + 2;
          auto cross = [](const double *o, const double *a, const double *b) {
            return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0]);
          };
          if (!(cross(p00, p10, p01) > 0 && cross(p10, p11, p00) > 0 &&
                cross(p11, p01, p10) > 0 && cross(p01, p00, p11) > 0)) {
            delete m;
            return fail(MEVP_ERR_ARG,
                        "mesh_create: element (%d,%d) is not a convex counter-clockwise "
                        "quadrilateral",
                        kx, ky);
          }
        }
      *out = m;
      return MEVP_OK;
    }
  }
  for (int i = 0; i < nx; ++i)
    if (!(m->xline[i + 1] > m->xline[i])) {
      delete m;
      return fail(MEVP_ERR_ARG, "mesh_create: x coordinates must increase (column %d)", i);
    }
  for (int j = 0; j < ny; ++j)
    if (!(m->yline[j + 1] > m->yline[j])) {
      delete m;
      return fail(MEVP_ERR_ARG, "mesh_create: y coordinates must increase (row %d)", j);
    }
  *out = m;
  return MEVP_OK;
}

int mevp_mesh_create_nodes(int nx, int ny, const double *node_xy, mevp_mesh **out) {
  if (!out) return fail(MEVP_ERR_ARG, "mesh_create_nodes: out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1)
    return fail(MEVP_ERR_ARG, "mesh_create_nodes: nx=%d ny=%d must be >= 1", nx, ny);
  if (!node_xy) return fail(MEVP_ERR_ARG, "mesh_create_nodes: node_xy is NULL");
  const long long nw = 2LL * nx + 1, nh = 2LL * ny + 1, nn = nw * nh;
  if (nn >= (1LL << 31) - 1)
    return fail(MEVP_ERR_ARG, "mesh_create_nodes: too many nodes (%lld)", nn);
  for (long long i = 0; i < 2 * nn; ++i)
    if (!std::isfinite(node_xy[i]))
      return fail(MEVP_ERR_ARG, "mesh_create_nodes: non-finite node %lld", i / 2);
  // det J of every element's Q2 map must be positive: checked at a 5 x 5
  // grid of reference points (corners, edge and interior points)
  auto lag = [](int a, double t) {
    return a == 0 ? (1 - t) * (1 - 2 * t) : a == 1 ? 4 * t * (1 - t) : t * (2 * t - 1);
  };
  auto dlag = [](int a, double t) { return a == 0 ? 4 * t - 3 : a == 1 ? 4 - 8 * t : 4 * t - 1; };
  for (int ky = 0; ky < ny; ++ky)
    for (int kx = 0; kx < nx; ++kx)
      for (int qy = 0; qy <= 4; ++qy)
        for (int qx = 0; qx <= 4; ++qx) {
          const double xi = 0.25 * qx, eta = 0.25 * qy;
          double j00 = 0, j01 = 0, j10 = 0, j11 = 0;
          for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
              const double *p = node_xy + 2 * ((2LL * ky + b) * nw + 2LL * kx + a);
              const double gx = dlag(a, xi) * lag(b, eta), ge = lag(a, xi) * dlag(b, eta);
              j00 += p[0] * gx;
              j01 += p[0] * ge;
              j10 += p[1] * gx;
              j11 += p[1] * ge;
            }
          if (!(j00 * j11 - j01 * j10 > 0))
            return fail(MEVP_ERR_ARG,
                        "mesh_create_nodes: element (%d,%d) folds or is clockwise (det J <= 0 "
                        "at reference point (%g,%g))",
                        kx, ky, xi, eta);
        }
  mevp_mesh *m = new (std::nothrow) mevp_mesh;
  if (!m) return fail(MEVP_ERR_OOM, "mesh_create_nodes: host allocation failed");
  m->nx = nx;
  m->ny = ny;
  m->iso = true;
  m->nxy.assign(node_xy, node_xy + 2 * nn);
  m->xline.assign(nx + 1, 0.0);
  m->yline.assign(ny + 1, 0.0);
  *out = m;
  return MEVP_OK;
}

void mevp_mesh_destroy(mevp_mesh *mesh) { delete mesh; }

int mevp_state_workspace_bytes(const mevp_mesh *mesh, int n_stress, int n_adv, int precision,
                               size_t *bytes) {
  if (!mesh || !bytes) return fail(MEVP_ERR_ARG, "workspace_bytes: NULL argument");
  if (n_stress != 3 && n_stress != 6 && n_stress != 8)
    return fail(MEVP_ERR_ARG, "n_stress=%d: DG stress needs 3, 6 or 8 dofs", n_stress);
  if (n_adv != 1 && n_adv != 3 && n_adv != 6)
    return fail(MEVP_ERR_ARG, "n_adv=%d: H, A need 1, 3 or 6 dofs (DG0, DG1, DG2)", n_adv);
  if (precision != MEVP_FP64 && precision != MEVP_MIXED)
    return fail(MEVP_ERR_ARG, "precision=%d unknown", precision);
  *bytes = make_layout(mesh, n_stress, n_adv, precision).total;
  return MEVP_OK;
}

int mevp_state_create(const mevp_mesh *mesh, int n_stress, int n_adv, int precision,
                      void *cuda_stream, void *workspace, size_t workspace_bytes,
                      mevp_state **out) {
  if (!out) return fail(MEVP_ERR_ARG, "state_create: out is NULL");
  *out = nullptr;
  size_t need = 0;
  int rc = mevp_state_workspace_bytes(mesh, n_stress, n_adv, precision, &need);
  if (rc) return rc;
  if (workspace && workspace_bytes < need)
    return fail(MEVP_ERR_OOM, "state_create: workspace %zu bytes < %zu needed", workspace_bytes,
                need);
  if (workspace && ((uintptr_t)workspace & 255))
    return fail(MEVP_ERR_ARG, "state_create: workspace must be 256-byte aligned");
  mevp_state *s = new (std::nothrow) mevp_state;
  if (!s) return fail(MEVP_ERR_OOM, "state_create: host allocation failed");
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "cudaGetDevice");
  }
  s->mesh = mesh;
  s->ns = n_stress;
  s->na = n_adv;
  s->prec = precision;
  s->stream = (cudaStream_t)cuda_stream;
  if (workspace) {
    s->ws = workspace;
  } else {
    e = cudaMalloc(&s->ws, need);
    if (e != cudaSuccess) {
      delete s;
      cudaGetLastError();
      return fail(MEVP_ERR_OOM, "state_create: cudaMalloc(%zu) failed: %s", need,
                  cudaGetErrorString(e));
    }
    s->owns_ws = true;
  }
  s->ws_bytes = need;
  const Layout L = make_layout(mesh, n_stress, n_adv, precision);
  char *b = (char *)s->ws;
  DevState &d = s->d;
  d.nx = mesh->nx;
  d.ny = mesh->ny;
  d.ne = mesh->nx * mesh->ny;
  d.nw = 2 * mesh->nx + 1;
  d.nh = 2 * mesh->ny + 1;
  d.nn = d.nw * d.nh;
  d.ns = n_stress;
  d.na = n_adv;
  d.prec = precision;
  d.nsm = 1;
  if (cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
      d.nsm < 1) {
    cudaGetLastError();
    d.nsm = 1;
  }
  d.xline = (const double *)(b + L.xline);
  d.yline = (const double *)(b + L.yline);
  d.xy = mesh->general ? (const double2 *)(b + L.xy) : nullptr;
  d.nxy = mesh->iso ? (const double2 *)(b + L.nxy) : nullptr;
  const bool geo64 = (mesh->general || mesh->iso) && precision == MEVP_FP64;
  d.mfac = geo64 ? (double *)(b + L.mfac) : nullptr;
  d.isoJ = mesh->iso && precision == MEVP_FP64 ? (double *)(b + L.isoJ) : nullptr;
  d.lines = (double *)(b + L.lines);
  s->pstar_buf = (double *)(b + L.pstar);
  s->adv1 = (double *)(b + L.adv1);
  s->adv2 = (double *)(b + L.adv2);
  d.flags = (int *)(b + L.flags);
  d.pstar = nullptr;
  d.vel[0] = (double *)(b + L.vel0);
  d.vel[1] = (double *)(b + L.vel1);
  d.S = (double *)(b + L.S);
  d.S32[0] = (float *)(b + L.S32a);
  d.S32[1] = (float *)(b + L.S32b);
  d.H = (double *)(b + L.H);
  d.A = (double *)(b + L.A);
  d.tau = (double *)(b + L.tau);
  d.vo = (double *)(b + L.vo);
  d.Pe = (double *)(b + L.Pe);
  d.Pg = (double *)(b + L.Pg);
  d.nodec = (double *)(b + L.nodec);
  d.mass = (double *)(b + L.mass);
  d.fbuf = (double *)(b + L.fbuf);
  d.fbuf32 = (float *)(b + L.fbuf32);
  d.diag = (double *)(b + L.diag);
  if (precision == MEVP_MIXED) {
    e = mevp::setup_mixed_kernels();
    if (e != cudaSuccess) {
      if (s->owns_ws) cudaFree(s->ws);
      delete s;
      return cuda_fail(e, "state_create: kernel attributes");
    }
    d.vel4[0] = (float4 *)(b + L.vel2a);
    d.vel4[1] = (float4 *)(b + L.vel2b);
    d.Pe32 = (float *)(b + L.Pe32);
    d.Pg32 = (float *)(b + L.Pg32);
    d.map32ab = (float4 *)(b + L.map32ab);
    d.map32c = (float2 *)(b + L.map32c);
    d.iso32 = mesh->iso ? (float4 *)(b + L.iso32) : nullptr;
    d.mfac32 = (mesh->general || mesh->iso) ? (float *)(b + L.mfac32) : nullptr;
    d.nodec4 = (float4 *)(b + L.nodec32);
    d.vo2 = (float2 *)(b + L.vo2);
    d.lines32 = (float2 *)(b + L.lines32);
    e = mevp::make_mix_maps(d, &s->maps);
    if (e != cudaSuccess) {
      if (s->owns_ws) cudaFree(s->ws);
      delete s;
      return cuda_fail(e, "state_create: tensor maps of the mixed kernels");
    }
  }
  int r2 = MEVP_OK;
  e = cudaMemsetAsync(s->ws, 0, need, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void *)d.xline, mesh->xline.data(), sizeof(double) * (d.nx + 1),
                        cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void *)d.yline, mesh->yline.data(), sizeof(double) * (d.ny + 1),
                        cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && mesh->general)
    e = cudaMemcpyAsync((void *)d.xy, mesh->xy.data(), sizeof(double) * mesh->xy.size(),
                        cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && mesh->iso)
    e = cudaMemcpyAsync((void *)d.nxy, mesh->nxy.data(), sizeof(double) * mesh->nxy.size(),
                        cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && mesh->iso) e = mevp::setup_iso_kernels();
  if (e == cudaSuccess && mesh->general && !mesh->iso) e = mevp::setup_general_kernels();
  if (e == cudaSuccess && d.mfac) e = mevp::launch_geom_factors(d, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) r2 = cuda_fail(e, "state_create: initialise workspace");
  if (r2) {
    if (s->owns_ws) cudaFree(s->ws);
    delete s;
    return r2;
  }
  *out = s;
  return MEVP_OK;
}

void mevp_state_destroy(mevp_state *s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  for (cudaEvent_t e : s->events) cudaEventDestroy(e);
  for (auto &g : s->graphs) cudaGraphExecDestroy(g.exec);
  if (s->owns_ws) cudaFree(s->ws);
  delete s;
}

int mevp_set_params(mevp_state *s, const mevp_params *p) {
  int rc = check_state(s);
  if (rc) return rc;
  if (!p) return fail(MEVP_ERR_ARG, "set_params: NULL");
  const double v[] = {p->Pstar, p->C,  p->e,         p->DeltaMin,  p->alpha,      p->beta,
                      p->dt,    p->rho_ice, p->rho_water, p->Cw, p->coriolis_f};
  for (double x : v)
    if (!std::isfinite(x)) return fail(MEVP_ERR_ARG, "set_params: non-finite parameter");
  if (p->Pstar < 0 || p->C < 0) return fail(MEVP_ERR_ARG, "set_params: Pstar, C must be >= 0");
  if (!(p->e > 0)) return fail(MEVP_ERR_ARG, "set_params: e must be > 0");
  if (!(p->DeltaMin > 0)) return fail(MEVP_ERR_ARG, "set_params: DeltaMin must be > 0");
  if (!(p->alpha >= 1)) return fail(MEVP_ERR_ARG, "set_params: alpha must be >= 1");
  if (!(p->beta >= 0)) return fail(MEVP_ERR_ARG, "set_params: beta must be >= 0");
  if (!(p->dt > 0)) return fail(MEVP_ERR_ARG, "set_params: dt must be > 0");
  if (!(p->rho_ice > 0)) return fail(MEVP_ERR_ARG, "set_params: rho_ice must be > 0");
  if (p->rho_water < 0 || p->Cw < 0)
    return fail(MEVP_ERR_ARG, "set_params: rho_water, Cw must be >= 0");
  s->prm = *p;
  s->rheo = mevp::make_rheo(*p);
  s->have_params = true;
  drop_graphs(s);
  return MEVP_OK;
}

int mevp_set_ice(mevp_state *s, const double *H, const double *A, int on_device) {
  int rc = check_state(s);
  if (rc) return rc;
  const size_t n = (size_t)s->na * s->d.ne;
  if ((rc = copy_in(s, s->d.H, H, n, on_device, "set_ice H"))) return rc;
  return copy_in(s, s->d.A, A, n, on_device, "set_ice A");
}

int mevp_set_forcing(mevp_state *s, const double *tau, const double *v_ocean, int on_device) {
  int rc = check_state(s);
  if (rc) return rc;
  const size_t n = 2 * (size_t)s->d.nn;
  if ((rc = copy_in(s, s->d.tau, tau, n, on_device, "set_forcing tau"))) return rc;
  if (v_ocean) {
    if ((rc = copy_in(s, s->d.vo, v_ocean, n, on_device, "set_forcing v_ocean"))) return rc;
    if (!s->has_vo) drop_graphs(s);
    s->has_vo = true;
  } else {
    MEVP_CUDA(cudaMemsetAsync(s->d.vo, 0, n * sizeof(double), s->stream), "set_forcing");
    if (s->has_vo) drop_graphs(s);
    s->has_vo = false;
  }
  return MEVP_OK;
}

int mevp_set_strength_field(mevp_state *s, const double *Pstar, int on_device) {
  int rc = check_state(s);
  if (rc) return rc;
  if (!Pstar) {
    s->d.pstar = nullptr;
    s->has_pstar = false;
    drop_graphs(s);
    return MEVP_OK;
  }
  if ((rc = copy_in(s, s->pstar_buf, Pstar, (size_t)s->d.ne, on_device, "set_strength_field")))
    return rc;
  s->d.pstar = s->pstar_buf;
  s->has_pstar = true;
  drop_graphs(s);
  return MEVP_OK;
}

int mevp_set_velocity(mevp_state *s, const double *uv, int on_device) {
  int rc = check_state(s);
  if (rc) return rc;
  rc = copy_in(s, s->d.vel[s->cur], uv, 2 * (size_t)s->d.nn, on_device, "set_velocity");
  if (rc || s->prec != MEVP_MIXED) return rc;
  cudaError_t e = mevp::launch_vel_split(s->d, s->cur, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_velocity split");
  return MEVP_OK;
}

int mevp_set_stress(mevp_state *s, const double *S, int on_device) {
  int rc = check_state(s);
  if (rc) return rc;
  rc = copy_in(s, s->d.S, S, 3 * (size_t)s->ns * s->d.ne, on_device, "set_stress");
  if (rc || s->prec != MEVP_MIXED) return rc;
  cudaError_t e = mevp::launch_stress_to_f32(s->d, s->cur, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_stress convert");
  return MEVP_OK;
}

int mevp_advect(mevp_state *s, int n_steps) {
  mevp::NvtxRange nvtx_range_("mevp_advect");
  int rc = check_state(s);
  if (rc) return rc;
  if (n_steps < 0) return fail(MEVP_ERR_ARG, "advect: n_steps=%d < 0", n_steps);
  if (!s->have_params) return fail(MEVP_ERR_STATE, "advect: parameters not set");
  if (n_steps == 0) return MEVP_OK;
  cudaError_t e = cudaSuccess;
  if (s->prec == MEVP_MIXED) e = mevp::launch_vel_join(s->d, s->cur, s->stream);
  for (int k = 0; k < n_steps && e == cudaSuccess; ++k)
    e = mevp::launch_advect_step(s->d, s->d.vel[s->cur], s->prm.dt, s->adv1, s->adv2, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "advect launch");
  return MEVP_OK;
}

int mevp_begin_step(mevp_state *s) {
  mevp::NvtxRange nvtx_range_("mevp_begin_step");
  int rc = check_state(s);
  if (rc) return rc;
  if (!s->have_params) return fail(MEVP_ERR_STATE, "begin_step: parameters not set");
  cudaError_t e = s->prec == MEVP_MIXED
                      ? mevp::launch_prepare_mixed(s->d, s->prm, s->has_vo, s->cur, s->stream)
                      : mevp::launch_prepare(s->d, s->prm, s->has_vo, s->cur, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "begin_step launch");
  s->prepared = true;
  return MEVP_OK;
}

int mevp_run_subcycles(mevp_state *s, int n) {
  mevp::NvtxRange nvtx_range_("mevp_run_subcycles");
  int rc = check_state(s);
  if (rc) return rc;
  if (n < 0) return fail(MEVP_ERR_ARG, "run_subcycles: n=%d < 0", n);
  if (!s->prepared) return fail(MEVP_ERR_STATE, "run_subcycles: call mevp_begin_step first");
  // The legacy default stream cannot be captured: launch directly there.
  const bool graphs = s->use_graphs && s->stream != nullptr;
  int i = 0;
  while (i < n) {
    if (s->nan_every > 0 && s->since_check >= s->nan_every) {
      cudaError_t e = mevp::launch_nan_check(s->d, s->cur, s->stream);
      if (e != cudaSuccess) return cuda_fail(e, "run_subcycles watchdog");
      s->since_check = 0;
    }
    const bool timed = s->timing && (s->timed_calls % s->timing) == 0;
    const int to_check = s->nan_every > 0 ? (int)(s->nan_every - s->since_check) : n;
    if (timed || !graphs || n - i < kMinGraphChunk || to_check < kMinGraphChunk) {
      cudaEvent_t *ev = nullptr;
      if (timed) {
        while (s->events.size() < s->ev_used + 3) {
          cudaEvent_t e;
          MEVP_CUDA(cudaEventCreate(&e), "run_subcycles timing event");
          s->events.push_back(e);
        }
        ev = &s->events[s->ev_used];
        s->ev_used += 3;
      }
      cudaError_t e = launch_one(s, s->cur, ev);
      if (e != cudaSuccess) return cuda_fail(e, "run_subcycles launch");
      s->cur ^= 1;
      if (s->timing) s->timed_calls++;
      s->since_check++;
      ++i;
      continue;
    }
    // untimed run up to the next timed subcycle or watchdog scan (or the
    // end), in graph chunks
    int len = n - i;
    if (len > kMaxGraphChunk) len = kMaxGraphChunk;
    if (len > to_check) len = to_check;
    if (s->timing) {
      const long long to_next = s->timing - (s->timed_calls % s->timing);
      if (len > to_next) len = (int)to_next;
    }
    cudaGraphExec_t exec = nullptr;
    if ((rc = chunk_graph(s, s->cur, len, &exec))) return rc;
    MEVP_CUDA(cudaGraphLaunch(exec, s->stream), "run_subcycles graph launch");
    s->cur ^= (len & 1);
    if (s->timing) s->timed_calls += len;
    s->since_check += len;
    i += len;
  }
  if (s->nan_every > 0 && s->since_check >= s->nan_every) {
    cudaError_t e = mevp::launch_nan_check(s->d, s->cur, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "run_subcycles watchdog");
    s->since_check = 0;
  }
  return MEVP_OK;
}

int mevp_set_option(mevp_state *s, int option, int value) {
  int rc = check_state(s);
  if (rc) return rc;
  switch (option) {
    case MEVP_OPT_FUSED:
      if (value != 0 && value != 1) return fail(MEVP_ERR_ARG, "set_option: FUSED takes 0 or 1");
      s->fused = value != 0;
      drop_graphs(s);
      return MEVP_OK;
    case MEVP_OPT_NAN_CHECK:
      if (value < 0) return fail(MEVP_ERR_ARG, "set_option: NAN_CHECK takes k >= 0");
      s->nan_every = value;
      s->since_check = 0;
      return MEVP_OK;
    case MEVP_OPT_STALL_TEST:
      if (value != 0 && value != 1) return fail(MEVP_ERR_ARG, "set_option: STALL_TEST takes 0 or 1");
      s->stall_test = value;
      drop_graphs(s);
      return MEVP_OK;
    case MEVP_OPT_GRAPHS:
      if (value != 0 && value != 1) return fail(MEVP_ERR_ARG, "set_option: GRAPHS takes 0 or 1");
      s->use_graphs = value != 0;
      return MEVP_OK;
    default:
      return fail(MEVP_ERR_ARG, "set_option: unknown option %d", option);
  }
}

int mevp_timing_enable(mevp_state *s, int on) {
  int rc = check_state(s);
  if (rc) return rc;
  if (on < 0) return fail(MEVP_ERR_ARG, "timing_enable: stride %d < 0", on);
  s->timing = on;
  s->timed_calls = 0;
  s->ev_used = 0;
  return MEVP_OK;
}

int mevp_timing_read(mevp_state *s, double *ms, long long *launches) {
  int rc = check_state(s);
  if (rc) return rc;
  if (!ms || !launches) return fail(MEVP_ERR_ARG, "timing_read: NULL output");
  MEVP_CUDA(cudaStreamSynchronize(s->stream), "timing_read sync");
  ms[0] = ms[1] = 0.0;
  launches[0] = launches[1] = 0;
  for (size_t i = 0; i + 3 <= s->ev_used; i += 3) {
    float a = 0.f, b = 0.f;
    MEVP_CUDA(cudaEventElapsedTime(&a, s->events[i], s->events[i + 1]), "timing_read");
    MEVP_CUDA(cudaEventElapsedTime(&b, s->events[i + 1], s->events[i + 2]), "timing_read");
    ms[0] += a;
    ms[1] += b;
    launches[0] += 1;
    launches[1] += 1;
  }
  s->ev_used = 0;
  return MEVP_OK;
}

int mevp_read_field(mevp_state *s, int field, double *dst, size_t count, int on_device) {
  mevp::NvtxRange nvtx_range_("mevp_read_field");
  int rc = check_state(s);
  if (rc) return rc;
  if (!dst) return fail(MEVP_ERR_ARG, "read_field: dst is NULL");
  const DevState &d = s->d;
  const size_t nn = d.nn, ne = d.ne, ns = s->ns;
  const double *src = nullptr;
  size_t n = 0;
  cudaError_t e = cudaSuccess;
  const bool mx = s->prec == MEVP_MIXED;
  switch (field) {
    case MEVP_U: case MEVP_V:
      if (mx) e = mevp::launch_vel_join(d, s->cur, s->stream);
      src = d.vel[s->cur] + (field == MEVP_V ? nn : 0);
      n = nn;
      break;
    case MEVP_S11: case MEVP_S12: case MEVP_S22:
      if (mx) e = mevp::launch_stress_to_f64(d, s->cur, s->stream);
      src = d.S + (size_t)(field - MEVP_S11) * ns * ne;
      n = ns * ne;
      break;
    case MEVP_E11: case MEVP_E12: case MEVP_E22:
      if (mx) e = mevp::launch_vel_join(d, s->cur, s->stream);
      if (e == cudaSuccess) e = mevp::launch_strain_diag(d, s->cur, s->stream);
      src = d.diag + (size_t)(field - MEVP_E11) * ns * ne;
      n = ns * ne;
      break;
    case MEVP_FORCE_X: case MEVP_FORCE_Y:
      if (mx) e = mevp::launch_stress_to_f64(d, s->cur, s->stream);
      if (e == cudaSuccess) e = mevp::launch_force_diag(d, s->stream);
      src = d.diag + (size_t)(field - MEVP_FORCE_X) * nn;
      n = nn;
      break;
    case MEVP_H: src = d.H; n = (size_t)s->na * ne; break;
    case MEVP_A: src = d.A; n = (size_t)s->na * ne; break;
    case MEVP_NODAL_MASS: src = d.mass; n = nn; break;
    default: return fail(MEVP_ERR_ARG, "read_field: unknown field %d", field);
  }
  if (e != cudaSuccess) return cuda_fail(e, "read_field diagnostic launch");
  if (count < n) return fail(MEVP_ERR_ARG, "read_field: count %zu < field size %zu", count, n);
  MEVP_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            s->stream),
            "read_field copy");
  if (!on_device) MEVP_CUDA(cudaStreamSynchronize(s->stream), "read_field sync");
  return MEVP_OK;
}

int mevp_sync(mevp_state *s) {
  int rc = check_state(s);
  if (rc) return rc;
  MEVP_CUDA(cudaStreamSynchronize(s->stream), "sync");
  MEVP_CUDA(cudaGetLastError(), "sync");
#ifdef MEVP_CHECKED
  {
    int site = 0;
    MEVP_CUDA(cudaMemcpy(&site, s->d.flags + 1, sizeof(int), cudaMemcpyDeviceToHost), "sync");
    if (site) {
      MEVP_CUDA(cudaMemset(s->d.flags + 1, 0, sizeof(int)), "sync");
      return fail(MEVP_ERR_BOUNDS, "sync: out-of-bounds access at kernel site %d", site);
    }
  }
#endif
  {
    int stalled = 0;
    MEVP_CUDA(cudaMemcpy(&stalled, s->d.flags + 2, sizeof(int), cudaMemcpyDeviceToHost), "sync");
    if (stalled) {
      MEVP_CUDA(cudaMemset(s->d.flags + 2, 0, sizeof(int)), "sync");
      return fail(MEVP_ERR_TIMEOUT, "sync: a bounded device wait gave up (staging copies of "
                                    "the fused kernel did not complete)");
    }
  }
  if (s->nan_every > 0) {
    int flag = 0;
    MEVP_CUDA(cudaMemcpy(&flag, s->d.flags, sizeof(int), cudaMemcpyDeviceToHost), "sync");
    if (flag) {
      MEVP_CUDA(cudaMemset(s->d.flags, 0, sizeof(int)), "sync");
      return fail(MEVP_ERR_NAN, "sync: the watchdog found a non-finite velocity");
    }
  }
  return MEVP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// mevp_run_subcycles_noalloc: the subcycle loop for callers that cannot
// allocate device memory.  Its scratch (per-element ice strength, per-node
// constants and mass, per-element nodal forces, and the second velocity
// buffer) lives in one file-scope device array that every call shares.
// ---------------------------------------------------------------------------
static constexpr size_t kNoAllocScratchBytes = (size_t)MEVP_NOALLOC_SCRATCH_BYTES;

// One array per process and device, held from module load until exit.  Host
// code must not use its name as an address (it is a host-side stand-in);
// the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Scratch layout for an nx x ny mesh: offsets (bytes, 256-aligned) of the
// regions and the total.
struct NoAllocLayout {
  size_t flags, lines, Pe, nodec, mass, fbuf, vel2, total;
};

NoAllocLayout noalloc_layout(size_t nx, size_t ny, size_t ne, size_t nn) {
  NoAllocLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  L.flags = take(sizeof(int) * 4);
  L.lines = take(sizeof(double) * 2 * (nx + ny));
  L.Pe = take(sizeof(double) * ne);
  L.nodec = take(sizeof(double) * 6 * nn);
  L.mass = take(sizeof(double) * nn);
  L.fbuf = take(sizeof(double) * 18 * ne);
  L.vel2 = take(sizeof(double) * 2 * nn);
  L.total = off;
  return L;
}

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
int noalloc_scratch(int device, void **out) {
  if (device < 0 || device >= kMaxDevices)
    return fail(MEVP_ERR_UNSUPPORTED, "run_subcycles_noalloc: device index %d >= %d", device,
                kMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "run_subcycles_noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return MEVP_OK;
}

// Sets *bad when a coordinate line does not increase strictly (one thread
// per interval of xline, then of yline).
__global__ void k_lines_increasing(const double *xline, int nx, const double *yline, int ny,
                                   int *bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nx) {
    if (!(xline[i + 1] > xline[i])) atomicOr(bad, 1);
  } else if (i < nx + ny) {
    const int j = i - nx;
    if (!(yline[j + 1] > yline[j])) atomicOr(bad, 1);
  }
}

// True when p is device (or managed) memory usable from `device`.
bool is_device_ptr(const void *p, int device) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) &&
         a.device == device;
}

}  // namespace

extern "C" int mevp_run_subcycles_noalloc(int nx, int ny, int n_stress, const mevp_params *p,
                                          const double *xline, const double *yline,
                                          const double *H, const double *A, const double *tau,
                                          const double *v_ocean, double *vel, double *S, int n,
                                          void *cuda_stream) {
  mevp::NvtxRange nvtx_range_("mevp_run_subcycles_noalloc");
  if (nx < 1 || ny < 1)
    return fail(MEVP_ERR_ARG, "run_subcycles_noalloc: nx=%d ny=%d must be >= 1", nx, ny);
  if (n_stress != 3 && n_stress != 6 && n_stress != 8)
    return fail(MEVP_ERR_ARG, "run_subcycles_noalloc: n_stress=%d must be 3, 6 or 8", n_stress);
  if (n < 0) return fail(MEVP_ERR_ARG, "run_subcycles_noalloc: n=%d < 0", n);
  if (!p) return fail(MEVP_ERR_ARG, "run_subcycles_noalloc: params is NULL");
  const long long nn_ll = (2LL * nx + 1) * (2LL * ny + 1);
  if (nn_ll >= (1LL << 31) - 1) return fail(MEVP_ERR_ARG, "run_subcycles_noalloc: mesh too large");
  const size_t ne = (size_t)nx * ny, nn = (size_t)nn_ll;
  const NoAllocLayout L = noalloc_layout((size_t)nx, (size_t)ny, ne, nn);
  if (L.total > kNoAllocScratchBytes)
    return fail(MEVP_ERR_ARG,
                "run_subcycles_noalloc: a %dx%d mesh needs %zu scratch bytes, more than the "
                "%zu-byte static scratch (19*N_e + 9*N_n + 2*(nx+ny) doubles; 128x128 fits)",
                nx, ny, L.total, kNoAllocScratchBytes);
  // parameters: same admissible ranges as mevp_set_params
  const double pv[] = {p->Pstar, p->C,       p->e,      p->DeltaMin, p->alpha,      p->beta,
                       p->dt,    p->rho_ice, p->rho_water, p->Cw,    p->coriolis_f};
  for (double x : pv)
    if (!std::isfinite(x)) return fail(MEVP_ERR_ARG, "run_subcycles_noalloc: non-finite parameter");
  if (p->Pstar < 0 || p->C < 0 || !(p->e > 0) || !(p->DeltaMin > 0) || !(p->alpha >= 1) ||
      !(p->beta >= 0) || !(p->dt > 0) || !(p->rho_ice > 0) || p->rho_water < 0 || p->Cw < 0)
    return fail(MEVP_ERR_ARG, "run_subcycles_noalloc: parameter out of range");
  int device = -1;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_fail(e, "run_subcycles_noalloc: cudaGetDevice");
  const void *ptrs[] = {xline, yline, H, A, tau, vel, S};
  const char *names[] = {"xline", "yline", "H", "A", "tau", "vel", "S"};
  for (int i = 0; i < 7; ++i)
    if (!ptrs[i] || !is_device_ptr(ptrs[i], device))
      return fail(MEVP_ERR_ARG, "run_subcycles_noalloc: %s must be device memory of device %d",
                  names[i], device);
  if (v_ocean && !is_device_ptr(v_ocean, device))
    return fail(MEVP_ERR_ARG, "run_subcycles_noalloc: v_ocean must be device memory or NULL");
  void *scratch = nullptr;
  int rc = noalloc_scratch(device, &scratch);
  if (rc) return rc;

  const Rheo r = mevp::make_rheo(*p);

  char *b = (char *)scratch;
  DevState d{};
  d.nx = nx;
  d.ny = ny;
  d.ne = (int)ne;
  d.nw = 2 * nx + 1;
  d.nh = 2 * ny + 1;
  d.nn = (int)nn;
  d.ns = n_stress;
  d.na = 1;
  d.nsm = 1;
  if (cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      d.nsm < 1) {
    cudaGetLastError();
    d.nsm = 1;
  }
  d.prec = MEVP_FP64;
  d.xline = xline;
  d.yline = yline;
  d.lines = (double *)(b + L.lines);
  d.vel[0] = vel;
  d.vel[1] = (double *)(b + L.vel2);
  d.S = S;
  d.H = (double *)H;
  d.A = (double *)A;
  d.tau = (double *)tau;
  d.vo = (double *)v_ocean;
  d.Pe = (double *)(b + L.Pe);
  d.nodec = (double *)(b + L.nodec);
  d.mass = (double *)(b + L.mass);
  d.fbuf = (double *)(b + L.fbuf);
  d.flags = (int *)(b + L.flags);
  const bool has_vo = v_ocean != nullptr;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // The status words are the only scratch read before this call writes
  // them: clear them, then check the coordinate lines on the device and wait
  // for that one word (the only wait of the call).
  e = cudaMemsetAsync(d.flags, 0, sizeof(int) * 4, st);
  if (e != cudaSuccess) return cuda_fail(e, "run_subcycles_noalloc: clearing the status words");
  k_lines_increasing<<<(nx + ny + 255) / 256, 256, 0, st>>>(xline, nx, yline, ny, d.flags + 3);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "run_subcycles_noalloc: line check launch");
  int lines_bad = 0;
  e = cudaMemcpyAsync(&lines_bad, d.flags + 3, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "run_subcycles_noalloc: line check");
  if (lines_bad)
    return fail(MEVP_ERR_ARG,
                "run_subcycles_noalloc: xline and yline must increase strictly");
  // v^n := vel at entry; every other scratch word is written before it is
  // read, so nothing else in the shared array has to be cleared first.
  e = mevp::launch_prepare(d, *p, has_vo, 0, st);
  if (e != cudaSuccess) return cuda_fail(e, "run_subcycles_noalloc: prepare launch");
  int cur = 0;
  for (int i = 0; i < n; ++i) {
    e = mevp::launch_subcycle_f64(d, r, has_vo, cur, st, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "run_subcycles_noalloc: subcycle launch");
    cur ^= 1;
  }
  if (cur == 1) {  // odd count: the result sits in the scratch velocity buffer
    e = cudaMemcpyAsync(vel, d.vel[1], sizeof(double) * 2 * nn, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "run_subcycles_noalloc: copy back");
  }
#ifdef MEVP_CHECKED
  {  // the bounds-checked build waits and reports a skipped out-of-bounds access
    int site = 0;
    e = cudaMemcpyAsync(&site, d.flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "run_subcycles_noalloc: status read");
    if (site)
      return fail(MEVP_ERR_BOUNDS, "run_subcycles_noalloc: out-of-bounds access at kernel site %d",
                  site);
  }
#endif
  return MEVP_OK;
}
