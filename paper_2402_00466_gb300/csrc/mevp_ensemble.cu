// mevp_ensemble.cu -- the ensemble entry points of include/mevp.h.
//
// An ensemble advances many independent domains (existing states of uneven
// sizes and kinds, one precision, one stream) together.  Per subcycle, the
// members on rectilinear meshes with 3 or 6 stress dofs and DG0 ice are
// batched: in the mixed precision one persistent launch covers their
// (member, tile) work list, in FP64 one persistent element launch per stress
// space their element blocks, and one persistent node launch the nodes of
// all members.
// The other members (8 stress dofs, DG1/DG2 ice, general or curved meshes)
// run their single-state launches (FP64: the element launch) within the same
// stream and graphs: batching every variant into one kernel would make its
// register allocation spill for all members.  Runs of subcycles are replayed as CUDA graphs, and
// the tile shape (mixed) or element block size (FP64) is chosen by timing the
// candidates on the ensemble itself.  Per element and per node the arithmetic
// is that of the single-state kernels, so an ensemble step gives bitwise the
// results of stepping each member alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "mevp_internal.cuh"

using mevp::EnsMember;
using mevp::EnsWork;

struct mevp_ensemble {
  std::vector<mevp_state *> members;
  int prec = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  int shape = 1;                      // index into the tile / block candidates
  std::vector<EnsMember> host_mem;    // descriptors as uploaded
  EnsMember *d_mem = nullptr;
  EnsWork *d_work = nullptr;          // mixed: tiles; FP64: element blocks
  EnsWork *d_nwork = nullptr;         // FP64: node-slot blocks
  int nwork = 0, nnwork = 0;
  size_t work_cap = 0, nwork_cap = 0;
  int grid = 0, grid_n = 0;
  // FP64: the element work is two sublists of d_work, the 3-dof members'
  // first (n3 items), then the 6-dof members' (grid3 / grid6 blocks)
  int n3 = 0, grid3 = 0, grid6 = 0;
  std::vector<int> solo;              // members stepped with their own launches
  bool use_graphs = true;
  struct Graph {
    int flip, len;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
};

namespace {

// runs of 4 to 512 subcycles are one graph launch each
constexpr int kMinGraphChunk = 4;
constexpr int kMaxGraphChunk = 512;

int efail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return mevp::api_fail(code, buf);
}

void drop_graphs(mevp_ensemble *e) {
  for (auto &g : e->graphs) cudaGraphExecDestroy(g.exec);
  e->graphs.clear();
}

int shape_count(int prec) { return prec == MEVP_MIXED ? mevp::kMixTileCount : mevp::kF64BlockCount; }

// Whether a member's element work goes into the batched launch.
bool batched(const mevp_state *s) { return !s->d.xy && !s->d.nxy && s->na == 1 && s->ns != 8; }

// Relative per-element cost (FP64 flop counts of the rectilinear element
// kernel), for ordering the batched work largest first.
long long member_cost(const mevp_state *s) {
  return (long long)s->d.ne * (s->ns == 3 ? 474 : 1055);
}

// Work lists for the current shape, members ordered by decreasing cost.
int build_work(mevp_ensemble *e) {
  std::vector<int> order(e->members.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return member_cost(e->members[a]) > member_cost(e->members[b]);
  });
  std::vector<EnsWork> w, nw;
  e->solo.clear();
  for (int m : order)
    if (!batched(e->members[m])) e->solo.push_back(m);
  if (e->prec == MEVP_MIXED) {
    for (int m : order) {
      const mevp_state *s = e->members[m];
      if (!batched(s)) continue;
      int tx = 0, ty = 0;
      mevp::mixed_tile_count(e->shape, s->d.nx, s->d.ny, &tx, &ty);
      for (int y = 0; y < ty; ++y)
        for (int x = 0; x < tx; ++x) w.push_back({m, x, y});
    }
  } else {
    const int B = mevp::kF64Blocks[e->shape];
    for (int pass = 0; pass < 2; ++pass) {  // 3-dof members, then 6-dof
      for (int m : order) {
        const mevp_state *s = e->members[m];
        if (!batched(s) || (s->ns == 3) != (pass == 0)) continue;
        for (int b = 0; b * B < s->d.ne; ++b) w.push_back({m, b, 0});
      }
      if (pass == 0) e->n3 = (int)w.size();
    }
    for (int m : order) {
      const mevp_state *s = e->members[m];
      const int slots = (s->d.nx + 1) * (s->d.ny + 1);
      for (int b = 0; b * mevp::kNodeSlotBlock < slots; ++b) nw.push_back({m, b, 0});
    }
  }
  auto upload = [&](std::vector<EnsWork> &v, EnsWork *&dptr, size_t &cap) -> int {
    if (v.empty()) return MEVP_OK;
    if (v.size() > cap) {
      if (dptr) cudaFree(dptr);
      dptr = nullptr;
      cudaError_t err = cudaMalloc(&dptr, v.size() * sizeof(EnsWork));
      if (err != cudaSuccess) {
        cudaGetLastError();
        cap = 0;
        return efail(MEVP_ERR_OOM, "ensemble: work list allocation failed");
      }
      cap = v.size();
    }
    cudaError_t err = cudaMemcpy(dptr, v.data(), v.size() * sizeof(EnsWork), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return mevp::api_cuda_fail(err, "ensemble: work list upload");
    return MEVP_OK;
  };
  int rc = upload(w, e->d_work, e->work_cap);
  if (!rc) rc = upload(nw, e->d_nwork, e->nwork_cap);
  if (rc) return rc;
  e->nwork = (int)w.size();
  e->nnwork = (int)nw.size();
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->device);
  if (e->prec == MEVP_MIXED) {
    const int per_sm = mevp::mixed_tile_ctas_per_sm(e->shape);
    e->grid = std::max(1, std::min(e->nwork, sms * per_sm));
  } else {
    const int n6 = e->nwork - e->n3;
    e->grid3 = std::max(1, std::min(e->n3, sms * mevp::f64_block_ctas_per_sm(e->shape, 3)));
    e->grid6 = std::max(1, std::min(n6, sms * mevp::f64_block_ctas_per_sm(e->shape, 6)));
    e->grid_n = std::max(1, std::min(e->nnwork, sms * mevp::f64_node_ctas_per_sm()));
  }
  drop_graphs(e);
  return MEVP_OK;
}

// Descriptors of the members as they are now; re-uploaded (and graphs
// dropped) when they changed since the last upload.  Returns the flip that
// maps each member's current buffer to its uploaded base buffer.
int sync_descriptors(mevp_ensemble *e, int *flip) {
  const size_t n = e->members.size();
  bool same = e->host_mem.size() == n;
  int f = -1;
  if (same) {
    for (size_t m = 0; m < n && same; ++m) {
      const mevp_state *s = e->members[m];
      const EnsMember &h = e->host_mem[m];
      const int fm = s->cur ^ h.base_cur;
      if (f < 0) f = fm;
      same = fm == f && h.has_vo == (int)s->has_vo &&
             std::memcmp(&h.r, &s->rheo, sizeof(mevp::Rheo)) == 0;
      if (same && e->prec == MEVP_MIXED) {
        const mevp::MixArgs ma = mevp::make_mixargs(s->rheo, s->prm, s->has_vo);
        same = std::memcmp(&ma, &h.ma, sizeof ma) == 0;
      }
    }
  }
  if (same) {
    *flip = f < 0 ? 0 : f;
    return MEVP_OK;
  }
  std::vector<EnsMember> hm(n);
  for (size_t m = 0; m < n; ++m) {
    const mevp_state *s = e->members[m];
    std::memset(&hm[m], 0, sizeof(EnsMember));
    hm[m].d = s->d;
    hm[m].r = s->rheo;
    hm[m].ma = mevp::make_mixargs(s->rheo, s->prm, s->has_vo);
    hm[m].has_vo = s->has_vo ? 1 : 0;
    hm[m].base_cur = s->cur;
  }
  cudaError_t err = cudaStreamSynchronize(e->stream);
  if (err == cudaSuccess)
    err = cudaMemcpy(e->d_mem, hm.data(), n * sizeof(EnsMember), cudaMemcpyHostToDevice);
  if (err != cudaSuccess) return mevp::api_cuda_fail(err, "ensemble: descriptor upload");
  e->host_mem.swap(hm);
  drop_graphs(e);
  *flip = 0;
  return MEVP_OK;
}

// One subcycle of every member.  Mixed: the batched tile launch, then each
// other member's fused single-state launch.  FP64: each other member's own
// element launch, the batched element launches (3-dof, then 6-dof members),
// then the node launch over all members.  Member m's current buffer is
// base_cur(m) ^ flip.
cudaError_t launch_one(mevp_ensemble *e, int flip) {
  cudaError_t err = cudaSuccess;
  if (e->prec == MEVP_MIXED) {
    if (e->nwork > 0)
      err = mevp::launch_ensemble_mixed(e->d_mem, e->d_work, e->nwork, e->shape, e->grid, flip,
                                        e->stream);
    for (size_t i = 0; i < e->solo.size() && err == cudaSuccess; ++i) {
      const mevp_state *s = e->members[e->solo[i]];
      const int cur = e->host_mem[e->solo[i]].base_cur ^ flip;
      err = mevp::launch_subcycle_mixed(s->d, s->rheo, s->prm, s->has_vo, cur, e->stream,
                                        nullptr, true, s->maps);
    }
    return err;
  }
  for (size_t i = 0; i < e->solo.size() && err == cudaSuccess; ++i) {
    const mevp_state *s = e->members[e->solo[i]];
    const int cur = e->host_mem[e->solo[i]].base_cur ^ flip;
    err = mevp::launch_element_f64(s->d, s->rheo, cur, e->stream);
  }
  if (err == cudaSuccess)
    err = mevp::launch_ensemble_f64(e->d_mem, e->d_work, e->n3, 3, e->shape, e->grid3, flip,
                                    e->stream);
  if (err == cudaSuccess)
    err = mevp::launch_ensemble_f64(e->d_mem, e->d_work + e->n3, e->nwork - e->n3, 6, e->shape,
                                    e->grid6, flip, e->stream);
  if (err != cudaSuccess) return err;
  return mevp::launch_ensemble_f64_node(e->d_mem, e->d_nwork, e->nnwork, e->grid_n, flip,
                                        e->stream);
}

int chunk_graph(mevp_ensemble *e, int flip, int len, cudaGraphExec_t *out) {
  for (auto &g : e->graphs)
    if (g.flip == flip && g.len == len) {
      *out = g.exec;
      return MEVP_OK;
    }
  cudaGraph_t graph = nullptr;
  cudaError_t err = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal);
  if (err != cudaSuccess) return mevp::api_cuda_fail(err, "ensemble: begin capture");
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < len && le == cudaSuccess; ++k) le = launch_one(e, flip ^ (k & 1));
  err = cudaStreamEndCapture(e->stream, &graph);
  if (le != cudaSuccess || err != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return mevp::api_cuda_fail(le != cudaSuccess ? le : err, "ensemble: capture");
  }
  cudaGraphExec_t exec = nullptr;
  err = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (err != cudaSuccess) return mevp::api_cuda_fail(err, "ensemble: instantiate");
  e->graphs.push_back({flip, len, exec});
  *out = exec;
  return MEVP_OK;
}

int check_ensemble(const mevp_ensemble *e) {
  if (!e) return efail(MEVP_ERR_ARG, "ensemble is NULL");
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return mevp::api_cuda_fail(err, "cudaGetDevice");
  if (dev != e->device)
    return efail(MEVP_ERR_STATE, "current device %d is not the ensemble's device %d", dev,
                 e->device);
  return MEVP_OK;
}

// n subcycles of every member, flipping the members' buffer index.
int run(mevp_ensemble *e, int n, bool graphs_allowed) {
  int flip = 0;
  int rc = sync_descriptors(e, &flip);
  if (rc) return rc;
  const bool graphs = graphs_allowed && e->use_graphs && e->stream != nullptr;
  int i = 0;
  while (i < n) {
    if (!graphs || n - i < kMinGraphChunk) {
      cudaError_t err = launch_one(e, flip);
      if (err != cudaSuccess) return mevp::api_cuda_fail(err, "ensemble: launch");
      flip ^= 1;
      ++i;
      continue;
    }
    const int len = std::min(n - i, kMaxGraphChunk);
    cudaGraphExec_t exec = nullptr;
    if ((rc = chunk_graph(e, flip, len, &exec))) return rc;
    cudaError_t err = cudaGraphLaunch(exec, e->stream);
    if (err != cudaSuccess) return mevp::api_cuda_fail(err, "ensemble: graph launch");
    flip ^= (len & 1);
    i += len;
  }
  if (n & 1)
    for (mevp_state *s : e->members) s->cur ^= 1;
  return MEVP_OK;
}

}  // namespace

extern "C" {

int mevp_ensemble_create(mevp_state *const *members, int n, mevp_ensemble **out) {
  if (!out) return efail(MEVP_ERR_ARG, "ensemble_create: out is NULL");
  *out = nullptr;
  if (!members || n < 1) return efail(MEVP_ERR_ARG, "ensemble_create: need at least one member");
  for (int i = 0; i < n; ++i) {
    int rc = mevp::api_check_state(members[i]);
    if (rc) return rc;
    for (int j = 0; j < i; ++j)
      if (members[j] == members[i])
        return efail(MEVP_ERR_ARG, "ensemble_create: member %d repeats member %d", i, j);
    if (members[i]->prec != members[0]->prec)
      return efail(MEVP_ERR_ARG, "ensemble_create: members must share one precision");
    if (members[i]->stream != members[0]->stream)
      return efail(MEVP_ERR_ARG, "ensemble_create: members must share one stream");
  }
  mevp_ensemble *e = new (std::nothrow) mevp_ensemble;
  if (!e) return efail(MEVP_ERR_OOM, "ensemble_create: host allocation failed");
  e->members.assign(members, members + n);
  e->prec = members[0]->prec;
  e->device = members[0]->device;
  e->stream = members[0]->stream;
  e->shape = 1;
  cudaError_t err = cudaMalloc(&e->d_mem, sizeof(EnsMember) * n);
  if (err != cudaSuccess) {
    cudaGetLastError();
    delete e;
    return efail(MEVP_ERR_OOM, "ensemble_create: descriptor allocation failed");
  }
  int rc = build_work(e);
  if (rc) {
    mevp_ensemble_destroy(e);
    return rc;
  }
  *out = e;
  return MEVP_OK;
}

void mevp_ensemble_destroy(mevp_ensemble *e) {
  if (!e) return;
  cudaStreamSynchronize(e->stream);
  drop_graphs(e);
  if (e->d_mem) cudaFree(e->d_mem);
  if (e->d_work) cudaFree(e->d_work);
  if (e->d_nwork) cudaFree(e->d_nwork);
  delete e;
}

int mevp_ensemble_shapes(int precision, int *dims, int max, int *count) {
  if (precision != MEVP_FP64 && precision != MEVP_MIXED)
    return efail(MEVP_ERR_ARG, "ensemble_shapes: precision %d unknown", precision);
  const int n = shape_count(precision);
  if (count) *count = n;
  for (int i = 0; i < n && i < max && dims; ++i) {
    if (precision == MEVP_MIXED) {
      dims[2 * i] = mevp::kMixTiles[i][0];
      dims[2 * i + 1] = mevp::kMixTiles[i][1];
    } else {
      dims[2 * i] = mevp::kF64Blocks[i];
      dims[2 * i + 1] = 1;
    }
  }
  return MEVP_OK;
}

int mevp_ensemble_set_shape(mevp_ensemble *e, int shape) {
  int rc = check_ensemble(e);
  if (rc) return rc;
  if (shape < 0 || shape >= shape_count(e->prec))
    return efail(MEVP_ERR_ARG, "ensemble_set_shape: shape %d out of range", shape);
  if (shape == e->shape) return MEVP_OK;
  cudaError_t err = cudaStreamSynchronize(e->stream);
  if (err != cudaSuccess) return mevp::api_cuda_fail(err, "ensemble_set_shape");
  e->shape = shape;
  return build_work(e);
}

int mevp_ensemble_set_graphs(mevp_ensemble *e, int on) {
  int rc = check_ensemble(e);
  if (rc) return rc;
  e->use_graphs = on != 0;
  return MEVP_OK;
}

int mevp_ensemble_begin_step(mevp_ensemble *e) {
  int rc = check_ensemble(e);
  if (rc) return rc;
  for (mevp_state *s : e->members)
    if ((rc = mevp_begin_step(s))) return rc;
  return MEVP_OK;
}

int mevp_ensemble_run_subcycles(mevp_ensemble *e, int n) {
  mevp::NvtxRange nvtx_range_("mevp_ensemble_run_subcycles");
  int rc = check_ensemble(e);
  if (rc) return rc;
  if (n < 0) return efail(MEVP_ERR_ARG, "ensemble_run_subcycles: n=%d < 0", n);
  for (size_t m = 0; m < e->members.size(); ++m)
    if (!e->members[m]->prepared)
      return efail(MEVP_ERR_STATE, "ensemble_run_subcycles: member %zu needs mevp_begin_step", m);
  return run(e, n, true);
}

int mevp_ensemble_autotune(mevp_ensemble *e, int trial_subcycles, int *best) {
  mevp::NvtxRange nvtx_range_("mevp_ensemble_autotune");
  int rc = check_ensemble(e);
  if (rc) return rc;
  if (trial_subcycles < 1) return efail(MEVP_ERR_ARG, "ensemble_autotune: trial_subcycles < 1");
  for (size_t m = 0; m < e->members.size(); ++m)
    if (!e->members[m]->prepared)
      return efail(MEVP_ERR_STATE, "ensemble_autotune: member %zu needs mevp_begin_step", m);
  // snapshot the fields the trials overwrite: current velocity and stress
  struct Snap {
    void *vel;
    void *S;
    size_t vbytes, sbytes;
    int cur;
  };
  std::vector<Snap> snaps;
  size_t total = 0;
  for (mevp_state *s : e->members) {
    Snap sn{};
    sn.cur = s->cur;
    if (e->prec == MEVP_MIXED) {
      sn.vbytes = sizeof(float4) * s->d.nn;
      sn.sbytes = sizeof(float) * 3 * s->ns * s->d.ne;
    } else {
      sn.vbytes = sizeof(double) * 2 * s->d.nn;
      sn.sbytes = sizeof(double) * 3 * s->ns * s->d.ne;
    }
    total += sn.vbytes + sn.sbytes;
    snaps.push_back(sn);
  }
  char *buf = nullptr;
  cudaError_t err = cudaMalloc(&buf, total);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return efail(MEVP_ERR_OOM, "ensemble_autotune: snapshot allocation of %zu bytes failed", total);
  }
  auto fields = [&](size_t m, void *&v, void *&S) {
    mevp_state *s = e->members[m];
    if (e->prec == MEVP_MIXED) {
      v = s->d.vel4[snaps[m].cur];
      S = s->d.S32[snaps[m].cur];
    } else {
      v = s->d.vel[snaps[m].cur];
      S = s->d.S;
    }
  };
  size_t off = 0;
  for (size_t m = 0; m < snaps.size(); ++m) {
    void *v, *S;
    fields(m, v, S);
    snaps[m].vel = buf + off;
    off += snaps[m].vbytes;
    snaps[m].S = buf + off;
    off += snaps[m].sbytes;
    cudaMemcpyAsync(snaps[m].vel, v, snaps[m].vbytes, cudaMemcpyDeviceToDevice, e->stream);
    cudaMemcpyAsync(snaps[m].S, S, snaps[m].sbytes, cudaMemcpyDeviceToDevice, e->stream);
  }
  const int original = e->shape;
  int choice = original;
  float best_ms = 0.f;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  for (int c = 0; c < shape_count(e->prec) && !rc; ++c) {
    if ((rc = mevp_ensemble_set_shape(e, c))) break;
    if ((rc = run(e, 2, false))) break;  // warm-up
    cudaEventRecord(t0, e->stream);
    if ((rc = run(e, trial_subcycles, false))) break;
    cudaEventRecord(t1, e->stream);
    err = cudaEventSynchronize(t1);
    if (err != cudaSuccess) {
      rc = mevp::api_cuda_fail(err, "ensemble_autotune: trial");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (c == 0 || ms < best_ms) {
      best_ms = ms;
      choice = c;
    }
  }
  // restore the members exactly as they were
  for (size_t m = 0; m < snaps.size(); ++m) {
    e->members[m]->cur = snaps[m].cur;
    void *v, *S;
    fields(m, v, S);
    cudaMemcpyAsync(v, snaps[m].vel, snaps[m].vbytes, cudaMemcpyDeviceToDevice, e->stream);
    cudaMemcpyAsync(S, snaps[m].S, snaps[m].sbytes, cudaMemcpyDeviceToDevice, e->stream);
  }
  err = cudaStreamSynchronize(e->stream);
  cudaFree(buf);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (!rc && err != cudaSuccess) rc = mevp::api_cuda_fail(err, "ensemble_autotune: restore");
  if (rc) {
    mevp_ensemble_set_shape(e, original);
    return rc;
  }
  if ((rc = mevp_ensemble_set_shape(e, choice))) return rc;
  if (best) *best = choice;
  return MEVP_OK;
}

}  // extern "C"
