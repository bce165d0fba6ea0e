// Whole decompositions as one CUDA graph.
//
// Per mode the graph holds the initial-guess chain (Sec. 4) followed by a
// conditional WHILE node whose body is one ALS sweep (one tensor pass plus the
// small FP64 kernels); mixed-precision modes have a first WHILE node of
// tensor-core bulk sweeps. The stop rule (Eq. 5.01) is evaluated on the device by
// the single-CTA TEST kernel, which clears the loop condition when the mode is
// done, so a full st-HOSVD-ALS or t-HOSVD-ALS runs with no host round trip.
// Graphs are built once per context and output-pointer set and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace tals {

struct GraphEntry {
  int kind = 0;                       // 0 st-HOSVD, 1 t-HOSVD
  const void* A = nullptr;            // the input tensor the graph reads
  void* G = nullptr;
  void* U[TALS_MAX_NDIM] = {};
  cudaGraphExec_t exec = nullptr;
  int nsp = 0;                        // t-HOSVD: spart entries of the last projection
};

struct GraphCache {
  std::vector<GraphEntry> entries;
};

namespace {

tals_status ensure_streams(tals_ctx* c) {
  for (int i = 0; i < 2; ++i)
    if (!c->cap[i]) {
      cudaError_t e = cudaStreamCreateWithFlags(&c->cap[i], cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    }
  if (!c->graphs) c->graphs = new GraphCache();
  return TALS_OK;
}

// Append, on c->cap[0] (capturing), a conditional WHILE node whose body (captured
// on c->cap[1]) is `body`; the loop's handle goes to j.cond for the body's TEST
// kernel.
template <typename Body>
tals_status capture_while(tals_ctx* c, ModeJob& j, Body body) {
  cudaStream_t cs = c->cap[0];
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) return cuda_fail(e, "capture info");
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return cuda_fail(e, "conditional handle");
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t wnode;
  std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
  e = cudaGraphAddNode(&wnode, g, dv.data(), nullptr, dv.size(), &p);
  if (e != cudaSuccess) return cuda_fail(e, "while node");
  e = cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return cuda_fail(e, "capture dependencies");
  cudaGraph_t bg = p.conditional.phGraph_out[0];
  cudaStream_t bs = c->cap[1];
  e = cudaStreamBeginCaptureToGraph(bs, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return cuda_fail(e, "body capture");
  c->stream = bs;
  j.cond = (unsigned long long)h;
  j.has_cond = 1;
  tals_status st = body();
  cudaGraph_t body_out = nullptr;
  e = cudaStreamEndCapture(bs, &body_out);
  c->stream = cs;
  j.has_cond = 0;
  if (st != TALS_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "body capture end");
  return TALS_OK;
}

// Capture, on c->cap[0] (already capturing), the init chain, the sweep loop(s)
// and the factor copy of one mode. Modes that run mixed-precision bulk sweeps
// get two loops: the tensor-core sweeps (left when the bulk phase ends) and the
// FP32 sweeps (left when Eq. 5.01 fires).
tals_status capture_mode(tals_ctx* c, ModeJob& j, bool set_norm_a, void* U_out) {
  tals_status st = mode_setup(c, j);
  if (st != TALS_OK) return st;
  cudaStream_t cs = c->cap[0];
  c->stream = cs;
  j.has_cond = 0;
  if (mixed_tc_mode(c, j)) {
    const int grid = mixed_grid(c, j);
    if (grid < 1) return fail(TALS_ENOTSUP, "no room for the tensor-core partials");
    if ((st = mixed_init_launch(c, j, set_norm_a, grid)) != TALS_OK) return st;
    if ((st = capture_while(c, j, [&] { return mixed_bulk_sweep_launch(c, j, grid); })) != TALS_OK)
      return st;
  } else {
    if ((st = mode_init_launch(c, j, set_norm_a)) != TALS_OK) return st;
  }
  if ((st = capture_while(c, j, [&] { return mode_sweep_launch(c, j); })) != TALS_OK) return st;
  if (U_out) {
    cudaError_t e = launch_copy(U_out, c->Lt, (size_t)j.v.I * j.R * c->esz, cs);
    if (e != cudaSuccess) return cuda_fail(e, "factor copy");
  }
  return TALS_OK;
}

GraphEntry* find(tals_ctx* c, int kind, void* G, void* const* U) {
  for (auto& en : c->graphs->entries) {
    if (en.kind != kind || en.G != G || en.A != c->A) continue;
    bool same = true;
    for (int n = 0; n < c->N; ++n)
      if (en.U[n] != (U ? U[n] : nullptr)) same = false;
    if (same) return &en;
  }
  return nullptr;
}

tals_status build(tals_ctx* c, int kind, void* G_out, void* const* U_out, GraphEntry* out) {
  cudaStream_t user = c->stream;
  cudaStream_t cs = c->cap[0];
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return cuda_fail(e, "begin capture");
  tals_status st = TALS_OK;
  const int N = c->N;
  long long d[TALS_MAX_NDIM];
  for (int m = 0; m < N; ++m) d[m] = c->dims[m];
  if (kind == 0) {
    const void* cur = c->A;
    for (int idx = 0; idx < N && st == TALS_OK; ++idx) {
      const int n = c->order[idx];
      ModeJob j;
      j.n = n;
      j.v = view_of(d, N, n);
      j.R = c->ranks[n];
      j.X = cur;
      j.Wdest = (idx == N - 1) ? G_out : c->tbuf[idx & 1];
      st = capture_mode(c, j, idx == 0, U_out ? U_out[n] : nullptr);
      cur = j.Wdest;
      d[n] = c->ranks[n];
    }
  } else {
    for (int n = 0; n < N && st == TALS_OK; ++n) {
      ModeJob j;
      j.n = n;
      j.v = view_of(d, N, n);
      j.R = c->ranks[n];
      j.X = c->A;
      j.Wdest = (n == N - 1) ? c->tbuf[0] : nullptr;
      st = capture_mode(c, j, n == 0, U_out[n]);
    }
    d[N - 1] = c->ranks[N - 1];
    const void* cur = c->tbuf[0];
    for (int m = 0; m < N - 1 && st == TALS_OK; ++m) {
      ModeView v = view_of(d, N, m);
      void* dest = (m == N - 2) ? G_out : c->tbuf[(m + 1) & 1];
      c->stream = cs;   // project_mode launches on the context's stream
      st = project_mode(c, cur, v, c->ranks[m], U_out[m], dest, &out->nsp);
      cur = dest;
      d[m] = c->ranks[m];
    }
    if (st == TALS_OK) {
      e = cudaMemcpyAsync(c->host_d, c->spart, out->nsp * sizeof(double), cudaMemcpyDeviceToHost, cs);
      if (e != cudaSuccess) st = cuda_fail(e, "stats copy");
    }
  }
  if (st == TALS_OK) {
    e = cudaMemcpyAsync(c->st_host, c->st, TALS_MAX_NDIM * sizeof(ModeState),
                        cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->host_d + c->host_d_n - 1, c->norm_a2, sizeof(double),
                          cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) st = cuda_fail(e, "stats copy");
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cs, &g);
  c->stream = user;
  if (st != TALS_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "end capture");
  e = cudaGraphInstantiate(&out->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
  out->kind = kind;
  out->G = G_out;
  out->A = c->A;
  for (int n = 0; n < N; ++n) out->U[n] = U_out ? U_out[n] : nullptr;
  return TALS_OK;
}

// The cached graph for (kind, c->A, G, U), built on first use.
tals_status entry(tals_ctx* c, int kind, void* G_out, void* const* U_out, GraphEntry** out) {
  tals_status st = ensure_streams(c);
  if (st != TALS_OK) return st;
  GraphEntry* en = find(c, kind, G_out, U_out);
  if (!en) {
    GraphEntry fresh;
    if ((st = build(c, kind, G_out, U_out, &fresh)) != TALS_OK) return st;
    c->graphs->entries.push_back(fresh);
    en = &c->graphs->entries.back();
  }
  *out = en;
  return TALS_OK;
}

// Status and statistics of the last decomposition launched on c->stream, once
// the stream has been synchronized (the graph's last nodes copy them to pinned
// host memory).
tals_status collect(tals_ctx* c, int kind, const GraphEntry* en, tals_stats* stats) {
  tals_status st;
  if ((st = mixed_check(c)) != TALS_OK) return st;
  // statistics from the pinned copies written by the graph's last nodes
  tals_stats local;
  std::memset(&local, 0, sizeof(local));
  const int N = c->N;
  for (int n = 0; n < N; ++n) {
    const ModeState& ms = c->st_host[n];
    local.err_per_mode[n] = ms.e_cur;
    local.sweeps[n] = ms.k;
    local.bulk_sweeps[n] = ms.bulk;
    local.tc_sweeps[n] = ms.tc_resid ? ms.k - ms.bulk : 0;
    local.split_capable[n] = ms.split_ok;
    local.split_sweeps[n] = ms.nsplit;
    local.two_product[n] = ms.prod;
    local.converged[n] = ms.converged;
    if (ms.status && !local.status) local.status = ms.status;
  }
  const double na2 = c->host_d[c->host_d_n - 1];
  local.norm_a = std::sqrt(na2);
  if (kind == 0) {
    double e2 = 0.0;
    for (int n = 0; n < N; ++n) e2 += local.err_per_mode[n] * local.err_per_mode[n];
    local.rel_err = na2 > 0 ? std::sqrt(e2 / na2) : 0.0;
    for (int i = 0; i < N; ++i) local.order[i] = c->order[i];
  } else {
    double g2 = 0.0;
    for (int i = 0; i < en->nsp; ++i) g2 += c->host_d[i];
    local.rel_err = t_hosvd_rel_err(c, na2, g2);
    for (int i = 0; i < N; ++i) local.order[i] = i;
  }
  if (stats) *stats = local;
  if (local.status)
    return fail((tals_status)local.status,
                "a Gram matrix was not positive definite (truncation above the numerical rank, "
                "Remark 3)");
  return TALS_OK;
}

tals_status run(tals_ctx* c, int kind, void* G_out, void* const* U_out, tals_stats* stats) {
  GraphEntry* en = nullptr;
  tals_status st = entry(c, kind, G_out, U_out, &en);
  if (st != TALS_OK) return st;
  cudaError_t e = cudaGraphLaunch(en->exec, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  return collect(c, kind, en, stats);
}

}  // namespace

tals_status st_hosvd_graph_launch(tals_ctx* c, void* G_out, void* const* U_out) {
  GraphEntry* en = nullptr;
  tals_status st = entry(c, 0, G_out, U_out, &en);
  if (st != TALS_OK) return st;
  cudaError_t e = cudaGraphLaunch(en->exec, c->stream);
  return e == cudaSuccess ? TALS_OK : cuda_fail(e, "graph launch");
}

tals_status st_hosvd_graph_collect(tals_ctx* c, void* G_out, void* const* U_out, tals_stats* stats) {
  GraphEntry* en = find(c, 0, G_out, U_out);
  if (!en) return fail(TALS_EINVAL, "no st-HOSVD graph launched for these buffers");
  return collect(c, 0, en, stats);
}

tals_status st_hosvd_graph(tals_ctx* c, void* G_out, void* const* U_out, tals_stats* st) {
  return run(c, 0, G_out, U_out, st);
}

tals_status t_hosvd_graph(tals_ctx* c, void* G_out, void* const* U_out, tals_stats* st) {
  return run(c, 1, G_out, U_out, st);
}

void graphs_destroy(tals_ctx* c) {
  if (c->graphs) {
    for (auto& en : c->graphs->entries)
      if (en.exec) cudaGraphExecDestroy(en.exec);
    delete c->graphs;
    c->graphs = nullptr;
  }
  for (int i = 0; i < 2; ++i)
    if (c->cap[i]) {
      cudaStreamDestroy(c->cap[i]);
      c->cap[i] = nullptr;
    }
}

}  // namespace tals
