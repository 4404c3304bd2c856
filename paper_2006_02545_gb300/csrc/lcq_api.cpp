// C ABI of liblcq: contexts, near lists, corrections, corrected potentials.
// Host orchestration only; every numerical step runs in the kernels of lcq_kernels.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <functional>
#include <thread>
#include <vector>

#include "lcq_internal.h"
#include "lcq_launch.h"

using namespace lcq;

namespace {

const char* kStatusNames[] = {"ok",
                              "invalid argument",
                              "non-finite coordinates",
                              "degenerate patch (Jacobian <= 0 at a node)",
                              "adaptive refinement reached max_depth",
                              "internal capacity exceeded",
                              "CUDA runtime error",
                              "device out of memory",
                              "reference tables could not be built",
                              "timeout"};

lcq_status fail(lcq_ctx* c, lcq_status s, const char* msg) {
  if (c) c->last_error = msg;
  return s;
}

lcq_status cuda_fail(lcq_ctx* c, cudaError_t e, const char* where) {
  if (c) {
    c->last_error = std::string(where) + ": " + cudaGetErrorString(e);
  }
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? LCQ_ERR_OOM : LCQ_ERR_CUDA;
}

#define CK(call)                                             \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

template <class T>
cudaError_t dalloc(cudaStream_t st, T** p, size_t count) {
  *p = nullptr;
  return cudaMallocAsync(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T), st);
}

template <class T>
void dfree(cudaStream_t st, T*& p) {
  if (p) cudaFreeAsync(p, st);
  p = nullptr;
}

// Runs f when the enclosing scope ends unless dismissed: a call that fails part-way
// releases what it has set up (the partly built handle, its work buffers).
template <class F>
class ScopeExit {
 public:
  explicit ScopeExit(F f) : f_(std::move(f)) {}
  ~ScopeExit() {
    if (armed_) f_();
  }
  void dismiss() { armed_ = false; }
  ScopeExit(const ScopeExit&) = delete;
  ScopeExit& operator=(const ScopeExit&) = delete;

 private:
  F f_;
  bool armed_ = true;
};
template <class F>
ScopeExit<F> on_exit(F f) {
  return ScopeExit<F>(std::move(f));
}

int default_self_order(double eps) {
  const double e = std::min(std::max(eps, 1e-15), 1e-1);
  const double digits = -log10(e);
  const int o = (int)ceil(1.2 * digits - 1e-9) + 3;
  return std::min(24, std::max(6, o));
}

lcq_status ensure_rules(lcq_ctx* ctx) {
  if (ctx->rules_ready) return LCQ_OK;
  RuleTables& r = ctx->rules;
  if (!build_rule_tables(&r)) return fail(ctx, LCQ_ERR_TABLES, "rule tables");
  cudaStream_t st = ctx->stream;
  auto undo = on_exit([&] {
    dfree(st, r.doff);
    dfree(st, r.du);
    dfree(st, r.dv);
    dfree(st, r.dw);
    dfree(st, r.dgl_off);
    dfree(st, r.dgl_x);
    dfree(st, r.dgl_w);
  });
  CK(dalloc(st, &r.doff, r.off.size()));
  CK(dalloc(st, &r.du, r.u.size()));
  CK(dalloc(st, &r.dv, r.v.size()));
  CK(dalloc(st, &r.dw, r.w.size()));
  CK(dalloc(st, &r.dgl_off, r.gl_off.size()));
  CK(dalloc(st, &r.dgl_x, r.gl_x.size()));
  CK(dalloc(st, &r.dgl_w, r.gl_w.size()));
  CK(cudaMemcpyAsync(r.doff, r.off.data(), r.off.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(r.du, r.u.data(), r.u.size() * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(r.dv, r.v.data(), r.v.size() * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(r.dw, r.w.data(), r.w.size() * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(r.dgl_off, r.gl_off.data(), r.gl_off.size() * sizeof(int),
                     cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(r.dgl_x, r.gl_x.data(), r.gl_x.size() * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(r.dgl_w, r.gl_w.data(), r.gl_w.size() * 8, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  undo.dismiss();
  ctx->rules_ready = true;
  return LCQ_OK;
}

// A degree's device tables are all present (dV set) or none is: a failed upload frees
// what it allocated, so that the next call starts again.
lcq_status ensure_deg(lcq_ctx* ctx, int d) {
  DegTables& t = ctx->deg[d];
  if (t.dV) return LCQ_OK;
  if (!build_deg_tables(d, &t)) return fail(ctx, LCQ_ERR_TABLES, "degree tables");
  cudaStream_t st = ctx->stream;
  auto undo = on_exit([&] {
    dfree(st, t.dV);
    dfree(st, t.dnodes);
    dfree(st, t.dDuv);
  });
  const int n = t.n;
  std::vector<double> nodes(3 * n);
  for (int i = 0; i < n; ++i) {
    nodes[i] = t.u[i];
    nodes[n + i] = t.v[i];
    nodes[2 * n + i] = t.w[i];
  }
  CK(dalloc(st, &t.dV, (size_t)n * n));
  CK(dalloc(st, &t.dnodes, (size_t)3 * n));
  CK(cudaMemcpyAsync(t.dV, t.V.data(), (size_t)n * n * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(t.dnodes, nodes.data(), (size_t)3 * n * 8, cudaMemcpyHostToDevice, st));
  std::vector<double> duv(t.Du);
  duv.insert(duv.end(), t.Dv.begin(), t.Dv.end());
  CK(dalloc(st, &t.dDuv, duv.size()));
  CK(cudaMemcpyAsync(t.dDuv, duv.data(), duv.size() * 8, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  undo.dismiss();
  return LCQ_OK;
}


// Grid over the centroid box b[0..2]..b[3..5] with cell edge a little above max eta_j R_j
// (b[6]), so that a ball of radius eta_j R_j never reaches beyond the neighbouring cells even
// after rounding of the cell coordinates; coarsened until it has at most
// max(4096, 2 P) cells.
GridSpec make_grid(const double* b, int64_t P) {
  double ext = 0.0;
  for (int a = 0; a < 3; ++a) ext = std::max(ext, b[3 + a] - b[a]);
  double h = b[6] * (1.0 + 1e-6);
  if (!(h > ext * 1e-9)) h = std::max(ext * 1e-9, 1e-300);
  const int64_t cap = std::max<int64_t>(4096, 2 * P);
  GridSpec g{};
  for (;;) {
    g.inv_h = 1.0 / h;
    int64_t tot = 1;
    int n[3];
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      const double f = std::floor((b[3 + a] - b[a]) * g.inv_h);
      if (!(f < 1e6)) {
        ok = false;
        break;
      }
      n[a] = (int)f + 1;
      tot *= n[a];
    }
    if (ok && tot <= cap) {
      for (int a = 0; a < 3; ++a) g.lo[a] = b[a];
      g.nx = n[0];
      g.ny = n[1];
      g.nz = n[2];
      return g;
    }
    h *= 1.25;
  }
}
}  // namespace

// ============================================================================ API
extern "C" {

void lcq_params_default(lcq_params* p) {
  if (!p) return;
  p->eps = 1e-6;
  p->eta = -1.0;
  p->eta1 = 1.25;
  p->eps_loosen = 1.0;
  p->max_depth = 24;
  p->m_max = 24;
  p->self_order = 0;
  p->leaf_order = 0;
  p->n_test_dirs = 0;
  p->test_dirs = nullptr;
}

const char* lcq_status_string(lcq_status s) {
  const int i = (int)s;
  if (i < 0 || i > 9) return "unknown status";
  return kStatusNames[i];
}

const char* lcq_last_error(const lcq_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

lcq_status lcq_ref_nodes(int deg, double* u, double* v, double* w) {
  if (deg < 1 || deg > kMaxDeg || !u || !v || !w) return LCQ_ERR_ARG;
  DegTables t;
  if (!build_deg_tables(deg, &t)) return LCQ_ERR_TABLES;
  for (int i = 0; i < t.n; ++i) {
    u[i] = t.u[i];
    v[i] = t.v[i];
    w[i] = t.w[i];
  }
  return LCQ_OK;
}

lcq_status lcq_create(lcq_ctx** out, int device, void* cuda_stream) {
  if (!out) return LCQ_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return e != cudaSuccess ? LCQ_ERR_CUDA : LCQ_ERR_ARG;
  }
  lcq_ctx* ctx = new lcq_ctx();
  ctx->device = device;
  ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  auto undo = on_exit([&] { lcq_destroy(ctx); });
  CK(cudaSetDevice(device));
  CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
  CK(cudaMalloc(&ctx->d_status, sizeof(int)));
  CK(cudaMalloc(&ctx->d_counters, 8 * sizeof(long long)));
  CK(cudaMalloc(&ctx->d_sched, 16 * sizeof(int)));
  CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_counters, 0, 8 * sizeof(long long), ctx->stream));
  CK(upload_constants(ctx->stream));
  CK(upload_constants_adjoint(ctx->stream));
  for (int i = 0; i < 8; ++i) CK(cudaEventCreate(&ctx->ev[i]));
  int prio_least = 0, prio_greatest = 0;
  CK(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
  CK(cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, prio_least));
  CK(cudaStreamCreateWithPriority(&ctx->hi, cudaStreamNonBlocking, prio_greatest));
  CK(cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&ctx->done, cudaEventDisableTiming));
  for (int i = 0; i < 2; ++i) CK(cudaEventCreate(&ctx->ev_self[i]));
  lcq_status s = ensure_rules(ctx);
  if (s != LCQ_OK) return s;
  undo.dismiss();
  *out = ctx;
  return LCQ_OK;
}

void lcq_destroy(lcq_ctx* ctx) {
  if (!ctx) return;
  for (auto& kv : ctx->tune) {
    if (kv.second.e0) cudaEventDestroy(kv.second.e0);
    if (kv.second.e1) cudaEventDestroy(kv.second.e1);
  }
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (int d = 0; d <= kMaxDeg; ++d) {
    dfree(ctx->stream, ctx->deg[d].dV);
    dfree(ctx->stream, ctx->deg[d].dnodes);
    dfree(ctx->stream, ctx->deg[d].dDuv);
  }
  RuleTables& r = ctx->rules;
  dfree(ctx->stream, r.doff);
  dfree(ctx->stream, r.du);
  dfree(ctx->stream, r.dv);
  dfree(ctx->stream, r.dw);
  dfree(ctx->stream, r.dgl_off);
  dfree(ctx->stream, r.dgl_x);
  dfree(ctx->stream, r.dgl_w);
  if (ctx->work) cudaFreeAsync(ctx->work, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  for (int i = 0; i < 8; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  for (cudaStream_t* sp : {&ctx->side, &ctx->hi})
    if (*sp) {
      cudaStreamSynchronize(*sp);
      cudaStreamDestroy(*sp);
    }
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  if (ctx->join) cudaEventDestroy(ctx->join);
  if (ctx->done) cudaEventDestroy(ctx->done);
  for (int i = 0; i < 2; ++i)
    if (ctx->ev_self[i]) cudaEventDestroy(ctx->ev_self[i]);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_counters);
  cudaFree(ctx->d_sched);
  cudaGetLastError();
  delete ctx;
}

lcq_status lcq_sync(lcq_ctx* ctx, int64_t timeout_ms) {
  if (!ctx) return LCQ_ERR_ARG;
  cudaSetDevice(ctx->device);
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t q = cudaStreamQuery(ctx->stream);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return cuda_fail(ctx, q, "cudaStreamQuery");
    if (timeout_ms >= 0) {
      const auto el = std::chrono::duration_cast<std::chrono::milliseconds>(
                          std::chrono::steady_clock::now() - t0).count();
      if (el > timeout_ms) return fail(ctx, LCQ_ERR_TIMEOUT, "lcq_sync timed out");
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  int st = 0;
  CK(cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemset(ctx->d_status, 0, sizeof(int)));
  if (st & kStNonFinite) return fail(ctx, LCQ_ERR_NONFINITE, "non-finite coordinates");
  if (st & kStDegenerate) return fail(ctx, LCQ_ERR_DEGENERATE_PATCH, "degenerate patch");
  if (st & kStCapacity) return fail(ctx, LCQ_ERR_CAPACITY, "work storage exceeded");
  if (st & kStMaxDepth) return fail(ctx, LCQ_ERR_MAX_DEPTH, "max_depth reached");
  return LCQ_OK;
}

lcq_status lcq_stage_times(lcq_ctx* ctx, float* ms6, int64_t* launches) {
  if (!ctx) return LCQ_ERR_ARG;
  cudaSetDevice(ctx->device);
  CK(cudaStreamSynchronize(ctx->stream));
  if (ms6) {
    CK(cudaEventElapsedTime(&ms6[0], ctx->ev[0], ctx->ev[1]));
    for (int i = 0; i < 5; ++i) CK(cudaEventElapsedTime(&ms6[1 + i], ctx->ev[2 + i], ctx->ev[3 + i]));
    // the self weights run on the low-priority stream, concurrently with stages 1-3
    CK(cudaEventElapsedTime(&ms6[4], ctx->ev_self[0], ctx->ev_self[1]));
  }
  if (launches) *launches = ctx->launches_near + ctx->launches_corr;
  return LCQ_OK;
}

lcq_status lcq_counters(lcq_ctx* ctx, int64_t* out8) {
  if (!ctx || !out8) return LCQ_ERR_ARG;
  cudaSetDevice(ctx->device);
  CK(cudaStreamSynchronize(ctx->stream));
  long long h[8];
  CK(cudaMemcpy(h, ctx->d_counters, sizeof(h), cudaMemcpyDeviceToHost));
  for (int i = 0; i < 8; ++i) out8[i] = h[i];
  out8[5] = ctx->last_group_size;
  out8[6] = ctx->last_items;
  out8[7] = ctx->last_forms;
  return LCQ_OK;
}

// ---------------------------------------------------------------------------- near lists
static lcq_status build_near_impl(lcq_ctx* ctx, const lcq_surface* surf, int n_groups,
                                  const int64_t* group_patch_off, const double* tgt_xyz,
                                  const int64_t* tgt_node, const int32_t* tgt_group, int64_t NT,
                                  const lcq_params* params, lcq_near** out) {
  if (!ctx || !surf || !params || !out || NT < 0) return fail(ctx, LCQ_ERR_ARG, "null argument");
  *out = nullptr;
  const int64_t P = surf->n_patches;
  if (P <= 0 || !surf->deg || !surf->node_off || !surf->xyz)
    return fail(ctx, LCQ_ERR_ARG, "empty or incomplete surface");
  const bool grouped = group_patch_off != nullptr;
  if (grouped) {
    if (n_groups < 1 || group_patch_off[0] != 0 || group_patch_off[n_groups] != P)
      return fail(ctx, LCQ_ERR_ARG, "surface ranges must start at 0 and end at n_patches");
    for (int g = 0; g < n_groups; ++g)
      if (group_patch_off[g + 1] <= group_patch_off[g])
        return fail(ctx, LCQ_ERR_ARG, "every surface of a batch needs at least one patch");
  }
  if (NT > 0 && (!tgt_xyz || !tgt_node)) return fail(ctx, LCQ_ERR_ARG, "null targets");
  if (NT >= (int64_t)0x7fffffff) return fail(ctx, LCQ_ERR_ARG, "more than 2^31-2 targets");
  if (!(params->eps > 0.0) || !(params->eta1 > 0.0))
    return fail(ctx, LCQ_ERR_ARG, "eps and eta1 must be positive");
  if (surf->node_off[0] != 0) return fail(ctx, LCQ_ERR_ARG, "node_off[0] != 0");
  for (int64_t j = 0; j < P; ++j) {
    const int d = surf->deg[j];
    if (d < 1 || d > kMaxDeg) return fail(ctx, LCQ_ERR_ARG, "degree outside 1..10");
    if (surf->node_off[j + 1] - surf->node_off[j] != n_basis(d))
      return fail(ctx, LCQ_ERR_ARG, "node_off inconsistent with degrees");
  }
  const int64_t N = surf->node_off[P];
  if (N >= (int64_t)0x7fffffff) return fail(ctx, LCQ_ERR_ARG, "more than 2^31-1 nodes");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  ctx->launches_near = 0;
  LaunchCommon lc{st, ctx->num_sms, &ctx->launches_near};
  CK(cudaEventRecord(ctx->ev[0], st));

  lcq_near* nr = new lcq_near();
  nr->params = *params;
  nr->params.test_dirs = nullptr;
  nr->params.n_test_dirs = 0;
  nr->n_patches = P;
  nr->n_targets = NT;
  nr->n_points = N;
  nr->deg_h.assign(surf->deg, surf->deg + P);
  nr->node_off_h.assign(surf->node_off, surf->node_off + P + 1);
  nr->stream = st;
  nr->device = ctx->device;
  auto undo = on_exit([&] { lcq_near_destroy(nr); });
  // work buffers of this call, released on every return (the success path frees them
  // itself as soon as they are no longer needed)
  int64_t* goff = nullptr;
  double* bnd = nullptr;
  unsigned long long *cell_cnt = nullptr, *cell_cur = nullptr;
  int64_t* cell_ptr = nullptr;
  int32_t* cell_patch = nullptr;
  int64_t* scr = nullptr;
  int64_t *row_np = nullptr, *row_nnz = nullptr;
  unsigned long long *npair = nullptr, *nad = nullptr, *nself = nullptr, *pcur = nullptr,
                     *scur = nullptr;
  int32_t *row_tmp = nullptr, *ptmp = nullptr, *stmp = nullptr;
  auto tmp_free = on_exit([&] {
    dfree(st, goff);
    dfree(st, bnd);
    dfree(st, cell_cnt);
    dfree(st, cell_cur);
    dfree(st, cell_ptr);
    dfree(st, cell_patch);
    dfree(st, scr);
    dfree(st, row_np);
    dfree(st, row_nnz);
    dfree(st, npair);
    dfree(st, nad);
    dfree(st, nself);
    dfree(st, pcur);
    dfree(st, scur);
    dfree(st, row_tmp);
    dfree(st, ptmp);
    dfree(st, stmp);
  });
  nr->grouped = grouped;
  nr->n_groups = grouped ? n_groups : 1;
  if (grouped) nr->gpatch_off.assign(group_patch_off, group_patch_off + n_groups + 1);
  std::vector<std::vector<int>> lists(kMaxDeg + 1);
  for (int64_t j = 0; j < P; ++j) lists[surf->deg[j]].push_back((int)j);
  for (int d = 1; d <= kMaxDeg; ++d) {
    if (lists[d].empty()) continue;
    lcq_status s = ensure_deg(ctx, d);
    if (s != LCQ_OK) return s;
    nr->n_max = std::max(nr->n_max, n_basis(d));
    nr->plist_count[d] = (int)lists[d].size();
    CK(dalloc(st, &nr->plist_dev[d], lists[d].size()));
    CK(cudaMemcpyAsync(nr->plist_dev[d], lists[d].data(), lists[d].size() * sizeof(int),
                       cudaMemcpyHostToDevice, st));
  }
  const int64_t NTa = std::max<int64_t>(NT, 1);
  CK(dalloc(st, &nr->deg, P));
  CK(dalloc(st, &nr->node_off, P + 1));
  CK(cudaMemcpyAsync(nr->deg, surf->deg, P * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(nr->node_off, surf->node_off, (P + 1) * sizeof(int64_t),
                     cudaMemcpyHostToDevice, st));
  CK(dalloc(st, &nr->coef, (size_t)N * 3));
  CK(dalloc(st, &nr->cen, (size_t)P * 3));
  CK(dalloc(st, &nr->rad, P));
  CK(dalloc(st, &nr->dj, P));
  CK(dalloc(st, &nr->eta, P));
  CK(dalloc(st, &nr->eta1, P));
  CK(dalloc(st, &nr->tgt, (size_t)3 * NTa));
  CK(dalloc(st, &nr->tnode, NTa));
  CK(dalloc(st, &nr->tgt_patch, NTa));
  CK(dalloc(st, &nr->tgt_lnode, NTa));
  if (NT > 0) {
    CK(cudaMemcpyAsync(nr->tgt, tgt_xyz, (size_t)3 * NT * 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(nr->tnode, tgt_node, (size_t)NT * 8, cudaMemcpyDeviceToDevice, st));
    launch_tgt_patch(lc, nr->tgt, nr->tnode, NT, nr->node_off, P, N, nr->tgt_patch, nr->tgt_lnode,
                     ctx->d_status);
  }
  for (int d = 1; d <= kMaxDeg; ++d) {
    if (!nr->plist_count[d]) continue;
    launch_geom(d, lc, nr->plist_dev[d], nr->plist_count[d], nr->node_off, surf->xyz, N, ctx->deg[d].dV,
                ctx->deg[d].dnodes, params->eta, params->eta1, nr->coef, nr->cen, nr->rad, nr->dj,
                nr->eta, nr->eta1, ctx->d_status);
  }
  CK(cudaGetLastError());
  if (grouped) {
    CK(dalloc(st, &goff, n_groups + 1));
    CK(cudaMemcpyAsync(goff, group_patch_off, (n_groups + 1) * 8, cudaMemcpyHostToDevice, st));
    CK(dalloc(st, &nr->pgroup, P));
    CK(dalloc(st, &nr->tgroup, std::max<int64_t>(NT, 1)));
    launch_groups(lc, NT, nr->tgt_patch, goff, n_groups, tgt_group, nr->pgroup, nr->tgroup,
                  ctx->d_status);
    dfree(st, goff);
  }
  NearArgs na{nr->tgt, NT, nr->cen, nr->rad, nr->eta, nr->eta1, nr->pgroup, nr->tgroup};
  // uniform grid over the patch centroids (cell edge >= max eta_j R_j)
  CK(dalloc(st, &bnd, 8));
  launch_grid_bounds(lc, na, P, bnd);
  double hb[7];
  CK(cudaMemcpyAsync(hb, bnd, sizeof(hb), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  {
    int hst = 0;
    CK(cudaMemcpy(&hst, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (hst & kStBadGroup) {
      cudaMemset(ctx->d_status, 0, sizeof(int));
      return fail(ctx, LCQ_ERR_ARG, "target surface index outside [0, n_surfaces)");
    }
    if (hst & (kStNonFinite | kStDegenerate)) {
      cudaMemset(ctx->d_status, 0, sizeof(int));
      return fail(ctx, (hst & kStNonFinite) ? LCQ_ERR_NONFINITE : LCQ_ERR_DEGENERATE_PATCH,
                  (hst & kStNonFinite) ? "non-finite coordinates" : "degenerate patch");
    }
  }
  const GridSpec g = make_grid(hb, P);
  const int64_t ncell = (int64_t)g.nx * g.ny * g.nz;
  CK(dalloc(st, &cell_cnt, ncell + 1));
  CK(dalloc(st, &cell_cur, ncell));
  CK(dalloc(st, &cell_ptr, ncell + 1));
  CK(dalloc(st, &cell_patch, P));
  CK(cudaMemsetAsync(cell_cnt, 0, (ncell + 1) * 8, st));
  CK(cudaMemsetAsync(cell_cur, 0, ncell * 8, st));
  const int64_t mx = std::max(std::max(NT, P), ncell) + 1;
  CK(dalloc(st, &scr, 2 * ((mx + 1023) / 1024) + 4096));
  launch_cell_bins(lc, na, P, g, cell_cnt, cell_ptr, cell_cur, cell_patch, scr);

  // rows: counts, offsets, then the sorted patches of each row and the CSR columns
  CK(dalloc(st, &row_np, NT + 1));
  CK(dalloc(st, &row_nnz, NT + 1));
  CK(dalloc(st, &npair, P + 1));
  CK(dalloc(st, &nad, P + 1));
  CK(dalloc(st, &nself, P + 1));
  CK(dalloc(st, &pcur, P));
  CK(dalloc(st, &scur, P));
  CK(cudaMemsetAsync(row_np, 0, (NT + 1) * 8, st));
  CK(cudaMemsetAsync(row_nnz, 0, (NT + 1) * 8, st));
  CK(cudaMemsetAsync(npair, 0, (P + 1) * 8, st));
  CK(cudaMemsetAsync(nad, 0, (P + 1) * 8, st));
  CK(cudaMemsetAsync(nself, 0, (P + 1) * 8, st));
  CK(cudaMemsetAsync(pcur, 0, P * 8, st));
  CK(cudaMemsetAsync(scur, 0, P * 8, st));
  if (NT > 0)
    launch_row_count(lc, na, g, cell_ptr, cell_patch, nr->tgt_patch, nr->deg, row_np, row_nnz);
  CK(dalloc(st, &nr->row_ptr, NT + 1));
  CK(dalloc(st, &nr->rowp_ptr, NT + 1));
  CK(dalloc(st, &nr->pair_ptr, P + 1));
  CK(dalloc(st, &nr->ad_ptr, P + 1));
  CK(dalloc(st, &nr->an_ptr, P + 1));
  CK(dalloc(st, &nr->self_ptr, P + 1));
  launch_scan(lc, row_nnz, nr->row_ptr, NT + 1, scr);
  launch_scan(lc, row_np, nr->rowp_ptr, NT + 1, scr);
  CK(cudaGetLastError());
  int64_t tot[2];
  CK(cudaMemcpyAsync(&tot[0], nr->row_ptr + NT, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&tot[1], nr->rowp_ptr + NT, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  nr->nnz = tot[0];
  const int64_t rowp_total = tot[1];
  CK(dalloc(st, &nr->col, nr->nnz));
  CK(dalloc(st, &nr->rowp_patch, rowp_total));
  CK(dalloc(st, &nr->rowp_off, rowp_total));
  CK(dalloc(st, &row_tmp, rowp_total));
  if (NT > 0)
    launch_row_fill(lc, na, g, cell_ptr, cell_patch, nr->tgt_patch, nr->deg, nr->node_off,
                    nr->rowp_ptr, nr->row_ptr, row_tmp, nr->rowp_patch, nr->rowp_off, nr->col,
                    npair, nad, nself);
  launch_scan(lc, reinterpret_cast<int64_t*>(npair), nr->pair_ptr, P + 1, scr);
  launch_scan(lc, reinterpret_cast<int64_t*>(nad), nr->ad_ptr, P + 1, scr);
  launch_scan(lc, reinterpret_cast<int64_t*>(nself), nr->self_ptr, P + 1, scr);
  CK(cudaGetLastError());
  std::vector<int64_t> h_np(P + 1), h_nad(P + 1), h_ns(P + 1);
  CK(cudaMemcpyAsync(h_np.data(), npair, (P + 1) * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h_nad.data(), nad, (P + 1) * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h_ns.data(), nself, (P + 1) * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<int64_t> an_h(P + 1);
  int64_t acc_p = 0, acc_a = 0, acc_s = 0, acc_n = 0;
  for (int64_t j = 0; j < P; ++j) {
    nr->max_adaptive = std::max(nr->max_adaptive, h_nad[j]);
    nr->max_pairs = std::max(nr->max_pairs, h_np[j]);
    nr->max_self = std::max(nr->max_self, h_ns[j]);
    an_h[j] = acc_n;
    acc_p += h_np[j];
    acc_a += h_nad[j];
    acc_s += h_ns[j];
    acc_n += h_np[j] - h_nad[j];
  }
  an_h[P] = acc_n;
  if (acc_p >= (int64_t)0x7fffffff)
    return fail(ctx, LCQ_ERR_CAPACITY, "more than 2^31-1 near pairs");
  // patches with adaptive targets, per degree, most adaptive targets first (the adaptive
  // kernel takes them in this order from a shared counter: longest jobs first)
  for (int d = 1; d <= kMaxDeg; ++d) {
    std::vector<int> l;
    for (int j : lists[d])
      if (h_nad[j] > 0) l.push_back(j);
    std::stable_sort(l.begin(), l.end(), [&](int a, int b) { return h_nad[a] > h_nad[b]; });
    nr->ad_count[d] = (int)l.size();
    for (int j : l) {
      nr->ad_total[d] += h_nad[j];
      nr->ad_max[d] = std::max(nr->ad_max[d], h_nad[j]);
      nr->ad_nad_h[d].push_back(h_nad[j]);
    }
    if (!l.empty()) {
      CK(dalloc(st, &nr->ad_list_dev[d], l.size()));
      CK(cudaMemcpyAsync(nr->ad_list_dev[d], l.data(), l.size() * sizeof(int),
                         cudaMemcpyHostToDevice, st));
    }
  }
  nr->n_pairs = acc_p;
  nr->n_adaptive = acc_a;
  nr->n_self = acc_s;
  nr->n_annulus = acc_n;
  CK(cudaMemcpyAsync(nr->an_ptr, an_h.data(), (P + 1) * 8, cudaMemcpyHostToDevice, st));
  CK(dalloc(st, &ptmp, nr->n_pairs));
  CK(dalloc(st, &stmp, nr->n_self));
  CK(dalloc(st, &nr->pair_tgt, nr->n_pairs));
  CK(dalloc(st, &nr->pair_ad, nr->n_pairs));
  CK(dalloc(st, &nr->pair_d2, nr->n_pairs));
  CK(dalloc(st, &nr->pair_csr, nr->n_pairs));
  CK(dalloc(st, &nr->ad_pair, nr->n_adaptive));
  CK(dalloc(st, &nr->an_pair, nr->n_annulus));
  CK(dalloc(st, &nr->self_tgt, nr->n_self));
  CK(dalloc(st, &nr->self_csr, nr->n_self));
  if (NT > 0)
    launch_patch_fill(lc, na, nr->tgt_patch, P, nr->pair_ptr, nr->ad_ptr, nr->an_ptr, nr->self_ptr,
                      nr->rowp_ptr, nr->rowp_patch, nr->rowp_off, nr->row_ptr, pcur, scur, ptmp,
                      stmp, nr->pair_tgt, nr->pair_ad, nr->pair_d2, nr->pair_csr, nr->ad_pair,
                      nr->an_pair, nr->self_tgt, nr->self_csr);
  dfree(st, bnd);
  dfree(st, cell_cnt);
  dfree(st, cell_cur);
  dfree(st, cell_ptr);
  dfree(st, cell_patch);
  dfree(st, pcur);
  dfree(st, scur);
  dfree(st, ptmp);
  dfree(st, stmp);
  dfree(st, row_tmp);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ctx->ev[1], st));
  dfree(st, row_np);
  dfree(st, row_nnz);
  dfree(st, npair);
  dfree(st, nad);
  dfree(st, nself);
  dfree(st, scr);
  undo.dismiss();
  *out = nr;
  return LCQ_OK;
}

lcq_status lcq_build_near_lists(lcq_ctx* ctx, const lcq_surface* surf, const double* tgt_xyz,
                                const int64_t* tgt_node, int64_t NT, const lcq_params* params,
                                lcq_near** out) {
  return build_near_impl(ctx, surf, 1, nullptr, tgt_xyz, tgt_node, nullptr, NT, params, out);
}

lcq_status lcq_build_near_lists_batched(lcq_ctx* ctx, const lcq_surface* surf, int n_surfaces,
                                        const int64_t* surface_patch_off, const double* tgt_xyz,
                                        const int64_t* tgt_node, const int32_t* tgt_surface,
                                        int64_t NT, const lcq_params* params, lcq_near** out) {
  if (!surface_patch_off) return fail(ctx, LCQ_ERR_ARG, "null surface ranges");
  return build_near_impl(ctx, surf, n_surfaces, surface_patch_off, tgt_xyz, tgt_node, tgt_surface,
                         NT, params, out);
}

lcq_status lcq_near_set_target_normals(lcq_near* nr, const double* tgt_normal) {
  if (!nr || !tgt_normal) return LCQ_ERR_ARG;
  lcq_ctx* ctx = nullptr;
  CK(cudaSetDevice(nr->device));
  cudaStream_t st = nr->stream;
  if (!nr->unrm) CK(dalloc(st, &nr->unrm, (size_t)3 * std::max<int64_t>(nr->n_targets, 1)));
  if (nr->n_targets > 0)
    CK(cudaMemcpyAsync(nr->unrm, tgt_normal, (size_t)3 * nr->n_targets * 8,
                       cudaMemcpyDeviceToDevice, st));
  dfree(st, nr->tnrm);  // recomputed at the next S' generation
  nr->tnrm = nullptr;
  return LCQ_OK;
}

lcq_status lcq_near_info(const lcq_near* nr, int64_t* n_pairs, int64_t* n_self,
                         int64_t* n_adaptive, int64_t* nnz) {
  if (!nr) return LCQ_ERR_ARG;
  if (n_pairs) *n_pairs = nr->n_pairs;
  if (n_self) *n_self = nr->n_self;
  if (n_adaptive) *n_adaptive = nr->n_adaptive;
  if (nnz) *nnz = nr->nnz;
  return LCQ_OK;
}

lcq_status lcq_near_export(lcq_near* nr, int64_t* pair_ptr, int32_t* tgt, uint8_t* adaptive,
                           double* centroid, double* radius) {
  if (!nr) return LCQ_ERR_ARG;
  lcq_ctx* ctx = nullptr;
  CK(cudaSetDevice(nr->device));
  cudaStream_t st = nr->stream;
  if (pair_ptr)
    CK(cudaMemcpyAsync(pair_ptr, nr->pair_ptr, (nr->n_patches + 1) * 8, cudaMemcpyDeviceToHost, st));
  if (tgt && nr->n_pairs)
    CK(cudaMemcpyAsync(tgt, nr->pair_tgt, nr->n_pairs * 4, cudaMemcpyDeviceToHost, st));
  if (adaptive && nr->n_pairs)
    CK(cudaMemcpyAsync(adaptive, nr->pair_ad, nr->n_pairs, cudaMemcpyDeviceToHost, st));
  if (centroid)
    CK(cudaMemcpyAsync(centroid, nr->cen, nr->n_patches * 3 * 8, cudaMemcpyDeviceToHost, st));
  if (radius) CK(cudaMemcpyAsync(radius, nr->rad, nr->n_patches * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return LCQ_OK;
}

void lcq_near_destroy(lcq_near* nr) {
  if (!nr) return;
  cudaSetDevice(nr->device);
  cudaStream_t st = nr->stream;
  for (int d = 0; d <= kMaxDeg; ++d) {
    dfree(st, nr->plist_dev[d]);
    dfree(st, nr->ad_list_dev[d]);
  }
  dfree(st, nr->deg);
  dfree(st, nr->node_off);
  dfree(st, nr->coef);
  dfree(st, nr->cen);
  dfree(st, nr->rad);
  dfree(st, nr->dj);
  dfree(st, nr->eta);
  dfree(st, nr->eta1);
  dfree(st, nr->tgt);
  dfree(st, nr->tnode);
  dfree(st, nr->tgt_patch);
  dfree(st, nr->tgt_lnode);
  dfree(st, nr->pgroup);
  dfree(st, nr->tgroup);
  dfree(st, nr->unrm);
  dfree(st, nr->tnrm);
  dfree(st, nr->row_ptr);
  dfree(st, nr->rowp_ptr);
  dfree(st, nr->rowp_patch);
  dfree(st, nr->rowp_off);
  dfree(st, nr->col);
  dfree(st, nr->pair_ptr);
  dfree(st, nr->pair_tgt);
  dfree(st, nr->pair_ad);
  dfree(st, nr->pair_d2);
  dfree(st, nr->pair_csr);
  dfree(st, nr->ad_ptr);
  dfree(st, nr->ad_pair);
  dfree(st, nr->an_ptr);
  dfree(st, nr->an_pair);
  dfree(st, nr->self_tgt);
  dfree(st, nr->self_csr);
  dfree(st, nr->self_ptr);
  cudaGetLastError();
  delete nr;
}

// ---------------------------------------------------------------------------- corrections
static Dev make_dev(lcq_ctx* ctx, const lcq_near* nr, const int32_t* q, int ldI,
                    const GroupParams* grp) {
  Dev dv{};
  dv.pgroup = grp ? nr->pgroup : nullptr;
  dv.grp = grp;
  dv.tnrm = nr->tnrm;
  dv.coef = nr->coef;
  dv.node_off = nr->node_off;
  dv.cen = nr->cen;
  dv.rad = nr->rad;
  dv.dj = nr->dj;
  dv.eta = nr->eta;
  dv.eta1 = nr->eta1;
  dv.tgt = nr->tgt;
  dv.NT = nr->n_targets;
  dv.tpatch = nr->tgt_patch;
  dv.tlnode = nr->tgt_lnode;
  dv.pair_ptr = nr->pair_ptr;
  dv.pair_tgt = nr->pair_tgt;
  dv.pair_d2 = nr->pair_d2;
  dv.pair_csr = nr->pair_csr;
  dv.ad_ptr = nr->ad_ptr;
  dv.ad_pair = nr->ad_pair;
  dv.an_ptr = nr->an_ptr;
  dv.an_pair = nr->an_pair;
  dv.self_ptr = nr->self_ptr;
  dv.self_tgt = nr->self_tgt;
  dv.self_csr = nr->self_csr;
  dv.n_self = nr->n_self;
  dv.q = q;
  dv.roff = ctx->rules.doff;
  dv.ru = ctx->rules.du;
  dv.rv = ctx->rules.dv;
  dv.rw = ctx->rules.dw;
  dv.gl_off = ctx->rules.dgl_off;
  dv.gl_x = ctx->rules.dgl_x;
  dv.gl_w = ctx->rules.dgl_w;
  for (int d = 0; d <= kMaxDeg; ++d) {
    dv.nodes_uv[d] = ctx->deg[d].dnodes;
    dv.duv[d] = ctx->deg[d].dDuv;
  }
  dv.counters = ctx->d_counters;
  dv.status = ctx->d_status;
  dv.ldI = ldI;
  return dv;
}

// Per-block workspace of the adaptive kernel (sized by the largest work item and the depth
// cap) and its grid.
static void adaptive_stride(lcq_ctx* ctx, const lcq_near* nr, int64_t A, int levels,
                            int64_t* stride_out, int* grid_out) {
  const int64_t n = nr->n_max;
  int64_t stride = A * n * 16 + A * 4 * n * 16 + (int64_t)levels * A * 4 * n * 16 +
                   (int64_t)levels * A * 4 + 2 * A * 4 + (int64_t)levels * 4 + 8 + A * 4 * 8 + 256;
  *stride_out = (stride + 255) / 256 * 256;
  int bps = 1;
  for (int d = 1; d <= kMaxDeg; ++d)
    if (nr->ad_count[d]) bps = std::max(bps, adaptive_blocks_per_sm(d));
  *grid_out = ctx->num_sms * bps;
}
// The same in the context's workspace, grown when needed.
static cudaError_t adaptive_work(lcq_ctx* ctx, const lcq_near* nr, int64_t A, int levels,
                                 int64_t* stride_out, int* grid_out) {
  int64_t stride = 0;
  int agrid = 0;
  adaptive_stride(ctx, nr, A, levels, &stride, &agrid);
  const size_t need = (size_t)stride * agrid;
  if (ctx->work_bytes < need) {
    if (ctx->work) {
      cudaError_t e = cudaFreeAsync(ctx->work, ctx->stream);
      if (e != cudaSuccess) return e;
    }
    ctx->work = nullptr;
    ctx->work_bytes = 0;
    cudaError_t e = cudaMallocAsync(&ctx->work, need, ctx->stream);
    if (e != cudaSuccess) return e;
    ctx->work_bytes = need;
  }
  *stride_out = stride;
  *grid_out = agrid;
  return cudaSuccess;
}

// ---------------------------------------------------------------------------- tuner
// Form of the pair evaluations in the moment kernels (pair_form): 0 FP64; for LCQ_MIXED
// 1 (FP32) for eps >= kMixedMinEps, 2 (two-float) for eps >= kTwoFloatMinEps, 0 below; 3 in
// a batch, where each surface's tolerance decides.  S' is always FP64.
static int pair_form_mode(lcq_precision precision, lcq_kernel kernel, const lcq_near* nr,
                          double eps0) {
  if (precision != LCQ_MIXED || kernel == LCQ_SP) return 0;
  if (nr->grouped) return 3;
  return eps0 >= kMixedMinEps ? 1 : (eps0 >= kTwoFloatMinEps ? 2 : 0);
}
// The forms a generation uses, as a bit mask (1: FP32, 2: two-float; 0: FP64 only); the
// two-float form needs a real k and a real alpha (the folded kernel constants).
static int forms_used(int mode, const KernelParams& kp, const std::vector<GroupParams>& grp) {
  auto one = [](int f, const KernelParams& p) {
    if (f == 1) return 1;
    if (f == 2 && p.ki == 0.0 && p.kind <= 2 && p.ai == 0.0) return 2;
    return 0;
  };
  if (mode != 3) return one(mode, kp);
  int m = 0;
  for (const GroupParams& g : grp)
    m |= one(g.eps >= kMixedMinEps ? 1 : (g.eps >= kTwoFloatMinEps ? 2 : 0), g.kp);
  return m;
}

// Tuner state of (degree, kernel, tolerance decade, precision, size class of the degree's
// adaptive work, batch or not), with its candidates on first use.
static lcq_tune& tune_state(lcq_ctx* ctx, const lcq_near* nr, int d, int kernel, double eps,
                            int form, int64_t slots) {
  const int dec = (int)std::floor(std::log10(eps)) + 40;
  int cls = 0;
  while ((int64_t(1) << cls) < nr->ad_total[d] + 1 && cls < 62) ++cls;
  const uint64_t key = (uint64_t)d | ((uint64_t)kernel << 4) | ((uint64_t)(dec & 63) << 8) |
                       ((uint64_t)cls << 15) | ((uint64_t)nr->grouped << 21) |
                       ((uint64_t)(nr->ad_max[d] > 16) << 22) | ((uint64_t)form << 23);
  lcq_tune& tu = ctx->tune[key];
  if (tu.cand.empty()) {
    std::vector<int> c;
    const int64_t amax = std::max<int64_t>(nr->ad_max[d], 1);
    c.push_back((int)std::min<int64_t>(amax, 0x7fffffff));  // whole patches
    // Splitting patches into groups only pays when whole patches leave slots idle or
    // unbalanced; with 16 or more whole patches per resident block (longest first) they do
    // neither, and timing the other candidates would cost whole generations.
    if ((int64_t)nr->ad_count[d] < 16 * slots) {
      for (int64_t ips : {1, 4, 16}) {
        const int64_t want = ips * slots;
        int64_t g = (nr->ad_total[d] + want - 1) / want;
        g = std::max<int64_t>(16, (g + 7) / 8 * 8);
        c.push_back((int)std::min<int64_t>(g, amax));
      }
      c.push_back((int)std::min<int64_t>(16, amax));
      // small adaptive work (fewer 16-target items than resident blocks): smaller groups
      // spread one patch's targets over more blocks, shortening the longest walk
      if ((nr->ad_total[d] + 15) / 16 < slots)
        for (int g : {8, 4, 2, 1}) c.push_back((int)std::min<int64_t>(g, amax));
    }
    std::sort(c.begin(), c.end(), std::greater<int>());
    c.erase(std::unique(c.begin(), c.end()), c.end());
    tu.cand = c;
    tu.ms_per.assign(c.size(), -1.0);
    cudaEventCreate(&tu.e0);
    cudaEventCreate(&tu.e1);
  }
  return tu;
}

// Collects a finished timing, then returns the candidate to use; *measure receives it when
// this launch is to be timed (else -1).
static int tune_pick(lcq_tune& tu, int* measure) {
  *measure = -1;
  if (tu.pending >= 0) {
    const cudaError_t q = cudaEventQuery(tu.e1);
    if (q == cudaSuccess) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, tu.e0, tu.e1) == cudaSuccess && tu.pend_pairs > 0.0) {
        const double v = ms / tu.pend_pairs;
        double& slot = tu.ms_per[tu.pending];
        slot = slot < 0.0 ? v : std::min(slot, v);
      }
      tu.pending = -1;
    } else if (q != cudaErrorNotReady) {
      cudaGetLastError();
      tu.pending = -1;
    }
  }
  int best = -1;
  for (size_t i = 0; i < tu.cand.size(); ++i) {
    if (tu.ms_per[i] < 0.0) {
      if (tu.pending < 0) {
        *measure = (int)i;
        return (int)i;
      }
      continue;
    }
    if (best < 0 || tu.ms_per[i] < tu.ms_per[best]) best = (int)i;
  }
  if (best >= 0) return best;
  return tu.pending >= 0 ? tu.pending : 0;
}

// The fastest candidate timed so far (the first when none is).
static int tune_best(const lcq_tune& tu) {
  int best = 0;
  for (size_t i = 0; i < tu.cand.size(); ++i)
    if (tu.ms_per[i] >= 0.0 && (tu.ms_per[best] < 0.0 || tu.ms_per[i] < tu.ms_per[best]))
      best = (int)i;
  return best;
}

// Work buffers and launch choices of one generation (gen_impl) or of a captured one
// (lcq_plan_create).
struct GenScratch {
  Dev dv{};
  double* ddirs = nullptr;
  int ndirs = 0;
  void *Is = nullptr, *In = nullptr, *InS = nullptr;
  double* fscr = nullptr;
  int fgrid = 0;
  int64_t *gng = nullptr, *gscr = nullptr, *ggofs[kMaxDeg + 1] = {nullptr};
  int gsz[kMaxDeg + 1] = {0};
  int tune_meas[kMaxDeg + 1] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
  lcq_tune* tune_st[kMaxDeg + 1] = {nullptr};
  int64_t A_eff = 0, astride = 0;
  int agrid = 0, levels = 0, sorder = 0, form = 0;
  void* work = nullptr;   // adaptive workspace (the context's, or the plan's own)
  bool own_work = false;
};

// A captured generation (lcq_plan_create): its own work buffers and the graph.
struct lcq_plan {
  lcq_ctx* ctx = nullptr;
  const lcq_near* near = nullptr;
  lcq_corr* corr = nullptr;
  lcq_params params{};
  GenScratch gs;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;   // kernel launches in the graph
};

// The far-order scratch, the work groups of the adaptive walk and the adaptive workspace.
// Group sizes: fixed_gsz where given, else the context's tuner (timing a candidate when
// `tune`, else each key's best so far).  With own_work the workspace belongs to gs alone.
static lcq_status gen_scratch(lcq_ctx* ctx, const lcq_near* nr, lcq_kernel kernel, double eps0,
                              const lcq_params* params, bool tune, GenScratch* gs,
                              const int* fixed_gsz = nullptr) {
  cudaStream_t st = ctx->stream;
  gs->fgrid = ctx->num_sms * 2;
  CK(dalloc(st, &gs->fscr, (size_t)gs->fgrid * 2 * kMaxTestPts * kMaxBasis * 2));
  gs->levels = params->max_depth;
  // Work groups of the adaptive walk: at most gsz[d] targets of one patch per item, chosen
  // per degree among candidates that give about 1, 4 or 16 items per resident block, 16
  // targets (fewer for small work) or whole patches; the grouping changes no result.
  ctx->last_group_size = 0;
  ctx->last_items = 0;
  if (nr->n_adaptive > 0) {
    int bps = 1;
    for (int d = 1; d <= kMaxDeg; ++d)
      if (nr->ad_count[d]) bps = std::max(bps, adaptive_blocks_per_sm(d));
    const int64_t slots = (int64_t)ctx->num_sms * bps;
    for (int d = 1; d <= kMaxDeg; ++d) {
      gs->tune_meas[d] = -1;
      if (!nr->ad_count[d]) continue;
      if (fixed_gsz && fixed_gsz[d] > 0) {
        gs->gsz[d] = fixed_gsz[d];
      } else {
        lcq_tune& tu = tune_state(ctx, nr, d, (int)kernel, eps0, gs->form, slots);
        gs->tune_st[d] = &tu;
        if (tune) {
          const int pick = tune_pick(tu, &gs->tune_meas[d]);
          gs->gsz[d] = tu.cand[pick];
        } else {
          gs->gsz[d] = tu.cand[tune_best(tu)];
        }
      }
      gs->A_eff = std::max<int64_t>(gs->A_eff, gs->gsz[d]);
      ctx->last_group_size = std::max(ctx->last_group_size, gs->gsz[d]);
      for (int64_t a : nr->ad_nad_h[d]) ctx->last_items += (a + gs->gsz[d] - 1) / gs->gsz[d];
    }
    if (gs->own_work) {
      adaptive_stride(ctx, nr, gs->A_eff, gs->levels, &gs->astride, &gs->agrid);
      CK(cudaMallocAsync(&gs->work, (size_t)gs->astride * gs->agrid, st));
    } else {
      CK(adaptive_work(ctx, nr, gs->A_eff, gs->levels, &gs->astride, &gs->agrid));
      gs->work = ctx->work;
    }
    int maxc = 0;
    for (int d = 1; d <= kMaxDeg; ++d) maxc = std::max(maxc, nr->ad_count[d]);
    CK(dalloc(st, &gs->gng, (size_t)maxc + 1));
    CK(dalloc(st, &gs->gscr, (size_t)2 * ((maxc + 1 + 1023) / 1024) + 64));
    for (int d = 1; d <= kMaxDeg; ++d)
      if (nr->ad_count[d]) CK(dalloc(st, &gs->ggofs[d], (size_t)nr->ad_count[d] + 1));
  }
  return LCQ_OK;
}

// Releases gs's buffers (stream-ordered).
static void gen_free(cudaStream_t st, GenScratch* gs) {
  if (gs->ddirs) dfree(st, gs->ddirs);
  if (gs->fscr) dfree(st, gs->fscr);
  if (gs->gng) dfree(st, gs->gng);
  if (gs->gscr) dfree(st, gs->gscr);
  for (int d = 1; d <= kMaxDeg; ++d)
    if (gs->ggofs[d]) dfree(st, gs->ggofs[d]);
  if (gs->Is) cudaFreeAsync(gs->Is, st);
  if (gs->In) cudaFreeAsync(gs->In, st);
  if (gs->InS) cudaFreeAsync(gs->InS, st);
  if (gs->own_work && gs->work) cudaFreeAsync(gs->work, st);
  *gs = GenScratch{};
}

// Stages 1-6 of a generation into c: launches, event records and stream waits only (no
// allocation and no host synchronization), so that the sequence can be captured into a
// CUDA graph.  `timed` adds the stage events and the tuner's timing events.
static lcq_status gen_launch(lcq_ctx* ctx, const lcq_near* nr, lcq_corr* c,
                             const lcq_params* params, const GenScratch& gs, bool timed) {
  cudaStream_t st = ctx->stream;
  const Dev& dv = gs.dv;
  const KernelParams& kp = c->kp;
  const double eps0 = c->eps0;
  CK(cudaMemsetAsync(c->leaves, 0, std::max<int64_t>(nr->n_pairs, 1) * 4, st));
  CK(cudaMemsetAsync(c->val, 0, std::max<int64_t>(nr->nnz, 1) * 16, st));
  CK(cudaMemsetAsync(ctx->d_counters, 0, 8 * sizeof(long long), st));
  // Stages 1-4 and 6 depend on one another and run on the highest-priority stream; the
  // self weights (5) depend on none of them and run on the lowest-priority one from the
  // start, so their blocks fill what the chain leaves idle (the small far-order and
  // smooth-rule launches, the end of the adaptive walk) without delaying it.
  CK(cudaEventRecord(ctx->fork, st));
  CK(cudaStreamWaitEvent(ctx->hi, ctx->fork, 0));
  CK(cudaStreamWaitEvent(ctx->side, ctx->fork, 0));
  LaunchCommon lh{ctx->hi, ctx->num_sms, &ctx->launches_corr};
  cudaStream_t sh = ctx->hi;
  if (timed) CK(cudaEventRecord(ctx->ev[2], sh));
  // 1. far order q_j and annulus order (Sec. 4.2, Eq. qj)
  for (int d = 1; d <= kMaxDeg; ++d) {
    if (!nr->plist_count[d]) continue;
    launch_farorder(d, lh, nr->plist_dev[d], nr->plist_count[d], dv, kp, eps0, params->m_max,
                    ctx->deg[d].normV, gs.ddirs, gs.ndirs, gs.fscr, gs.fgrid, c->q, c->q_near,
                    ctx->d_sched);
  }
  CK(cudaGetLastError());
  // 5. self weights (Sec. 4, Eq. errestself), on the low-priority stream
  if (timed) CK(cudaEventRecord(ctx->ev_self[0], ctx->side));
  if (nr->n_self > 0) {
    LaunchCommon ls{ctx->side, ctx->num_sms, &ctx->launches_corr};
    for (int d = 1; d <= kMaxDeg; ++d) {
      if (!nr->plist_count[d]) continue;
      launch_self(d, ls, dv, nr->deg, kp, gs.sorder, gs.InS);
    }
  }
  CK(cudaGetLastError());
  if (timed) CK(cudaEventRecord(ctx->ev_self[1], ctx->side));
  CK(cudaEventRecord(ctx->join, ctx->side));
  if (timed) CK(cudaEventRecord(ctx->ev[3], sh));
  // 2. smooth-rule moments of every near and self pair; 3. annulus moments
  for (int d = 1; d <= kMaxDeg; ++d) {
    if (!nr->plist_count[d]) continue;
    launch_rule_moments(d, lh, nr->plist_dev[d], nr->plist_count[d], dv, 3, c->q, c->q_near, kp,
                        gs.Is, gs.In, gs.form);
  }
  CK(cudaGetLastError());
  if (timed) CK(cudaEventRecord(ctx->ev[4], sh));
  // 4. adaptive near moments (Sec. 4.3)
  if (nr->n_adaptive > 0) {
    for (int d = 1; d <= kMaxDeg; ++d) {
      if (!nr->ad_count[d]) continue;
      const int cnt = nr->ad_count[d];
      lcq_tune* tu = gs.tune_st[d];
      const bool meas = timed && tu && gs.tune_meas[d] >= 0;
      if (meas) CK(cudaEventRecord(tu->e0, sh));
      launch_group_offsets(lh, nr->ad_list_dev[d], cnt, nr->ad_ptr, gs.gsz[d], gs.gng,
                           gs.ggofs[d], gs.gscr);
      launch_adaptive(d, lh, nr->ad_list_dev[d], cnt, dv, kp, eps0 * params->eps_loosen,
                      ctx->deg[d].normV, params->leaf_order, params->max_depth, gs.Is, gs.In,
                      c->leaves, gs.work, gs.astride, (int)gs.A_eff, gs.levels, gs.agrid,
                      ctx->d_status, ctx->d_sched + d, gs.form, gs.ggofs[d], gs.gsz[d]);
      if (meas) {
        CK(cudaEventRecord(tu->e1, sh));
        tu->pending = gs.tune_meas[d];
        tu->pend_pairs = (double)nr->ad_total[d];
      }
    }
    CK(cudaGetLastError());
  }
  if (timed) CK(cudaEventRecord(ctx->ev[5], sh));
  CK(cudaStreamWaitEvent(sh, ctx->join, 0));  // self weights done
  if (timed) CK(cudaEventRecord(ctx->ev[6], sh));
  // 6. c = V^T (I_near - I_smooth) into the CSR
  for (int d = 1; d <= kMaxDeg; ++d) {
    if (!nr->plist_count[d]) continue;
    launch_v2c(d, lh, nr->plist_dev[d], nr->plist_count[d], dv, ctx->deg[d].dV, gs.In, gs.Is,
               gs.InS, c->val);
  }
  CK(cudaGetLastError());
  if (timed) CK(cudaEventRecord(ctx->ev[7], sh));
  CK(cudaEventRecord(ctx->done, sh));
  CK(cudaStreamWaitEvent(st, ctx->done, 0));
  return LCQ_OK;
}

static lcq_status gen_impl(lcq_ctx* ctx, const lcq_near* nr, lcq_kernel kernel, int n_phys,
                           const lcq_surface_physics* phys, lcq_precision precision,
                           const lcq_params* params, lcq_corr** out) {
  if (!ctx || !nr || !params || !out || !phys) return fail(ctx, LCQ_ERR_ARG, "null argument");
  *out = nullptr;
  if (precision != LCQ_FP64 && precision != LCQ_MIXED)
    return fail(ctx, LCQ_ERR_ARG, "unsupported precision");
  if ((int)kernel < 0 || (int)kernel > 3) return fail(ctx, LCQ_ERR_ARG, "unknown kernel");
  if (kernel == LCQ_SP && nr->n_targets > nr->n_self && !nr->unrm)
    return fail(ctx, LCQ_ERR_ARG, "S' needs the normals of off-surface targets "
                                  "(lcq_near_set_target_normals)");
  if (n_phys != nr->n_groups)
    return fail(ctx, LCQ_ERR_ARG, "one physics record per surface of the near lists");
  for (int g = 0; g < n_phys; ++g) {
    const lcq_surface_physics& f = phys[g];
    if (!(f.eps > 0.0) || f.k_im < 0.0 || !isfinite(f.k_re) || !isfinite(f.k_im) ||
        !isfinite(f.alpha_re) || !isfinite(f.alpha_im) || !isfinite(f.beta_re) ||
        !isfinite(f.beta_im))
      return fail(ctx, LCQ_ERR_ARG, "eps must be > 0, Im k >= 0 and coefficients finite");
  }
  const double k_re = phys[0].k_re, k_im = phys[0].k_im;
  const double alpha_re = phys[0].alpha_re, alpha_im = phys[0].alpha_im;
  const double beta_re = phys[0].beta_re, beta_im = phys[0].beta_im;
  const double eps0 = phys[0].eps;
  if (params->m_max < 2 || params->m_max > kMaxRule || params->leaf_order < 0 ||
      params->leaf_order > kMaxRule || params->self_order < 0 || params->self_order > kMaxGL ||
      params->max_depth < 1 || params->max_depth > 24 || params->n_test_dirs < 0 ||
      params->n_test_dirs > kMaxTestPts - 10)
    return fail(ctx, LCQ_ERR_ARG, "parameter out of range");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  ctx->launches_corr = 0;
  LaunchCommon lc{st, ctx->num_sms, &ctx->launches_corr};
  const int64_t P = nr->n_patches;
  const KernelParams kp =
      make_kernel_params((int)kernel, k_re, k_im, alpha_re, alpha_im, beta_re, beta_im);

  lcq_corr* c = new lcq_corr();
  c->near = nr;
  c->stream = st;
  c->device = ctx->device;
  c->kernel = (int)kernel;
  c->n_patches = P;
  c->n_targets = nr->n_targets;
  c->nnz = nr->nnz;
  c->n_pairs = nr->n_pairs;
  c->n_self = nr->n_self;
  c->kp = kp;
  c->params = *params;
  c->params.test_dirs = nullptr;
  c->params.n_test_dirs = 0;
  c->eps0 = eps0;
  c->precision = (int)precision;
  auto undo = on_exit([&] { lcq_corr_destroy(c); });
  // the generation's work buffers; gen_free releases them on every return
  GenScratch gs;
  auto gs_free = on_exit([&] { gen_free(st, &gs); });
  CK(dalloc(st, &c->val, (size_t)2 * std::max<int64_t>(nr->nnz, 1)));
  CK(dalloc(st, &c->q, P));
  CK(dalloc(st, &c->q_near, P));
  CK(dalloc(st, &c->leaves, nr->n_pairs));

  // test directions
  std::vector<double> dirs;
  if (params->test_dirs && params->n_test_dirs > 0) {
    dirs.assign(params->test_dirs, params->test_dirs + 3 * params->n_test_dirs);
  } else {
    const int nd = 15;
    for (int k = 0; k < nd; ++k) {
      const double z = 1.0 - (2.0 * k + 1.0) / nd, r = sqrt(1.0 - z * z);
      const double phi = k * M_PI * (3.0 - sqrt(5.0));
      dirs.push_back(r * cos(phi));
      dirs.push_back(r * sin(phi));
      dirs.push_back(z);
    }
  }
  gs.ndirs = (int)dirs.size() / 3;
  CK(dalloc(st, &gs.ddirs, dirs.size()));
  CK(cudaMemcpyAsync(gs.ddirs, dirs.data(), dirs.size() * 8, cudaMemcpyHostToDevice, st));

  const int ldI = nr->n_max;
  const int64_t npr = std::max<int64_t>(nr->n_pairs, 1), nsf = std::max<int64_t>(nr->n_self, 1);
  CK(dalloc(st, reinterpret_cast<double**>(&gs.Is), (size_t)2 * npr * ldI));
  CK(dalloc(st, reinterpret_cast<double**>(&gs.In), (size_t)2 * npr * ldI));
  CK(dalloc(st, reinterpret_cast<double**>(&gs.InS), (size_t)2 * nsf * ldI));
  if (nr->grouped) {
    std::vector<GroupParams> gp(n_phys);
    for (int g = 0; g < n_phys; ++g) {
      const lcq_surface_physics& f = phys[g];
      gp[g].kp = make_kernel_params((int)kernel, f.k_re, f.k_im, f.alpha_re, f.alpha_im, f.beta_re,
                                    f.beta_im);
      gp[g].eps = f.eps;
      gp[g].eps_ad = f.eps * params->eps_loosen;
      gp[g].self_order = params->self_order > 0 ? params->self_order : default_self_order(f.eps);
    }
    CK(dalloc(st, &c->grp, gp.size()));
    CK(cudaMemcpyAsync(c->grp, gp.data(), gp.size() * sizeof(GroupParams), cudaMemcpyHostToDevice,
                       st));
    c->grp_h = gp;
  }
  if (kernel == LCQ_SP && !nr->tnrm && nr->n_targets > 0) {
    lcq_near* nw = const_cast<lcq_near*>(nr);
    CK(dalloc(st, &nw->tnrm, (size_t)3 * nr->n_targets));
    Dev d0 = make_dev(ctx, nr, c->q, ldI, c->grp);
    bool first = true;
    for (int d = 1; d <= kMaxDeg; ++d) {
      if (!nr->plist_count[d]) continue;
      launch_tgt_normals(d, lc, d0, nr->deg, nr->unrm, first && nr->unrm, nw->tnrm);
      first = false;
    }
  }
  Dev dv = make_dev(ctx, nr, c->q, ldI, c->grp);

  // the mixed form (FP32 or two-float pair evaluation in the smooth, annulus and adaptive
  // moments); per surface of a batch the kernels choose by the surface's tolerance
  const int form = pair_form_mode(precision, kernel, nr, eps0);
  c->form = form;
  ctx->last_forms = forms_used(form, c->kp, c->grp_h);
  gs.dv = dv;
  gs.form = form;
  gs.sorder = params->self_order > 0 ? params->self_order : default_self_order(eps0);
  lcq_status ls = gen_scratch(ctx, nr, kernel, eps0, params, true, &gs);
  if (ls == LCQ_OK) ls = gen_launch(ctx, nr, c, params, gs, true);
  if (ls != LCQ_OK) return ls;
  for (int d = 0; d <= kMaxDeg; ++d) c->gsz[d] = gs.gsz[d];
  gen_free(st, &gs);
  // stash the stream/device for later calls on the correction object
  c->q_h.clear();
  c->src_off = nullptr;
  c->dirs_h = dirs;
  undo.dismiss();
  *out = c;
  return LCQ_OK;
}

lcq_status lcq_gen_corrections(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* nr,
                               lcq_kernel kernel, double k_re, double k_im, double alpha_re,
                               double alpha_im, double beta_re, double beta_im,
                               lcq_precision precision, const lcq_params* params, lcq_corr** out) {
  (void)surf;
  if (!params) return fail(ctx, LCQ_ERR_ARG, "null argument");
  if (nr && nr->grouped)
    return fail(ctx, LCQ_ERR_ARG, "near lists of a batch: use lcq_gen_corrections_batched");
  const lcq_surface_physics f{k_re, k_im, alpha_re, alpha_im, beta_re, beta_im, params->eps};
  return gen_impl(ctx, nr, kernel, 1, &f, precision, params, out);
}

lcq_status lcq_gen_corrections_batched(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* nr,
                                       lcq_kernel kernel, int n_surfaces,
                                       const lcq_surface_physics* physics, lcq_precision precision,
                                       const lcq_params* params, lcq_corr** out) {
  (void)surf;
  if (nr && !nr->grouped)
    return fail(ctx, LCQ_ERR_ARG, "near lists were not built by lcq_build_near_lists_batched");
  return gen_impl(ctx, nr, kernel, n_surfaces, physics, precision, params, out);
}

static lcq_status ensure_q_host(lcq_ctx* ctx, lcq_corr* c) {
  if (!c->q_h.empty()) return LCQ_OK;
  CK(cudaSetDevice(c->device));
  c->q_h.resize(c->n_patches);
  CK(cudaMemcpyAsync(c->q_h.data(), c->q, c->n_patches * 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  int64_t acc = 0;
  std::vector<int64_t> off(c->n_patches + 1);
  for (int64_t j = 0; j < c->n_patches; ++j) {
    off[j] = acc;
    acc += (int64_t)c->q_h[j] * c->q_h[j];
  }
  off[c->n_patches] = acc;
  c->n_over = acc;
  CK(dalloc(c->stream, &c->src_off, c->n_patches + 1));
  CK(cudaMemcpyAsync(c->src_off, off.data(), (c->n_patches + 1) * 8, cudaMemcpyHostToDevice,
                     c->stream));
  if (c->grp) {
    const lcq_near* nr = c->near;
    c->gsrc_h.resize(nr->n_groups + 1);
    for (int g = 0; g <= nr->n_groups; ++g) c->gsrc_h[g] = off[nr->gpatch_off[g]];
    CK(dalloc(c->stream, &c->gsrc, c->gsrc_h.size()));
    CK(cudaMemcpyAsync(c->gsrc, c->gsrc_h.data(), c->gsrc_h.size() * 8, cudaMemcpyHostToDevice,
                       c->stream));
  }
  return LCQ_OK;
}

lcq_status lcq_corr_info(const lcq_corr* c, int64_t* nnz, int64_t* n_over, int* value_dtype) {
  if (!c) return LCQ_ERR_ARG;
  lcq_status s = ensure_q_host(nullptr, const_cast<lcq_corr*>(c));
  if (s != LCQ_OK) return s;
  if (nnz) *nnz = c->nnz;
  if (n_over) *n_over = c->n_over;
  if (value_dtype) *value_dtype = 0;
  return LCQ_OK;
}

lcq_status lcq_corr_export(lcq_corr* c, int64_t* row_ptr, int32_t* col, double* val) {
  if (!c || !c->near) return LCQ_ERR_ARG;
  lcq_ctx* ctx = nullptr;
  CK(cudaSetDevice(c->device));
  const lcq_near* nr = c->near;
  cudaStream_t st = c->stream;
  // cudaMemcpyDefault: the destinations may be host or device memory (unified addressing)
  if (row_ptr)
    CK(cudaMemcpyAsync(row_ptr, nr->row_ptr, (nr->n_targets + 1) * 8, cudaMemcpyDefault, st));
  if (col && c->nnz) CK(cudaMemcpyAsync(col, nr->col, c->nnz * 4, cudaMemcpyDefault, st));
  if (val && c->nnz) CK(cudaMemcpyAsync(val, c->val, c->nnz * 16, cudaMemcpyDefault, st));
  CK(cudaStreamSynchronize(st));
  return LCQ_OK;
}

lcq_status lcq_corr_export_stats(lcq_corr* c, int32_t* q, int32_t* q_near, int32_t* leaves) {
  if (!c) return LCQ_ERR_ARG;
  lcq_ctx* ctx = nullptr;
  CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  if (q) CK(cudaMemcpyAsync(q, c->q, c->n_patches * 4, cudaMemcpyDeviceToHost, st));
  if (q_near) CK(cudaMemcpyAsync(q_near, c->q_near, c->n_patches * 4, cudaMemcpyDeviceToHost, st));
  if (leaves && c->n_pairs)
    CK(cudaMemcpyAsync(leaves, c->leaves, c->n_pairs * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return LCQ_OK;
}

static lcq_status apply_impl(lcq_ctx* ctx, const lcq_near* nr, const lcq_corr* cc,
                             const double* sigma, double jump, double* out, int kind) {
  if (!ctx || !nr || !cc || !sigma || !out) return fail(ctx, LCQ_ERR_ARG, "null argument");
  if (cc->kernel != kind) return fail(ctx, LCQ_ERR_ARG, "kernel differs from the corrections'");
  if (cc->near != nr) return fail(ctx, LCQ_ERR_ARG, "corrections belong to another near list");
  lcq_corr* c = const_cast<lcq_corr*>(cc);
  CK(cudaSetDevice(ctx->device));
  lcq_status s = ensure_q_host(ctx, c);
  if (s != LCQ_OK) return s;
  cudaStream_t st = ctx->stream;
  long long napply = 0;
  LaunchCommon lc{st, ctx->num_sms, &napply};
  Dev dv = make_dev(ctx, nr, c->q, nr->n_max, c->grp);
  // the kernel constants fold into the sources when every surface has a real k and a real
  // alpha (kinds S, D, CFIE)
  auto foldable = [](const KernelParams& p) {
    return p.ki == 0.0 && p.kind <= 2 && p.ai == 0.0;
  };
  bool fold = foldable(c->kp);
  for (const GroupParams& g : c->grp_h) fold = fold && foldable(g.kp);
  double* src = nullptr;
  auto src_free = on_exit([&] { dfree(st, src); });
  CK(dalloc(st, &src, (size_t)(fold ? 10 : 9) * std::max<int64_t>(c->n_over, 1)));
  for (int d = 1; d <= kMaxDeg; ++d) {
    if (!nr->plist_count[d]) continue;
    launch_far_src(d, lc, nr->plist_dev[d], nr->plist_count[d], dv, ctx->deg[d].dV, c->q,
                   c->src_off, sigma, src, c->n_over, c->kp, fold);
  }
  launch_far_sum(lc, nr->tgt, nr->n_targets, src, c->n_over, c->kp, nr->tgt_patch, c->src_off,
                 c->grp ? nr->tgroup : nullptr, c->grp, c->gsrc,
                 kind == LCQ_SP ? nr->tnrm : nullptr, out, fold);
  launch_csr_apply(lc, nr->row_ptr, nr->col, c->val, sigma, nr->tnode, nr->n_targets, jump, out);
  CK(cudaGetLastError());
  return LCQ_OK;
}

lcq_status lcq_apply_corrected_S(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                                 const lcq_corr* corr, const double* sigma, double jump,
                                 double* out) {
  (void)surf;
  return apply_impl(ctx, near, corr, sigma, jump, out, LCQ_S);
}
lcq_status lcq_apply_corrected_D(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                                 const lcq_corr* corr, const double* sigma, double jump,
                                 double* out) {
  (void)surf;
  return apply_impl(ctx, near, corr, sigma, jump, out, LCQ_D);
}
lcq_status lcq_apply_corrected_CFIE(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                                    const lcq_corr* corr, const double* sigma, double jump,
                                    double* out) {
  (void)surf;
  return apply_impl(ctx, near, corr, sigma, jump, out, LCQ_CFIE);
}
lcq_status lcq_apply_corrected(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                               const lcq_corr* corr, lcq_kernel kernel, const void* sigma,
                               int sigma_dtype, double jump, double* out) {
  (void)surf;
  if (sigma_dtype == 0)
    return apply_impl(ctx, near, corr, static_cast<const double*>(sigma), jump, out, kernel);
  if (sigma_dtype != 1 || !ctx || !near || !sigma) return fail(ctx, LCQ_ERR_ARG, "sigma dtype");
  CK(cudaSetDevice(ctx->device));
  double* wide;
  CK(dalloc(ctx->stream, &wide, (size_t)2 * std::max<int64_t>(near->n_points, 1)));
  long long nl = 0;
  LaunchCommon lc{ctx->stream, ctx->num_sms, &nl};
  launch_widen_c64(lc, sigma, near->n_points, wide);
  const lcq_status s = apply_impl(ctx, near, corr, wide, jump, out, kernel);
  dfree(ctx->stream, wide);
  return s;
}

lcq_status lcq_apply_corrected_Sp(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* near,
                                  const lcq_corr* corr, const double* sigma, double jump,
                                  double* out) {
  (void)surf;
  return apply_impl(ctx, near, corr, sigma, jump, out, LCQ_SP);
}

// Oversampled far sources of every patch (positions, weighted normals, J w, interpolated
// density if sigma is given) into a new buffer [9][n_over].
static lcq_status far_sources(lcq_ctx* ctx, const lcq_near* nr, lcq_corr* c, const Dev& dv,
                              const LaunchCommon& lc, const double* sigma, double** src_out) {
  double* src;
  CK(dalloc(ctx->stream, &src, (size_t)9 * std::max<int64_t>(c->n_over, 1)));
  for (int d = 1; d <= kMaxDeg; ++d) {
    if (!nr->plist_count[d]) continue;
    launch_far_src(d, lc, nr->plist_dev[d], nr->plist_count[d], dv, ctx->deg[d].dV, c->q,
                   c->src_off, sigma, src, c->n_over);
  }
  *src_out = src;
  return LCQ_OK;
}

lcq_status lcq_apply_adjoint(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* nr,
                             const lcq_corr* cc, const double* g, double jump, double* out) {
  (void)surf;
  if (!ctx || !nr || !cc || !g || !out) return fail(ctx, LCQ_ERR_ARG, "null argument");
  if (cc->near != nr) return fail(ctx, LCQ_ERR_ARG, "corrections belong to another near list");
  lcq_corr* c = const_cast<lcq_corr*>(cc);
  CK(cudaSetDevice(ctx->device));
  lcq_status s = ensure_q_host(ctx, c);
  if (s != LCQ_OK) return s;
  cudaStream_t st = ctx->stream;
  long long nl = 0;
  LaunchCommon lc{st, ctx->num_sms, &nl};
  Dev dv = make_dev(ctx, nr, c->q, nr->n_max, c->grp);
  double *src = nullptr, *z = nullptr;
  auto tmp_free = on_exit([&] {
    dfree(st, src);
    dfree(st, z);
  });
  s = far_sources(ctx, nr, c, dv, lc, nullptr, &src);
  if (s != LCQ_OK) return s;
  CK(dalloc(st, &z, (size_t)2 * std::max<int64_t>(c->n_over, 1)));
  launch_far_sum_T(lc, dv, nr->n_patches, src, c->n_over, c->src_off, c->kp,
                   c->grp ? nr->tgroup : nullptr, g, z);
  for (int d = 1; d <= kMaxDeg; ++d) {
    if (!nr->plist_count[d]) continue;
    launch_adj_patch(d, lc, nr->plist_dev[d], nr->plist_count[d], dv, ctx->deg[d].dV, c->src_off, z,
                     c->val, g, jump, out);
  }
  CK(cudaGetLastError());
  return LCQ_OK;
}

lcq_status lcq_shape_gradient(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* nr,
                              const lcq_corr* cc, const double* sigma, const double* g,
                              double* out) {
  (void)surf;
  if (!ctx || !nr || !cc || !sigma || !g || !out) return fail(ctx, LCQ_ERR_ARG, "null argument");
  if (cc->near != nr) return fail(ctx, LCQ_ERR_ARG, "corrections belong to another near list");
  if (nr->n_self > 0)
    return fail(ctx, LCQ_ERR_ARG, "shape gradient: off-surface targets only (no self pairs)");
  if (cc->kernel == LCQ_SP)
    return fail(ctx, LCQ_ERR_ARG, "shape gradient: S, D or CFIE only");
  lcq_corr* c = const_cast<lcq_corr*>(cc);
  CK(cudaSetDevice(ctx->device));
  lcq_status s = ensure_q_host(ctx, c);
  if (s != LCQ_OK) return s;
  cudaStream_t st = ctx->stream;
  long long nl = 0;
  LaunchCommon lc{st, ctx->num_sms, &nl};
  const int ldI = nr->n_max;
  Dev dv = make_dev(ctx, nr, c->q, ldI, c->grp);
  const int64_t N = nr->n_points, P = nr->n_patches;
  double *shat = nullptr, *M = nullptr, *tg = nullptr, *src = nullptr, *Is = nullptr,
         *In = nullptr;
  int32_t* leaves = nullptr;
  auto tmp_free = on_exit([&] {
    dfree(st, shat);
    dfree(st, M);
    dfree(st, tg);
    dfree(st, src);
    dfree(st, Is);
    dfree(st, In);
    dfree(st, leaves);
  });
  CK(dalloc(st, &shat, (size_t)2 * N));
  CK(dalloc(st, &M, (size_t)3 * N));
  CK(dalloc(st, &tg, (size_t)12 * std::max<int64_t>(c->n_over, 1)));
  for (int d = 1; d <= kMaxDeg; ++d) {
    if (!nr->plist_count[d]) continue;
    launch_shat(d, lc, nr->plist_dev[d], nr->plist_count[d], nr->node_off, ctx->deg[d].dV, sigma,
                shat);
  }
  s = far_sources(ctx, nr, c, dv, lc, nullptr, &src);
  if (s != LCQ_OK) return s;
  // 1. far pairs through the rules q_j; 2. annulus pairs (both write M)
  launch_far_grad_sum(lc, dv, P, src, c->n_over, c->src_off, c->kp, c->grp ? nr->tgroup : nullptr,
                      g, tg);
  for (int d = 1; d <= kMaxDeg; ++d) {
    if (!nr->plist_count[d]) continue;
    launch_grad_rules(d, lc, nr->plist_dev[d], nr->plist_count[d], dv, c->kp, c->q_near,
                      c->src_off, c->n_over, tg, g, shat, M);
  }
  // 3. adaptive pairs: the union-tree kernel again, in gradient mode (adds to M)
  if (nr->n_adaptive > 0) {
    const lcq_params& pr = c->params;
    const int levels = pr.max_depth;
    int64_t stride;
    int agrid;
    CK(adaptive_work(ctx, nr, nr->max_adaptive, levels, &stride, &agrid));
    const int64_t npr = std::max<int64_t>(nr->n_pairs, 1);
    CK(dalloc(st, &Is, (size_t)2 * npr * ldI));
    CK(dalloc(st, &In, (size_t)2 * npr * ldI));
    CK(dalloc(st, &leaves, npr));
    if (pr.leaf_order <= 0)  // root moments of the adaptive pairs: the smooth rule q_j
      for (int d = 1; d <= kMaxDeg; ++d) {
        if (!nr->plist_count[d]) continue;
        launch_rule_moments(d, lc, nr->plist_dev[d], nr->plist_count[d], dv, 1, c->q, nullptr,
                            c->kp, Is, nullptr, c->form);
      }
    const GradArgs ga{g, shat, M};
    for (int d = 1; d <= kMaxDeg; ++d) {
      if (!nr->ad_count[d]) continue;
      launch_adaptive_grad(d, lc, nr->ad_list_dev[d], nr->ad_count[d], dv, c->kp,
                           c->eps0 * pr.eps_loosen, ctx->deg[d].normV, pr.leaf_order, pr.max_depth,
                           Is, In, leaves, ctx->work, stride, (int)nr->max_adaptive, levels, agrid,
                           ctx->d_status, ctx->d_sched + d,
                           c->form, ga);
    }
  }
  // 4. dL/dy = V^T M per patch
  for (int d = 1; d <= kMaxDeg; ++d) {
    if (!nr->plist_count[d]) continue;
    launch_grad_v2c(d, lc, nr->plist_dev[d], nr->plist_count[d], nr->node_off, ctx->deg[d].dV, M,
                    N, out);
  }
  CK(cudaGetLastError());
  return LCQ_OK;
}

// ---------------------------------------------------------------------------- plans
// The apply path's cached oversampling offsets follow q_j, which a plan launch recomputes.
static void corr_forget_q(lcq_corr* c) {
  c->q_h.clear();
  if (c->src_off) dfree(c->stream, c->src_off);
  if (c->gsrc) dfree(c->stream, c->gsrc);
  c->src_off = nullptr;
  c->gsrc = nullptr;
  c->gsrc_h.clear();
  c->n_over = 0;
}

lcq_status lcq_plan_create(lcq_ctx* ctx, const lcq_surface* surf, const lcq_near* nr,
                           lcq_corr* c, lcq_plan** out) {
  if (!ctx || !surf || !nr || !c || !out) return fail(ctx, LCQ_ERR_ARG, "null argument");
  *out = nullptr;
  if (c->near != nr || surf->n_patches != nr->n_patches || !surf->xyz)
    return fail(ctx, LCQ_ERR_ARG, "the corrections must come from these near lists and surface");
  if (c->device != ctx->device) return fail(ctx, LCQ_ERR_ARG, "corrections of another device");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  lcq_plan* p = new lcq_plan();
  p->ctx = ctx;
  p->near = nr;
  p->corr = c;
  p->params = c->params;
  GenScratch& gs = p->gs;
  const int ldI = nr->n_max;
  const int64_t npr = std::max<int64_t>(nr->n_pairs, 1), nsf = std::max<int64_t>(nr->n_self, 1);
  gs.dv = make_dev(ctx, nr, c->q, ldI, c->grp);
  gs.ndirs = (int)c->dirs_h.size() / 3;
  gs.form = c->form;
  gs.sorder = c->params.self_order > 0 ? c->params.self_order : default_self_order(c->eps0);
  gs.own_work = true;
  lcq_status ls = LCQ_OK;
  auto ck = [&](cudaError_t e, const char* what) {
    if (ls == LCQ_OK && e != cudaSuccess) ls = cuda_fail(ctx, e, what);
  };
  ck(dalloc(st, &gs.ddirs, std::max<size_t>(c->dirs_h.size(), 1)), "plan directions");
  if (ls == LCQ_OK && !c->dirs_h.empty())
    ck(cudaMemcpyAsync(gs.ddirs, c->dirs_h.data(), c->dirs_h.size() * 8, cudaMemcpyHostToDevice,
                       st), "plan directions");
  ck(dalloc(st, reinterpret_cast<double**>(&gs.Is), (size_t)2 * npr * ldI), "plan moments");
  ck(dalloc(st, reinterpret_cast<double**>(&gs.In), (size_t)2 * npr * ldI), "plan moments");
  ck(dalloc(st, reinterpret_cast<double**>(&gs.InS), (size_t)2 * nsf * ldI), "plan moments");
  if (ls == LCQ_OK)
    ls = gen_scratch(ctx, nr, (lcq_kernel)c->kernel, c->eps0, &p->params, false, &gs, c->gsz);
  ck(cudaStreamSynchronize(st), "plan set-up");
  // The context's stream may be the legacy default stream, which cannot be captured: the
  // sequence is captured on a private stream standing in for it (the graph is launched on
  // the context's stream).
  cudaStream_t cs = nullptr;
  const cudaStream_t saved = ctx->stream;
  ck(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
  if (ls == LCQ_OK) {
    // capture: the on-surface targets and the geometry of the current node coordinates
    // (and, for S', the target normals), then stages 1-6 into c
    ctx->launches_corr = 0;
    ctx->stream = cs;
    st = cs;
    ck(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed), "begin capture");
    if (ls == LCQ_OK) {
      long long launches = 0;
      LaunchCommon lc{st, ctx->num_sms, &launches};
      launch_tgt_from_nodes(lc, nr->tgt, nr->tnode, nr->n_targets, surf->xyz, nr->n_points);
      for (int d = 1; d <= kMaxDeg; ++d) {
        if (!nr->plist_count[d]) continue;
        launch_geom(d, lc, nr->plist_dev[d], nr->plist_count[d], nr->node_off, surf->xyz,
                    nr->n_points, ctx->deg[d].dV, ctx->deg[d].dnodes, nr->params.eta,
                    nr->params.eta1, nr->coef, nr->cen, nr->rad, nr->dj, nr->eta, nr->eta1,
                    ctx->d_status);
      }
      if (c->kernel == LCQ_SP && nr->tnrm) {
        bool first = true;
        for (int d = 1; d <= kMaxDeg; ++d) {
          if (!nr->plist_count[d]) continue;
          launch_tgt_normals(d, lc, gs.dv, nr->deg, nr->unrm, first && nr->unrm, nr->tnrm);
          first = false;
        }
      }
      const lcq_status lg = gen_launch(ctx, nr, c, &p->params, gs, false);
      cudaGraph_t g = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(st, &g);
      if (lg != LCQ_OK) ls = lg;
      ck(ee, "end capture");
      if (ls == LCQ_OK) ck(cudaGraphInstantiate(&p->exec, g, 0), "graph instantiate");
      if (g) cudaGraphDestroy(g);
      p->launches = launches + ctx->launches_corr;
    }
    ctx->stream = saved;
    st = saved;
  }
  if (cs) cudaStreamDestroy(cs);
  if (ls != LCQ_OK) {
    cudaGetLastError();
    gen_free(st, &gs);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    delete p;
    return ls;
  }
  *out = p;
  return LCQ_OK;
}

lcq_status lcq_plan_launch(lcq_plan* p) {
  if (!p) return LCQ_ERR_ARG;
  lcq_ctx* ctx = p->ctx;
  CK(cudaSetDevice(ctx->device));
  corr_forget_q(p->corr);
  CK(cudaGraphLaunch(p->exec, ctx->stream));
  ctx->launches_near = 0;
  ctx->launches_corr = p->launches;
  return LCQ_OK;
}

void lcq_plan_destroy(lcq_plan* p) {
  if (!p) return;
  cudaSetDevice(p->ctx->device);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  gen_free(p->ctx->stream, &p->gs);
  cudaGetLastError();
  delete p;
}

void lcq_corr_destroy(lcq_corr* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  dfree(c->stream, c->val);
  dfree(c->stream, c->q);
  dfree(c->stream, c->q_near);
  dfree(c->stream, c->leaves);
  dfree(c->stream, c->src_off);
  dfree(c->stream, c->grp);
  dfree(c->stream, c->gsrc);
  cudaGetLastError();
  delete c;
}

}  // extern "C"
