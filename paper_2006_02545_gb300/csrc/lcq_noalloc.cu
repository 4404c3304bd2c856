// Allocation-free entry point: adaptive near corrections of one patch, for callers that
// cannot allocate device memory (see lcq_adaptive_corrections_noalloc in include/lcq.h).
//
// Every device buffer the computation needs -- tables, patch geometry, the near-list
// view, the smooth and adaptive moments and the adaptive kernel's union-tree workspace --
// is carved out of one file-scope device array of fixed size.  The kernels are the same
// ones lcq_gen_corrections launches; only their storage differs.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "lcq_internal.h"
#include "lcq_launch.h"

namespace lcq {
namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;  // 8 MiB, held by every GPU that loads liblcq
constexpr int kNoAllocMaxTargets = 128;
constexpr int kNoAllocMaxDeg = 8;
constexpr int kNoAllocMaxDepth = 16;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Per-device set-up state: the device address of g_scratch (a host-side use of the
// symbol's name is not a device address) and whether the tables were uploaded.
struct DeviceState {
  bool ready = false;
  unsigned char* base = nullptr;
  int num_sms = 0;
};
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;

// Byte offsets of the regions inside g_scratch.
struct Layout {
  size_t status, counters, sched, plist, node_off, Vt, nodes, duv, coef, cen, rad, dj, eta, eta1, tpatch,
      tlnode, pair_ptr, pair_tgt, pair_d2, pair_csr, ad_ptr, ad_pair, an_ptr, an_pair, self_ptr,
      self_tgt, self_csr, q, qn, roff, ru, rv, rw, gl_off, gl_x, gl_w, Is, In, leaves, work;
  size_t end;
};

size_t bump(size_t* at, size_t bytes) {
  const size_t o = (*at + 255) & ~size_t(255);
  *at = o + bytes;
  return o;
}

Layout layout(const RuleTables& r, int64_t work_bytes) {
  constexpr int A = kNoAllocMaxTargets, n = (kNoAllocMaxDeg + 1) * (kNoAllocMaxDeg + 2) / 2;
  Layout L{};
  size_t at = 0;
  L.status = bump(&at, sizeof(int));
  L.counters = bump(&at, 8 * sizeof(long long));
  L.sched = bump(&at, sizeof(int));
  L.plist = bump(&at, sizeof(int));
  L.node_off = bump(&at, 2 * 8);
  L.Vt = bump(&at, n * n * 8);
  L.nodes = bump(&at, 3 * n * 8);
  L.duv = bump(&at, 2 * n * n * 8);
  L.coef = bump(&at, 3 * n * 8);
  L.cen = bump(&at, 3 * 8);
  L.rad = bump(&at, 8);
  L.dj = bump(&at, 8);
  L.eta = bump(&at, 8);
  L.eta1 = bump(&at, 8);
  L.tpatch = bump(&at, A * 4);
  L.tlnode = bump(&at, A * 4);
  L.pair_ptr = bump(&at, 2 * 8);
  L.pair_tgt = bump(&at, A * 4);
  L.pair_d2 = bump(&at, A * 8);
  L.pair_csr = bump(&at, A * 8);
  L.ad_ptr = bump(&at, 2 * 8);
  L.ad_pair = bump(&at, A * 4);
  L.an_ptr = bump(&at, 2 * 8);
  L.an_pair = bump(&at, 4);
  L.self_ptr = bump(&at, 2 * 8);
  L.self_tgt = bump(&at, 4);
  L.self_csr = bump(&at, 8);
  L.q = bump(&at, 4);
  L.qn = bump(&at, 4);
  L.roff = bump(&at, r.off.size() * sizeof(int));
  L.ru = bump(&at, r.u.size() * 8);
  L.rv = bump(&at, r.v.size() * 8);
  L.rw = bump(&at, r.w.size() * 8);
  L.gl_off = bump(&at, r.gl_off.size() * sizeof(int));
  L.gl_x = bump(&at, r.gl_x.size() * 8);
  L.gl_w = bump(&at, r.gl_w.size() * 8);
  L.Is = bump(&at, (size_t)A * n * 16);
  L.In = bump(&at, (size_t)A * n * 16);
  L.leaves = bump(&at, A * 4);
  L.work = bump(&at, (size_t)work_bytes);
  L.end = at;
  return L;
}

// Union-tree workspace of one k_adaptive block (same formula as lcq_gen_corrections).
int64_t work_stride(int64_t A, int64_t n, int levels) {
  int64_t s = A * n * 16 + A * 4 * n * 16 + (int64_t)levels * A * 4 * n * 16 +
              (int64_t)levels * A * 4 + 2 * A * 4 + (int64_t)levels * 4 + 8 + A * 4 * 8 + 256;
  return (s + 255) / 256 * 256;
}

// Host tables, built once per process.  Both are safe when several host threads make
// their first calls at the same time (different GPUs may be driven concurrently): the rule
// tables are a function-local static (initialized once, under the runtime's lock) and each
// degree's tables are built under std::call_once.
const RuleTables& host_rules() {
  static const RuleTables r = [] {
    RuleTables t;
    build_rule_tables(&t);
    return t;
  }();
  return r;
}

const DegTables& host_deg(int d) {
  static DegTables t[kMaxDeg + 1];
  static std::once_flag once[kMaxDeg + 1];
  std::call_once(once[d], [d] { build_deg_tables(d, &t[d]); });
  return t[d];
}

// Near-list view of "one patch, every target adaptive": identity pair lists.
__global__ void k_noalloc_view(int NT, int n, int32_t* tpatch, int32_t* tlnode, int64_t* pair_ptr,
                               int32_t* pair_tgt, double* pair_d2, int64_t* pair_csr,
                               int64_t* ad_ptr, int32_t* ad_pair, int64_t* an_ptr,
                               int64_t* self_ptr, int* plist, int64_t* node_off, int* status,
                               long long* counters) {
  for (int i = threadIdx.x; i < NT; i += blockDim.x) {
    tpatch[i] = -1;
    tlnode[i] = -1;
    pair_tgt[i] = i;
    pair_d2[i] = 0.0;
    pair_csr[i] = (int64_t)i * n;
    ad_pair[i] = i;
  }
  if (threadIdx.x == 0) {
    pair_ptr[0] = 0;
    pair_ptr[1] = NT;
    ad_ptr[0] = 0;
    ad_ptr[1] = NT;
    an_ptr[0] = an_ptr[1] = 0;
    self_ptr[0] = self_ptr[1] = 0;
    plist[0] = 0;
    node_off[0] = 0;
    node_off[1] = n;
    *status = 0;
  }
  if (threadIdx.x < 8) counters[threadIdx.x] = 0;
}

// Once per device, with that device current: the scratch array's device address, the
// per-device Koornwinder constants and the constant rule tables.
lcq_status setup_device(int dev, cudaStream_t st) {
  std::lock_guard<std::mutex> g(g_mu);
  DeviceState& s = g_dev[dev];
  if (s.ready) return LCQ_OK;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return LCQ_ERR_CUDA;
  }
  if (cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return LCQ_ERR_CUDA;
  }
  if (upload_constants(st) != cudaSuccess) {
    cudaGetLastError();
    return LCQ_ERR_CUDA;
  }
  const RuleTables& r = host_rules();
  const Layout L = layout(r, 0);
  unsigned char* b = static_cast<unsigned char*>(p);
  cudaError_t e = cudaSuccess;
  auto up = [&](size_t off, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + off, src, bytes, cudaMemcpyHostToDevice, st);
  };
  up(L.roff, r.off.data(), r.off.size() * sizeof(int));
  up(L.ru, r.u.data(), r.u.size() * 8);
  up(L.rv, r.v.data(), r.v.size() * 8);
  up(L.rw, r.w.data(), r.w.size() * 8);
  up(L.gl_off, r.gl_off.data(), r.gl_off.size() * sizeof(int));
  up(L.gl_x, r.gl_x.data(), r.gl_x.size() * 8);
  up(L.gl_w, r.gl_w.data(), r.gl_w.size() * 8);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LCQ_ERR_CUDA;
  }
  s.base = b;
  s.ready = true;
  return LCQ_OK;
}

}  // namespace
}  // namespace lcq

using namespace lcq;

extern "C" lcq_status lcq_adaptive_corrections_noalloc(
    int deg, const double* y, int64_t n_targets, const double* tgt_xyz, lcq_kernel kernel,
    double k_re, double k_im, double alpha_re, double alpha_im, double beta_re, double beta_im,
    int q, double eps, int max_depth, void* cuda_stream, double* out) {
  if (deg < 1 || deg > kNoAllocMaxDeg || n_targets < 1 || n_targets > kNoAllocMaxTargets ||
      max_depth < 1 || max_depth > kNoAllocMaxDepth)
    return LCQ_ERR_CAPACITY;
  if (!y || !tgt_xyz || !out || q < 1 || q > kMaxRule || !(eps > 0.0) || k_im < 0.0 ||
      (int)kernel < 0 || (int)kernel > 2)
    return LCQ_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return LCQ_ERR_CUDA;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  // the call copies host values and synchronizes its stream: not allowed in a capture
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return LCQ_ERR_ARG;
  }
  if (cap != cudaStreamCaptureStatusNone) return LCQ_ERR_ARG;
  lcq_status s = setup_device(dev, st);
  if (s != LCQ_OK) return s;
  const DeviceState& ds = g_dev[dev];
  const RuleTables& r = host_rules();
  const DegTables& dt = host_deg(deg);
  const int n = dt.n, NT = (int)n_targets;
  const int64_t stride = work_stride(NT, n, max_depth);
  const Layout L = layout(r, stride);
  if (L.end > kScratchBytes) return LCQ_ERR_CAPACITY;
  unsigned char* b = ds.base;
  auto I = [&](size_t off) { return reinterpret_cast<int*>(b + off); };
  auto I32 = [&](size_t off) { return reinterpret_cast<int32_t*>(b + off); };
  auto I64 = [&](size_t off) { return reinterpret_cast<int64_t*>(b + off); };
  auto F = [&](size_t off) { return reinterpret_cast<double*>(b + off); };

  // per-call tables of this degree
  double nodes[3 * kMaxBasis];
  for (int i = 0; i < n; ++i) {
    nodes[i] = dt.u[i];
    nodes[n + i] = dt.v[i];
    nodes[2 * n + i] = dt.w[i];
  }
  cudaError_t e = cudaMemcpyAsync(F(L.Vt), dt.V.data(), (size_t)n * n * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(F(L.nodes), nodes, (size_t)3 * n * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(F(L.duv), dt.Du.data(), dt.Du.size() * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(F(L.duv) + dt.Du.size(), dt.Dv.data(), dt.Dv.size() * 8,
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(I32(L.q), &q, sizeof(int), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LCQ_ERR_CUDA;
  }
  long long launches = 0;
  LaunchCommon lc{st, ds.num_sms, &launches};
  // everything the kernels read as zero or as list structure is (re)written each call
  k_noalloc_view<<<1, 128, 0, st>>>(NT, n, I32(L.tpatch), I32(L.tlnode), I64(L.pair_ptr),
                                    I32(L.pair_tgt), F(L.pair_d2), I64(L.pair_csr), I64(L.ad_ptr),
                                    I32(L.ad_pair), I64(L.an_ptr), I64(L.self_ptr), I(L.plist),
                                    I64(L.node_off), I(L.status),
                                    reinterpret_cast<long long*>(b + L.counters));
  const double eta_p = -1.0, eta1_p = 1.25;
  launch_geom(deg, lc, I(L.plist), 1, I64(L.node_off), y, n, F(L.Vt), F(L.nodes), eta_p, eta1_p,
              F(L.coef), F(L.cen), F(L.rad), F(L.dj), F(L.eta), F(L.eta1), I(L.status));
  const KernelParams kp =
      make_kernel_params((int)kernel, k_re, k_im, alpha_re, alpha_im, beta_re, beta_im);
  Dev dv{};
  dv.coef = F(L.coef);
  dv.node_off = I64(L.node_off);
  dv.cen = F(L.cen);
  dv.rad = F(L.rad);
  dv.dj = F(L.dj);
  dv.eta = F(L.eta);
  dv.eta1 = F(L.eta1);
  dv.tgt = tgt_xyz;
  dv.NT = NT;
  dv.tpatch = I32(L.tpatch);
  dv.tlnode = I32(L.tlnode);
  dv.pair_ptr = I64(L.pair_ptr);
  dv.pair_tgt = I32(L.pair_tgt);
  dv.pair_d2 = F(L.pair_d2);
  dv.pair_csr = I64(L.pair_csr);
  dv.ad_ptr = I64(L.ad_ptr);
  dv.ad_pair = I32(L.ad_pair);
  dv.an_ptr = I64(L.an_ptr);
  dv.an_pair = I32(L.an_pair);
  dv.self_ptr = I64(L.self_ptr);
  dv.self_tgt = I32(L.self_tgt);
  dv.self_csr = I64(L.self_csr);
  dv.n_self = 0;
  dv.q = I32(L.q);
  dv.roff = I(L.roff);
  dv.ru = F(L.ru);
  dv.rv = F(L.rv);
  dv.rw = F(L.rw);
  dv.gl_off = I(L.gl_off);
  dv.gl_x = F(L.gl_x);
  dv.gl_w = F(L.gl_w);
  dv.nodes_uv[deg] = F(L.nodes);
  dv.duv[deg] = F(L.duv);
  dv.counters = reinterpret_cast<long long*>(b + L.counters);
  dv.status = I(L.status);
  dv.ldI = n;
  // smooth-rule moments (the root of the adaptive walk), adaptive moments, V^T contraction
  launch_rule_moments(deg, lc, I(L.plist), 1, dv, 1, I32(L.q), nullptr, kp, F(L.Is), nullptr);
  launch_adaptive(deg, lc, I(L.plist), 1, dv, kp, eps, dt.normV, 0, max_depth, F(L.Is), F(L.In),
                  I32(L.leaves), b + L.work, stride, NT, max_depth, 1, I(L.status), I(L.sched));
  launch_v2c(deg, lc, I(L.plist), 1, dv, F(L.Vt), F(L.In), F(L.Is), nullptr, out);
  int hst = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, I(L.status), sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LCQ_ERR_CUDA;
  }
  if (hst & kStNonFinite) return LCQ_ERR_NONFINITE;
  if (hst & kStDegenerate) return LCQ_ERR_DEGENERATE_PATCH;
  if (hst & kStCapacity) return LCQ_ERR_CAPACITY;
  if (hst & kStMaxDepth) return LCQ_ERR_MAX_DEPTH;
  return LCQ_OK;
}
