// Internal declarations shared by the host API and the kernel launchers of liblcq.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/lcq.h"

namespace lcq {

constexpr int kMaxDeg = 10;
constexpr int kMaxBasis = (kMaxDeg + 1) * (kMaxDeg + 2) / 2;  // 66
constexpr int kMaxRule = 32;                                   // smooth rules m = 1..32
constexpr int kMaxGL = 32;                                     // Gauss-Legendre orders 1..32
constexpr int kMaxTestPts = 64;

inline int n_basis(int d) { return (d + 1) * (d + 2) / 2; }

// Device status bits (OR-ed into the status word by kernels).
enum : int {
  kStMaxDepth = 1,
  kStCapacity = 2,
  kStDegenerate = 4,
  kStNonFinite = 8,
  kStBadGroup = 16,
};

// The mixed form evaluates kernel values in FP32 for tolerances eps >= kMixedMinEps (with
// FP32 kernel values and contractions the result moves by about 1e-7 relative), in
// two-float arithmetic on the FP32 pipe for kMixedMinEps > eps >= kTwoFloatMinEps (about
// 1e-13 relative) and in FP64 below.
constexpr double kMixedMinEps = 1e-6;
constexpr double kTwoFloatMinEps = 1e-11;

// Kernel parameters (Sec. 3): K = alpha D + beta S for CFIE.
struct KernelParams {
  int kind;          // 0 S, 1 D, 2 CFIE, 3 S' (target normal n_x)
  double kr, ki;     // k = kr + i ki
  double ar, ai;     // alpha
  double br, bi;     // beta
  double eb, ea;     // rounding-envelope weights: |beta| and |alpha| (1,0 for S; 0,1 for D)
};

inline KernelParams make_kernel_params(int kind, double kr, double ki, double ar, double ai,
                                       double br, double bi) {
  KernelParams kp{kind, kr, ki, ar, ai, br, bi, 0.0, 0.0};
  if (kind == 0) {
    kp.ar = kp.ai = kp.br = kp.bi = 0.0;
    kp.eb = 1.0;
  } else if (kind == 1 || kind == 3) {
    kp.ar = kp.ai = kp.br = kp.bi = 0.0;
    kp.ea = 1.0;
  } else {
    kp.eb = __builtin_sqrt(br * br + bi * bi);
    kp.ea = __builtin_sqrt(ar * ar + ai * ai);
  }
  return kp;
}

// Physics of one independent surface of a batch (patches of a contiguous range): kernel,
// far-order tolerance eps, adaptive tolerance eps * eps_loosen, self-rule order.
struct GroupParams {
  KernelParams kp;
  double eps;
  double eps_ad;
  int self_order;
  int pad;
};

// Per-degree reference tables uploaded to the device (built on the host).
struct DegTables {
  int d = 0, n = 0;
  double normV = 0;
  std::vector<double> u, v, w;   // discretization nodes and weights [n]
  std::vector<double> V;         // values-to-coefficients, row-major [n][n] (row = nm)
  double* dV = nullptr;          // device copy of V
  double* dnodes = nullptr;      // device [3][n]: u, v, w
  // derivative projections [n][n_{d-1}]: d/du and d/dv of K_nm in the degree d-1 basis
  std::vector<double> Du, Dv;
  double* dDuv = nullptr;        // device copy: Du then Dv
};

// Smooth rule family and Gauss-Legendre tables on the device.
struct RuleTables {
  std::vector<int> off;          // off[m] = first node of rule m (m = 1..kMaxRule), size kMaxRule+2
  std::vector<double> u, v, w;
  std::vector<int> gl_off;       // Gauss-Legendre order g at gl_off[g], g = 1..kMaxGL
  std::vector<double> gl_x, gl_w;   // on [0,1]
  int* doff = nullptr;
  double* du = nullptr;
  double* dv = nullptr;
  double* dw = nullptr;
  int* dgl_off = nullptr;
  double* dgl_x = nullptr;
  double* dgl_w = nullptr;
};

// Host table construction (lcq_tables.cu).
bool build_deg_tables(int d, DegTables* t);
bool build_rule_tables(RuleTables* t);
void ref_nodes_host(int d, std::vector<double>* u, std::vector<double>* v);
void koornwinder_host(int d, double u, double v, double* K);

}  // namespace lcq

// ----------------------------------------------------------------------------- handles
// Online tuner of the adaptive walk's work-group size for one key (degree, kernel, tolerance
// decade, precision, size class of the adaptive work): every candidate is timed once, on the
// generations that use the key, by events around that degree's adaptive launch; later
// generations use the fastest.  The group size changes the schedule, never a result.
struct lcq_tune {
  std::vector<int> cand;        // candidate group sizes (targets per work item)
  std::vector<double> ms_per;   // adaptive milliseconds per adaptive pair, < 0 untried
  int pending = -1;             // candidate whose timing is in flight
  double pend_pairs = 0.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

struct lcq_ctx {
  int device = 0;
  std::map<uint64_t, lcq_tune> tune;
  int last_group_size = 0;      // largest work-group size of the last generation
  long long last_items = 0;     // adaptive work items of the last generation (host count)
  int last_forms = 0;           // pair evaluation forms of the last generation (bit 0 FP32, bit 1 two-float)
  cudaStream_t stream = nullptr;
  int* d_status = nullptr;
  long long* d_counters = nullptr;   // [8]
  int* d_sched = nullptr;            // dynamic-scheduling counters, one per degree
  int num_sms = 0;
  lcq::DegTables deg[lcq::kMaxDeg + 1];
  lcq::RuleTables rules;
  bool rules_ready = false;
  std::string last_error;
  // grow-only workspace for the adaptive kernel
  void* work = nullptr;
  size_t work_bytes = 0;
  // stage events: [0,1] near lists, [2..7] corrections
  cudaEvent_t ev[8] = {};
  // side stream: the self weights run beside far order, moments and adaptive integration
  // correction generation: the dependent stages run on `hi` (highest priority), the self
  // weights beside them on `side` (lowest), both forked from and joined back into `stream`
  cudaStream_t side = nullptr, hi = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, done = nullptr, ev_self[2] = {};
  long long launches_near = 0, launches_corr = 0;
};

struct lcq_near {
  int64_t n_patches = 0, n_targets = 0, n_points = 0;
  std::vector<int32_t> deg_h;
  std::vector<int64_t> node_off_h;
  int32_t* deg = nullptr;
  int64_t* node_off = nullptr;
  double* coef = nullptr;        // [N][3] Koornwinder coefficients of the charts
  double* cen = nullptr;         // [P][3]
  double* rad = nullptr;         // [P]
  double* dj = nullptr;          // [P]
  double* eta = nullptr;         // [P]
  double* eta1 = nullptr;        // [P]
  double* tgt = nullptr;         // [3][NT] copy of the targets
  int32_t* tgt_patch = nullptr;  // [NT]
  int32_t* tgt_lnode = nullptr;  // [NT] node index within its patch (-1 off surface)
  int64_t* tnode = nullptr;      // [NT] copy of the caller's global node ids
  int64_t* row_ptr = nullptr;    // [NT+1] CSR entries
  int64_t* rowp_ptr = nullptr;   // [NT+1] patches per row
  int32_t* rowp_patch = nullptr; // [sum] patch ids of each row, ascending
  int64_t* rowp_off = nullptr;   // [sum] entry offset of that patch inside the row
  int32_t* col = nullptr;        // [nnz]
  int64_t* pair_ptr = nullptr;   // [P+1] patch-major near pairs
  int32_t* pair_tgt = nullptr;   // [n_pairs]
  uint8_t* pair_ad = nullptr;    // [n_pairs] 1 = adaptive
  double* pair_d2 = nullptr;     // [n_pairs]
  int64_t* pair_csr = nullptr;   // [n_pairs] first CSR entry of the pair
  int64_t* ad_ptr = nullptr;     // [P+1]
  int32_t* ad_pair = nullptr;    // [n_adaptive] pair ids
  int64_t* an_ptr = nullptr;     // [P+1]
  int32_t* an_pair = nullptr;    // [n_annulus]
  int32_t* self_tgt = nullptr;   // [n_self]
  int64_t* self_csr = nullptr;   // [n_self]
  int64_t* self_ptr = nullptr;   // [P+1] self pairs grouped by patch
  int64_t n_pairs = 0, n_self = 0, n_adaptive = 0, n_annulus = 0, nnz = 0;
  int64_t max_adaptive = 0, max_pairs = 0, max_self = 0;
  lcq_params params{};
  // launch bookkeeping
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_max = 0;                              // largest n over the degrees present
  int plist_count[lcq::kMaxDeg + 1] = {0};    // patches of each degree
  int* plist_dev[lcq::kMaxDeg + 1] = {nullptr};
  int ad_count[lcq::kMaxDeg + 1] = {0};       // patches with adaptive targets, by degree,
  int* ad_list_dev[lcq::kMaxDeg + 1] = {nullptr};  // most adaptive targets first
  int64_t ad_total[lcq::kMaxDeg + 1] = {0};   // adaptive pairs of each degree
  int64_t ad_max[lcq::kMaxDeg + 1] = {0};     // largest adaptive set of each degree
  std::vector<int64_t> ad_nad_h[lcq::kMaxDeg + 1];  // adaptive targets of each listed patch
  // batches of independent surfaces (n_groups > 1 or built by the batched entry point)
  int n_groups = 1;
  bool grouped = false;
  std::vector<int64_t> gpatch_off;  // [n_groups+1] patch range of each surface
  int32_t* pgroup = nullptr;        // [P] surface of each patch
  int32_t* tgroup = nullptr;        // [NT] surface of each target
  // S': caller's normals of off-surface targets and the unit target normals in use
  double* unrm = nullptr;           // [3][NT]
  double* tnrm = nullptr;           // [3][NT]
};

struct lcq_corr {
  const lcq_near* near = nullptr;   // not owned; must outlive the correction object
  cudaStream_t stream = nullptr;
  int device = 0;
  int kernel = 0;
  int64_t n_patches = 0, n_targets = 0, nnz = 0, n_pairs = 0, n_self = 0, n_over = 0;
  lcq::KernelParams kp{};
  lcq_params params{};           // generation parameters (test directions dropped)
  double eps0 = 0.0;             // tolerance (first surface's in a batch)
  int precision = 0;             // lcq_precision of the generation
  int form = 0;                  // pair evaluation form of the moment kernels (pair_form)
  double* val = nullptr;         // [nnz][2]
  int32_t* q = nullptr;          // [P]
  int32_t* q_near = nullptr;     // [P]
  int32_t* leaves = nullptr;     // [n_pairs]
  int64_t* src_off = nullptr;    // [P+1] oversampled source offsets (apply)
  std::vector<int32_t> q_h;
  lcq::GroupParams* grp = nullptr;  // [n_groups] per-surface physics (batched), else null
  std::vector<lcq::GroupParams> grp_h;
  int64_t* gsrc = nullptr;          // [n_groups+1] oversampled source range of each surface
  std::vector<int64_t> gsrc_h;
  std::vector<double> dirs_h;       // far-order test directions of the generation
  int gsz[lcq::kMaxDeg + 1] = {0};  // adaptive work-group size of each degree
};
