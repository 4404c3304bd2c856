// Near lists of Sec. 4 (the set N_eta(Gamma_j) of targets inside the oversampled ball
// |x - c_j| <= eta R_j) built through a uniform grid over the patch centroids.
//
// The cell edge h is at least max_j eta R_j, so every patch whose ball holds a target has
// its centroid in the 3x3x3 cells around the target's cell.  The exact FP64 test decides
// membership, so the lists are the same as those of a search over all (target, patch)
// pairs; the grid only bounds the candidates.  Two orders are produced:
//   target-major  rowp_patch (patches of row t, ascending), rowp_off, col   -> CSR rows
//   patch-major   pair_tgt (targets of patch j, ascending), adaptive/annulus split, self
// Ascending order comes from sorting each row / patch segment, so the result does not
// depend on the order of the atomics that fill the buckets.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lcq_internal.h"
#include "lcq_launch.h"

namespace lcq {
namespace {

constexpr int kNT = 256;

struct NearView {
  const double* tgt;
  int64_t NT;
  const double* cen;
  const double* rad;
  const double* eta;
  const double* eta1;
  const int32_t* pgroup;  // null: one surface
  const int32_t* tgroup;
};

NearView nv(const NearArgs& a) {
  return {a.tgt, a.NT, a.cen, a.rad, a.eta, a.eta1, a.pgroup, a.tgroup};
}

// |x_t - c_j|^2 <= (eta_j R_j)^2 (the "<=" reading of the near condition)
__device__ __forceinline__ bool is_near(const NearView& v, int64_t t, int j, double* d2out) {
  const double d0 = v.tgt[t] - v.cen[3 * j], d1 = v.tgt[v.NT + t] - v.cen[3 * j + 1],
               d2 = v.tgt[2 * v.NT + t] - v.cen[3 * j + 2];
  const double d = d0 * d0 + d1 * d1 + d2 * d2;
  const double r = v.eta[j] * v.rad[j];
  *d2out = d;
  return d <= r * r;
}

__device__ __forceinline__ int n_basis_dev(int d) { return (d + 1) * (d + 2) / 2; }

// cell range [lo, hi] per axis of the 3x3x3 neighbourhood of point x (empty if lo > hi)
__device__ __forceinline__ void cell_range(const GridSpec& g, const double x[3], int lo[3],
                                           int hi[3]) {
  const int n[3] = {g.nx, g.ny, g.nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double f = floor((x[a] - g.lo[a]) * g.inv_h);
    const double l = fmax(f - 1.0, 0.0), h = fmin(f + 1.0, (double)(n[a] - 1));
    if (!(l <= h)) {  // also catches NaN
      lo[a] = 1;
      hi[a] = 0;
    } else {
      lo[a] = (int)l;
      hi[a] = (int)h;
    }
  }
}

__device__ __forceinline__ int64_t cell_of(const GridSpec& g, const double* cen, int j) {
  int c[3];
  const int n[3] = {g.nx, g.ny, g.nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double f = floor((cen[3 * j + a] - g.lo[a]) * g.inv_h);
    c[a] = (int)fmin(fmax(f, 0.0), (double)(n[a] - 1));
  }
  return ((int64_t)c[2] * g.ny + c[1]) * g.nx + c[0];
}

// Visits every patch j != own in the neighbourhood cells of target t that passes is_near.
template <class F>
__device__ __forceinline__ void for_near(const NearView& v, const GridSpec& g,
                                         const int64_t* __restrict__ cell_ptr,
                                         const int32_t* __restrict__ cell_patch, int64_t t,
                                         int own, F&& f) {
  const double x[3] = {v.tgt[t], v.tgt[v.NT + t], v.tgt[2 * v.NT + t]};
  const int tg = v.pgroup ? v.tgroup[t] : 0;
  int lo[3], hi[3];
  cell_range(g, x, lo, hi);
  for (int cz = lo[2]; cz <= hi[2]; ++cz)
    for (int cy = lo[1]; cy <= hi[1]; ++cy) {
      const int64_t base = ((int64_t)cz * g.ny + cy) * g.nx;
      const int64_t k0 = cell_ptr[base + (lo[0] <= hi[0] ? lo[0] : 0)];
      const int64_t k1 = lo[0] <= hi[0] ? cell_ptr[base + hi[0] + 1] : k0;
      for (int64_t k = k0; k < k1; ++k) {  // the row of cells is contiguous in cell order
        const int j = cell_patch[k];
        double d2;
        if (j != own && (!v.pgroup || v.pgroup[j] == tg) && is_near(v, t, j, &d2)) f(j, d2);
      }
    }
}

// ---------------------------------------------------------------------------- surfaces
// Surface of each target: that of its patch for on-surface targets, else the caller's
// (user may be null: surface 0).  A caller's value outside [0, G) sets kStBadGroup.
__global__ void k_tgt_group(int64_t NT, const int32_t* __restrict__ tpatch,
                            const int32_t* __restrict__ pgroup, const int32_t* __restrict__ user,
                            int G, int32_t* __restrict__ tgroup, int* __restrict__ status) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < NT;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int tp = tpatch[t];
    int g = 0;
    if (tp >= 0) {
      g = pgroup[tp];
    } else if (user) {
      g = user[t];
      if (g < 0 || g >= G) {
        atomicOr(status, (int)kStBadGroup);
        g = 0;
      }
    }
    tgroup[t] = g;
  }
}

// Surface of each patch of a batch, from the surfaces' patch ranges.
__global__ void k_patch_group(const int64_t* __restrict__ gpatch_off, int G,
                              int32_t* __restrict__ pgroup) {
  for (int g = blockIdx.x; g < G; g += gridDim.x)
    for (int64_t j = gpatch_off[g] + threadIdx.x; j < gpatch_off[g + 1]; j += blockDim.x)
      pgroup[j] = g;
}

// ---------------------------------------------------------------------------- grid
// One block: bounding box of the centroids and max eta_j R_j -> out[0..6].
__global__ void k_grid_bounds(const double* __restrict__ cen, const double* __restrict__ rad,
                              const double* __restrict__ eta, int64_t P, double* __restrict__ out) {
  __shared__ double s[7][32];
  double v[7] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.0};
  for (int64_t j = threadIdx.x; j < P; j += blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      v[a] = fmin(v[a], cen[3 * j + a]);
      v[3 + a] = fmax(v[3 + a], cen[3 * j + a]);
    }
    v[6] = fmax(v[6], eta[j] * rad[j]);
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int a = 0; a < 7; ++a) {
      const double w = __shfl_xor_sync(0xffffffffu, v[a], o);
      v[a] = (a < 3) ? fmin(v[a], w) : fmax(v[a], w);
    }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
    for (int a = 0; a < 7; ++a) s[a][warp] = v[a];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      for (int a = 0; a < 7; ++a) v[a] = (a < 3) ? fmin(v[a], s[a][w]) : fmax(v[a], s[a][w]);
    for (int a = 0; a < 7; ++a) out[a] = v[a];
  }
}

// Counting sort of the patches into the grid cells by centroid: counts, then (after a
// scan) the fill; the order within a cell is fixed later by the per-row sort.
__global__ void k_cell_count(const double* __restrict__ cen, int64_t P, GridSpec g,
                             unsigned long long* __restrict__ cnt) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P;
       j += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[cell_of(g, cen, (int)j)], 1ull);
}

// Fill pass of the counting sort.
__global__ void k_cell_fill(const double* __restrict__ cen, int64_t P, GridSpec g,
                            const int64_t* __restrict__ cell_ptr,
                            unsigned long long* __restrict__ cursor, int32_t* __restrict__ cell_patch) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = cell_of(g, cen, (int)j);
    const unsigned long long k = atomicAdd(&cursor[c], 1ull);
    cell_patch[cell_ptr[c] + (int64_t)k] = (int32_t)j;
  }
}

// ---------------------------------------------------------------------------- rows
// Thread per target: patches in row t (near patches plus the own patch) and entries.
__global__ void k_row_count(NearView v, GridSpec g, const int64_t* __restrict__ cell_ptr,
                            const int32_t* __restrict__ cell_patch,
                            const int32_t* __restrict__ tpatch, const int32_t* __restrict__ deg,
                            int64_t* __restrict__ row_np, int64_t* __restrict__ row_nnz) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < v.NT;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int tp = tpatch[t];
    long long cnt = 0, nnz = 0;
    if (tp >= 0) {
      cnt = 1;
      nnz = n_basis_dev(deg[tp]);
    }
    for_near(v, g, cell_ptr, cell_patch, t, tp, [&](int j, double) {
      ++cnt;
      nnz += n_basis_dev(deg[j]);
    });
    row_np[t] = cnt;
    row_nnz[t] = nnz;
  }
}

// Thread per target: the row's patches, unsorted, into tmp[rowp_ptr[t] ...].
__global__ void k_row_gather(NearView v, GridSpec g, const int64_t* __restrict__ cell_ptr,
                             const int32_t* __restrict__ cell_patch,
                             const int32_t* __restrict__ tpatch,
                             const int64_t* __restrict__ rowp_ptr, int32_t* __restrict__ tmp) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < v.NT;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int tp = tpatch[t];
    int64_t k = rowp_ptr[t];
    if (tp >= 0) tmp[k++] = tp;
    for_near(v, g, cell_ptr, cell_patch, t, tp, [&](int j, double) { tmp[k++] = j; });
  }
}

// Warp per target: rank-sort the row's patches, entry offsets, CSR columns; count the
// patch-major lists (self, near, adaptive) by atomics (counts do not depend on order).
__global__ void k_row_sort(NearView v, const int32_t* __restrict__ tpatch,
                           const int32_t* __restrict__ deg, const int64_t* __restrict__ node_off,
                           const int64_t* __restrict__ rowp_ptr, const int64_t* __restrict__ row_ptr,
                           const int32_t* __restrict__ tmp, int32_t* __restrict__ rowp_patch,
                           int64_t* __restrict__ rowp_off, int32_t* __restrict__ col,
                           unsigned long long* __restrict__ npair,
                           unsigned long long* __restrict__ nad,
                           unsigned long long* __restrict__ nself) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < v.NT;
       t += warps) {
    const int tp = tpatch[t];
    const int64_t b = rowp_ptr[t];
    const int m = (int)(rowp_ptr[t + 1] - b);
    for (int i = lane; i < m; i += 32) {
      const int e = tmp[b + i];
      int r = 0;
      for (int q = 0; q < m; ++q) r += tmp[b + q] < e;
      rowp_patch[b + r] = e;
      if (e == tp) {
        atomicAdd(&nself[e], 1ull);
      } else {
        atomicAdd(&npair[e], 1ull);
        double d2;
        is_near(v, t, e, &d2);
        const double r1 = v.eta1[e] * v.rad[e];
        if (d2 <= r1 * r1) atomicAdd(&nad[e], 1ull);
      }
    }
    __syncwarp();
    // exclusive prefix of n_j over the sorted row, 32 patches at a time
    int64_t carry = 0;
    const int64_t rb = row_ptr[t];
    for (int i0 = 0; i0 < m; i0 += 32) {
      const int i = i0 + lane;
      const int j = i < m ? rowp_patch[b + i] : 0;
      const int nj = i < m ? n_basis_dev(deg[j]) : 0;
      int s = nj;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      const int64_t off = carry + s - nj;
      if (i < m) {
        rowp_off[b + i] = off;
        const int64_t nb = node_off[j];
        for (int l = 0; l < nj; ++l) col[rb + off + l] = (int32_t)(nb + l);
      }
      carry += __shfl_sync(0xffffffffu, s, 31);
    }
  }
}

// ---------------------------------------------------------------------------- patches
// Thread per target: scatter row entries into the patch buckets (unsorted).
__global__ void k_pair_scatter(int64_t NT, const int32_t* __restrict__ tpatch,
                               const int64_t* __restrict__ rowp_ptr,
                               const int32_t* __restrict__ rowp_patch,
                               const int64_t* __restrict__ pair_ptr,
                               const int64_t* __restrict__ self_ptr,
                               unsigned long long* __restrict__ pcur,
                               unsigned long long* __restrict__ scur, int32_t* __restrict__ ptmp,
                               int32_t* __restrict__ stmp) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < NT;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int tp = tpatch[t];
    for (int64_t k = rowp_ptr[t]; k < rowp_ptr[t + 1]; ++k) {
      const int j = rowp_patch[k];
      if (j == tp)
        stmp[self_ptr[j] + (int64_t)atomicAdd(&scur[j], 1ull)] = (int32_t)t;
      else
        ptmp[pair_ptr[j] + (int64_t)atomicAdd(&pcur[j], 1ull)] = (int32_t)t;
    }
  }
}

// Block-wide exclusive prefix of 0/1 flags over one chunk of blockDim items; *total gets
// the chunk's count.  sm holds 33 ints.
__device__ __forceinline__ int flag_scan(int flag, int* sm, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, flag);
  __syncthreads();
  if (lane == 0) sm[warp] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int w = 0; w < nw; ++w) {
      const int c = sm[w];
      sm[w] = acc;
      acc += c;
    }
    sm[32] = acc;
  }
  __syncthreads();
  *total = sm[32];
  return sm[warp] + __popc(bal & ((1u << lane) - 1u));
}

constexpr int kSortStage = 1024;  // segments up to this size: rank sort in shared memory

// Sorts src[0, m) (distinct values) ascending into dst; block-wide.  Short segments: rank
// of each element (O(m^2), staged in shared memory).  Longer ones: bottom-up merge sort
// between src (scratch, overwritten) and dst, each element finding its place by a binary
// search in the partner run (O(m log^2 m)).
__device__ void block_sort(int32_t* __restrict__ src, int m, int32_t* __restrict__ dst,
                           int32_t* stage) {
  if (m <= kSortStage) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) stage[i] = src[i];
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const int e = stage[i];
      int r = 0;
      for (int q = 0; q < m; ++q) r += stage[q] < e;
      dst[r] = e;
    }
    __syncthreads();
    return;
  }
  int32_t* in = src;
  int32_t* out = dst;
  for (int w = 1; w < m; w <<= 1) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const int run = i / w, left = (run & ~1) * w;
      const int p0 = min((run ^ 1) * w, m), p1 = min(p0 + w, m);
      const int e = in[i];
      int lo = p0, hi = p1;  // first partner element not below e
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (in[mid] < e) lo = mid + 1; else hi = mid;
      }
      out[left + (i - run * w) + (lo - p0)] = e;
    }
    __syncthreads();
    int32_t* t = in;
    in = out;
    out = t;
  }
  if (in != dst) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) dst[i] = in[i];
    __syncthreads();
  }
}

__device__ __forceinline__ int64_t row_entry(const int64_t* rowp_ptr, const int32_t* rowp_patch,
                                             const int64_t* rowp_off, const int64_t* row_ptr,
                                             int64_t t, int j) {
  int64_t lo = rowp_ptr[t], hi = rowp_ptr[t + 1] - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (rowp_patch[mid] < j) lo = mid + 1; else hi = mid;
  }
  return row_ptr[t] + rowp_off[lo];
}

// Block per patch: sorted near targets, their squared distances, adaptive / annulus split
// (|x - c_j| <= eta_1 R_j), CSR positions; sorted self targets.
__global__ void __launch_bounds__(kNT) k_patch_fill(
    NearView v, int64_t P, const int64_t* __restrict__ pair_ptr, const int64_t* __restrict__ ad_ptr,
    const int64_t* __restrict__ an_ptr, const int64_t* __restrict__ self_ptr,
    const int64_t* __restrict__ rowp_ptr, const int32_t* __restrict__ rowp_patch,
    const int64_t* __restrict__ rowp_off, const int64_t* __restrict__ row_ptr,
    int32_t* __restrict__ ptmp, int32_t* __restrict__ stmp,
    int32_t* __restrict__ pair_tgt, uint8_t* __restrict__ pair_ad, double* __restrict__ pair_d2,
    int64_t* __restrict__ pair_csr, int32_t* __restrict__ ad_pair, int32_t* __restrict__ an_pair,
    int32_t* __restrict__ self_tgt, int64_t* __restrict__ self_csr) {
  __shared__ int32_t stage[kSortStage];
  __shared__ int sm[33];
  for (int64_t j = blockIdx.x; j < P; j += gridDim.x) {
    const int64_t pb = pair_ptr[j], sb = self_ptr[j];
    const int m = (int)(pair_ptr[j + 1] - pb), ms = (int)(self_ptr[j + 1] - sb);
    block_sort(ptmp + pb, m, pair_tgt + pb, stage);
    block_sort(stmp + sb, ms, self_tgt + sb, stage);
    int64_t abase = ad_ptr[j], nbase = an_ptr[j];
    const double r1 = v.eta1[j] * v.rad[j];
    for (int i0 = 0; i0 < m; i0 += blockDim.x) {
      const int i = i0 + threadIdx.x;
      bool ad = false;
      if (i < m) {
        const int64_t t = pair_tgt[pb + i];
        double d2;
        is_near(v, t, (int)j, &d2);
        ad = d2 <= r1 * r1;
        pair_ad[pb + i] = ad ? 1 : 0;
        pair_d2[pb + i] = d2;
        pair_csr[pb + i] = row_entry(rowp_ptr, rowp_patch, rowp_off, row_ptr, t, (int)j);
      }
      int tota, totn;
      const int apos = flag_scan(i < m && ad, sm, &tota);
      if (i < m && ad) ad_pair[abase + apos] = (int32_t)(pb + i);
      const int npos = flag_scan(i < m && !ad, sm, &totn);
      if (i < m && !ad) an_pair[nbase + npos] = (int32_t)(pb + i);
      abase += tota;
      nbase += totn;
    }
    for (int i = threadIdx.x; i < ms; i += blockDim.x) {
      const int64_t t = self_tgt[sb + i];
      self_csr[sb + i] = row_entry(rowp_ptr, rowp_patch, rowp_off, row_ptr, t, (int)j);
    }
    __syncthreads();
  }
}

int grid_for(const LaunchCommon& lc, int64_t n, int per_sm = 8) {
  const int64_t b = (n + kNT - 1) / kNT;
  const int64_t cap = (int64_t)lc.num_sms * per_sm;
  return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

void launch_groups(const LaunchCommon& lc, int64_t NT, const int32_t* tpatch,
                   const int64_t* gpatch_off, int G, const int32_t* user, int32_t* pgroup,
                   int32_t* tgroup, int* status) {
  ++*lc.launches;
  k_patch_group<<<G < lc.num_sms * 4 ? G : lc.num_sms * 4, kNT, 0, lc.stream>>>(gpatch_off, G,
                                                                                pgroup);
  if (NT > 0) {
    ++*lc.launches;
    k_tgt_group<<<grid_for(lc, NT), kNT, 0, lc.stream>>>(NT, tpatch, pgroup, user, G, tgroup,
                                                          status);
  }
}

void launch_grid_bounds(const LaunchCommon& lc, const NearArgs& a, int64_t P, double* out7) {
  ++*lc.launches;
  k_grid_bounds<<<1, 1024, 0, lc.stream>>>(a.cen, a.rad, a.eta, P, out7);
}

void launch_cell_bins(const LaunchCommon& lc, const NearArgs& a, int64_t P, const GridSpec& g,
                      unsigned long long* cnt, int64_t* cell_ptr, unsigned long long* cursor,
                      int32_t* cell_patch, int64_t* scan_scratch) {
  const int64_t nc = (int64_t)g.nx * g.ny * g.nz;
  ++*lc.launches;
  k_cell_count<<<grid_for(lc, P), kNT, 0, lc.stream>>>(a.cen, P, g, cnt);
  launch_scan(lc, reinterpret_cast<const int64_t*>(cnt), cell_ptr, nc + 1, scan_scratch);
  ++*lc.launches;
  k_cell_fill<<<grid_for(lc, P), kNT, 0, lc.stream>>>(a.cen, P, g, cell_ptr, cursor, cell_patch);
}

void launch_row_count(const LaunchCommon& lc, const NearArgs& a, const GridSpec& g,
                      const int64_t* cell_ptr, const int32_t* cell_patch, const int32_t* tpatch,
                      const int32_t* deg, int64_t* row_np, int64_t* row_nnz) {
  ++*lc.launches;
  k_row_count<<<grid_for(lc, a.NT), kNT, 0, lc.stream>>>(nv(a), g, cell_ptr, cell_patch, tpatch,
                                                          deg, row_np, row_nnz);
}

void launch_row_fill(const LaunchCommon& lc, const NearArgs& a, const GridSpec& g,
                     const int64_t* cell_ptr, const int32_t* cell_patch, const int32_t* tpatch,
                     const int32_t* deg, const int64_t* node_off, const int64_t* rowp_ptr,
                     const int64_t* row_ptr, int32_t* tmp, int32_t* rowp_patch, int64_t* rowp_off,
                     int32_t* col, unsigned long long* npair, unsigned long long* nad,
                     unsigned long long* nself) {
  ++*lc.launches;
  k_row_gather<<<grid_for(lc, a.NT), kNT, 0, lc.stream>>>(nv(a), g, cell_ptr, cell_patch, tpatch,
                                                           rowp_ptr, tmp);
  const int64_t wb = (a.NT + (kNT / 32) - 1) / (kNT / 32);
  const int gw = (int)(wb < 1 ? 1 : (wb < (int64_t)lc.num_sms * 16 ? wb : lc.num_sms * 16));
  ++*lc.launches;
  k_row_sort<<<gw, kNT, 0, lc.stream>>>(nv(a), tpatch, deg, node_off, rowp_ptr, row_ptr, tmp,
                                        rowp_patch, rowp_off, col, npair, nad, nself);
}

void launch_patch_fill(const LaunchCommon& lc, const NearArgs& a, const int32_t* tpatch, int64_t P,
                       const int64_t* pair_ptr, const int64_t* ad_ptr, const int64_t* an_ptr,
                       const int64_t* self_ptr, const int64_t* rowp_ptr, const int32_t* rowp_patch,
                       const int64_t* rowp_off, const int64_t* row_ptr, unsigned long long* pcur,
                       unsigned long long* scur, int32_t* ptmp, int32_t* stmp, int32_t* pair_tgt,
                       uint8_t* pair_ad, double* pair_d2, int64_t* pair_csr, int32_t* ad_pair,
                       int32_t* an_pair, int32_t* self_tgt, int64_t* self_csr) {
  ++*lc.launches;
  k_pair_scatter<<<grid_for(lc, a.NT), kNT, 0, lc.stream>>>(a.NT, tpatch, rowp_ptr, rowp_patch,
                                                             pair_ptr, self_ptr, pcur, scur, ptmp,
                                                             stmp);
  const int g = (int)(P < (int64_t)lc.num_sms * 8 ? (P > 0 ? P : 1) : lc.num_sms * 8);
  ++*lc.launches;
  k_patch_fill<<<g, kNT, 0, lc.stream>>>(nv(a), P, pair_ptr, ad_ptr, an_ptr, self_ptr, rowp_ptr,
                                         rowp_patch, rowp_off, row_ptr, ptmp, stmp, pair_tgt,
                                         pair_ad, pair_d2, pair_csr, ad_pair, an_pair, self_tgt,
                                         self_csr);
}

}  // namespace lcq
