// Device code shared by the forward kernels (lcq_kernels.cu) and the adjoint kernels
// (lcq_adjoint.cu): block-level helpers, the moment engine of Sec. 4.2-4.3 and the
// union-tree adaptive kernel, which the adjoint instantiates with gradient accumulation.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lcq_device.cuh"
#include "lcq_launch.h"
#include "lcq_tc.cuh"

namespace lcq {

constexpr int kThreads = 256;
constexpr double kRoundingFloor = 2e-13;  // multiple of the FP64 rounding envelope never asked below
constexpr double kF32Floor = 2e-6;        // the same for kernel values evaluated in FP32
constexpr double kTwoFloatFloor = 5e-11;  // and in two-float arithmetic (2^8 times the FP64 one)

// ============================================================================ helpers
// Form of the pair evaluations for patch j (block_moments_tc): mode 0, 1 or 2 as given; 3
// chooses per surface of a batch from its tolerance (FP32 for eps >= kMixedMinEps,
// two-float for eps >= kTwoFloatMinEps, FP64 below).
__device__ __forceinline__ int pair_form(const Dev& dv, int j, int mode) {
  if (mode != 3) return mode;
  if (!dv.pgroup) return 0;
  const double e = dv.grp[dv.pgroup[j]].eps;
  return e >= kMixedMinEps ? 1 : (e >= kTwoFloatMinEps ? 2 : 0);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide exclusive prefix of 0/1 flags for one chunk of blockDim items.
// Returns this thread's position; *total receives the chunk's count.  Uses sm[33].
__device__ __forceinline__ int block_flag_scan(int flag, int* sm, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, flag);
  const int inwarp = __popc(bal & ((1u << lane) - 1u));
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
  return sm[warp] + inwarp;
}

// Kernel of patch j: its surface's in a batch of independent surfaces, else the launch's.
// Patch of oversampled source q: the largest j with src_off[j] <= q.
__device__ __forceinline__ int patch_of_source(const int64_t* src_off, int64_t P, int64_t q) {
  int64_t lo = 0, hi = P;  // largest j with src_off[j] <= q
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) / 2;
    if (src_off[mid] <= q) lo = mid; else hi = mid;
  }
  return (int)lo;
}

__device__ __forceinline__ KernelParams patch_kp(const Dev& dv, int j, const KernelParams& kp) {
  return dv.pgroup ? dv.grp[dv.pgroup[j]].kp : kp;
}

__device__ __forceinline__ double eta_default(int d) {
  const int p = d + 1;
  return p <= 4 ? 2.75 : (p <= 8 ? 2.0 : 1.25);
}

// ============================================================================ moments
template <int D>
struct Cfg {
  static constexpr int n = (D + 1) * (D + 2) / 2;
  static constexpr int CH = 128;  // nodes per chunk (two blocks per SM fit in shared memory)
  static constexpr int BS = n + 1;
  static constexpr int TT = 16;
  // doubles of shared workspace used by block_moments
  static constexpr int WS = CH * BS + 7 * CH + 3 * TT * CH + 6 * TT;
};

struct SegMap {
  double ax, ay, e1x, e1y, e2x, e2y, det;
};

// Moments I[i][seg][nm] = sum_{q in seg} w_q K(x_i, X_q) J_q K_nm(u_q, v_q) for a smooth
// rule (Q nodes) pushed onto nseg affine images of T0, for T targets, in FP64 throughout
// (the far order q_j, whose decisions compare these moments, and the moments of the
// smallest degrees, block_moments_any).  Geometry is evaluated once per chunk of nodes and
// shared by all targets (Sec. 4.3 reuse).
// TA: target accessor (pos(i, x[3])); out row of target i: out + orow(i) * ostride.
// Positions are relative to the patch centroid cen (the coefficients cf describe
// X - cen); cfd holds the derivative series of load_coef_derivs, which replace the
// derivative recurrences.  With ENV, eout[i * nseg + seg] also receives the summed FP64
// rounding envelope (through the basis rows' column of ones).
template <int D, bool ENV = false, class TA, class OR>
__device__ void block_moments(const double* cf, const double* cfd, const double* __restrict__ ru,
                              const double* __restrict__ rv, const double* __restrict__ rw, int Q,
                              const SegMap* segs, int nseg, const TA& ta, int T, OR orow,
                              int64_t ostride, const KernelParams& kp, double* sm,
                              const double* cen, double R = 0.0, double* eout = nullptr) {
  using C = Cfg<D>;
  double* B = sm;
  double* Xs = B + C::CH * C::BS;
  double* Ns = Xs + 3 * C::CH;
  double* Js = Ns + 3 * C::CH;
  cplx* G = reinterpret_cast<cplx*>(Js + C::CH);
  double* Ev = reinterpret_cast<double*>(G + C::TT * C::CH);
  double* tx = Ev + C::TT * C::CH;
  double* tn = tx + 3 * C::TT;  // target normals (S')
  static_assert(C::n < C::BS, "the basis rows need a spare column");
  (void)ostride;
  const KernelParamsF kf = to_f32(kp);
  const bool has_ki = kp.ki != 0.0;
  const int total = nseg * Q;
  // The rules are conical products, rows of mr nodes sharing v, and every segment map
  // here keeps v a function of the rule's v alone (e1y = 0: T0 and all its midpoint
  // descendants); the v-only factors of the basis and chart sums are then formed once per
  // row (kw_row_factors), into the tile area, which is free during the geometry phase.
  const int mr = (int)lrint(sqrt((double)Q));
  bool by_rows = mr * mr == Q;
  for (int sg = 0; sg < nseg; ++sg) by_rows = by_rows && segs[sg].e1y == 0.0;
  using RW = KwRow<D>;
  constexpr int kRowMax = 3 * C::TT * C::CH / RW::size;
  double* rows = reinterpret_cast<double*>(G);
  for (int c0 = 0; c0 < total; c0 += C::CH) {
    const int nch = min(C::CH, total - c0);
    const int row0 = by_rows ? c0 / mr : 0;
    const bool use_rows = by_rows && (c0 + nch - 1) / mr - row0 + 1 <= kRowMax;
    __syncthreads();
    if (use_rows) {
      // one thread per (row, m): the rows spread over all warps, hence all SM sub-partitions
      const int nrow = (c0 + nch - 1) / mr - row0 + 1;
      for (int e = threadIdx.x; e < nrow * (D + 1); e += blockDim.x) {
        const int m = e / nrow, rr = e - m * nrow;  // m-major: the lanes share m
        const int rg = row0 + rr, sg = rg / mr, l0 = (rg - sg * mr) * mr;
        const SegMap& S = segs[sg];
        kw_row_factors<D>(S.ay + ru[l0] * S.e1y + rv[l0] * S.e2y, m, cf, cfd,
                          rows + rr * RW::size);
      }
      __syncthreads();
    }
    for (int ql = threadIdx.x; ql < nch; ql += blockDim.x) {
      const int q = c0 + ql;
      const int sg = q / Q, l = q - sg * Q;
      const SegMap& S = segs[sg];
      const double r0 = ru[l], r1 = rv[l];
      const double u = S.ax + r0 * S.e1x + r1 * S.e2x;
      const double w = rw[l] * S.det;
      double X[3], Xu[3], Xv[3], Nn[3];
      if (use_rows) {
        kw_geometry_row<D>(u, rows + (q / mr - row0) * RW::size, X, Xu, Xv, B + ql * C::BS);
      } else {
        const double v = S.ay + r0 * S.e1y + r1 * S.e2y;
        kw_geometry_proj<D>(u, v, cf, cfd, X, Xu, Xv, B + ql * C::BS);
      }
      if (ENV) B[ql * C::BS + C::n] = 1.0;  // the envelope's column
      cross3(Xu, Xv, Nn);
      const double J = sqrt(Nn[0] * Nn[0] + Nn[1] * Nn[1] + Nn[2] * Nn[2]);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Xs[c * C::CH + ql] = X[c];
        Ns[c * C::CH + ql] = Nn[c] * w;
      }
      Js[ql] = J * w;
    }
    __syncthreads();
    for (int t0 = 0; t0 < T; t0 += C::TT) {
      const int nt = min(C::TT, T - t0);
      if (threadIdx.x < nt) {
        double* xp = tx + 3 * threadIdx.x;
        ta.pos(t0 + threadIdx.x, xp);
        xp[0] -= cen[0];
        xp[1] -= cen[1];
        xp[2] -= cen[2];
        if (kp.kind == 3) ta.nrm(t0 + threadIdx.x, xp, tn + 3 * threadIdx.x);
      }
      __syncthreads();
      // kernel values by the table sincos and the Newton-refined 1/sqrt; with ENV the
      // FP64 form with its rounding envelope
      for (int e = threadIdx.x; e < nt * nch; e += blockDim.x) {
        const int i = e / nch, ql = e - i * nch;
        if (ENV) {
          double ev = 0.0;
          G[i * C::CH + ql] = kernel_eval(kp, tx[3 * i], tx[3 * i + 1], tx[3 * i + 2], Xs[ql],
                                          Xs[C::CH + ql], Xs[2 * C::CH + ql], Ns[ql],
                                          Ns[C::CH + ql], Ns[2 * C::CH + ql], Js[ql], R, &ev,
                                          tn + 3 * i);
          Ev[i * C::CH + ql] = ev;
        } else {
          float unused;
          G[i * C::CH + ql] = kernel_eval_tc(kp, kf, g_sct, tx[3 * i], tx[3 * i + 1],
                                             tx[3 * i + 2], Xs[ql], Xs[C::CH + ql],
                                             Xs[2 * C::CH + ql], Ns[ql], Ns[C::CH + ql],
                                             Ns[2 * C::CH + ql], Js[ql], 0.0f, 0.0f, &unused,
                                             tn + 3 * i, has_ki);
        }
      }
      __syncthreads();
      // one thread per (target, nm), outputs packed densely; with ENV the extra index nm = n
      // sums the envelope through the basis rows' column of ones.  Node ranges are uniform
      // across the block, so the loops do not diverge.
      constexpr int W = C::n + (ENV ? 1 : 0);
      const int nout = nt * W;
      for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        const int i = o / W, nm = o - i * W;
        const bool env = ENV && nm == C::n;
        for (int sg = 0; sg < nseg; ++sg) {
          const int qa = max(sg * Q - c0, 0), qb = min((sg + 1) * Q - c0, nch);
          if (qa >= qb) continue;
          const bool first = sg * Q >= c0;  // the segment starts in this chunk
          double are = 0.0, aim = 0.0;
          const double* pr = env ? Ev + i * C::CH : &G[i * C::CH].re;
          const int st = env ? 1 : 2;
          const double* pi = env ? pr : pr + 1;
          for (int ql = qa; ql < qb; ++ql) {
            const double bv = B[ql * C::BS + nm];
            are = fma(pr[ql * st], bv, are);
            aim = fma(pi[ql * st], bv, aim);
          }
          if (env) {
            double* ed = eout + (int64_t)(t0 + i) * nseg + sg;
            *ed = first ? are : *ed + are;
          } else {
            cplx* dst = reinterpret_cast<cplx*>(orow(t0 + i)) + (int64_t)sg * C::n + nm;
            if (first) {
              dst->re = are;
              dst->im = aim;
            } else {
              dst->re += are;
              dst->im += aim;
            }
          }
        }
      }
      __syncthreads();
    }
  }
}

// The split of kernel rows for the tensor-core moments (block_moments_tc below), with the
// contraction over the nodes on the tensor cores by the exact NS-slice split (lcq_tc.cuh):
// NS = 8 for FP64 kernel values, NS = 5 for the mixed form's FP32 ones.
// Chunks never straddle a segment: segment sg's Q nodes are cut into parts of at most
// TcCfg::CH nodes, each padded with zero columns to a multiple of 16 (the MMA depth), and
// each chunk's contribution is assembled in FP64 and written (first part) or added.
// Per chunk: (1) geometry, thread per node: X, N w, J w and the basis row (FP64); (2) per
// tile of 8 targets: kernel values and envelopes, thread per (target, node); (3) one warp
// per target splits the Re and Im rows of its kernel values on their own power-of-two
// scales into NS f16 slices; (4) one warp per n-tile of 8 basis columns slices its basis
// values (fixed per-column bounds) into MMA fragments and accumulates the diagonals
// i + j <= 8 (FP64; i + j < 5 for the mixed form) over
// the chunk's 16-node steps with mma.sync, then assembles and stores the 8 x 8 complex
// block.  smb: TcCfg<D>::BYTES of shared memory (16-byte aligned); sct: the sincos table.
// Rows t (Re) and t + 8 (Im) of the kernel values, VPL consecutive columns q0.. per lane,
// on their own power-of-two scales into NS f16 slices of the swizzled A array (one warp).
template <int D, int NS, int VPL, class V>
__device__ __forceinline__ void split_row_pair(const V* re, const V* im, bool on, uint16_t* Asl,
                                               int t, int q0, int* rowE) {
  using C = TcCfg<D>;
  int fr = 0, fi = 0;
  bool bad = false;
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int a = exp_field(re[v]), b = exp_field(im[v]);
    bad = bad || exp_nonfinite(a, V()) || exp_nonfinite(b, V());
    fr = max(fr, a);
    fi = max(fi, b);
  }
  fr = (int)__reduce_max_sync(0xffffffffu, (unsigned)fr);
  fi = (int)__reduce_max_sync(0xffffffffu, (unsigned)fi);
  bad = __any_sync(0xffffffffu, bad);
  const int Er = exp_bound(fr, V()), Ei = exp_bound(fi, V());
  if ((threadIdx.x & 31) == 0) {
    rowE[t] = !on ? 0 : (bad ? kPoisonExp : Er);
    rowE[t + 8] = !on ? 0 : (bad ? kPoisonExp : Ei);
  }
#pragma unroll
  for (int part = 0; part < 2; ++part) {
    const V* x = part ? im : re;
    const int E = part ? Ei : Er;
    const int row = t + 8 * part;
    unsigned long long M[VPL];
    uint32_t sg[VPL / 2];
#pragma unroll
    for (int v = 0; v < VPL; ++v) M[v] = on ? fix_mag<NS>(x[v], E) : 0ull;
#pragma unroll
    for (int v = 0; v < VPL / 2; ++v) sg[v] = sign_bits(x[2 * v], x[2 * v + 1]);
    uint16_t* dst = Asl + C::swz(row, q0);
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      uint16_t* d = dst + (size_t)i * 16 * C::CH;
      const uint32_t w0 = half2_ints(slice_of<NS>(M[0], i), slice_of<NS>(M[1], i), sg[0]);
      if (VPL == 4) {
        const uint32_t w1 = half2_ints(slice_of<NS>(M[2], i), slice_of<NS>(M[3], i), sg[1]);
        *reinterpret_cast<uint2*>(d) = make_uint2(w0, w1);
      } else {
        *reinterpret_cast<uint32_t*>(d) = w0;
      }
    }
  }
}

// The 8 slices of basis value K_nm (column idx) of node k into the swizzled B array.
template <int D>
__device__ __forceinline__ void store_basis_slices(uint16_t* Bsl, int idx, int k, double v) {
  using C = TcCfg<D>;
  const unsigned long long M = fix_mag<8>(v, c_kwexp[idx]);
  const bool neg = __double2hiint(v) < 0;
  uint16_t* b = Bsl + C::swz(idx, k);
#pragma unroll
  for (int i = 0; i < 8; i += 2) {
    const uint32_t h = half2_pair(slice_of<8>(M, i), slice_of<8>(M, i + 1), neg);
    b[(size_t)i * C::NP * C::CH] = (uint16_t)(h & 0xffffu);
    b[(size_t)(i + 1) * C::NP * C::CH] = (uint16_t)(h >> 16);
  }
}

// One n-tile (basis columns 8 ct .. 8 ct + 7) of one piece of the chunk (columns kbeg ..
// kend - 1, one segment sg): the diagonals d = i + j < ND of the slice products over the
// k-steps (A and B fragments by ldmatrix), then the assembled complex 8 x 8 block into the
// outputs (stored when first, else added).
template <int D, int NS, int ND, class OR>
__device__ __forceinline__ void tc_tile(const uint16_t* Bsl, const uint16_t* Asl, const int* rowE,
                                        int ct, int kbeg, int kend, int nt, int t0, int sg,
                                        bool first, OR orow) {
  using C = TcCfg<D>;
  constexpr int n = C::n;
  constexpr int NB = (NS + 1) / 2;  // slice pairs of B loaded per k-step
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  float acc[ND][4];
#pragma unroll
  for (int d = 0; d < ND; ++d) acc[d][0] = acc[d][1] = acc[d][2] = acc[d][3] = 0.0f;
  const int arow = (lane & 7) + ((lane >> 3) & 1) * 8, acol = (lane >> 4) * 8;
  const int brow = ct * 8 + (lane & 7), bcol = ((lane >> 3) & 1) * 8, bsl = lane >> 4;
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    uint32_t bf[2 * NB][2];
#pragma unroll
    for (int p = 0; p < NB; ++p) {
      uint32_t r[4];
      ldsm_x4(r, Bsl + (size_t)(2 * p + bsl) * C::NP * C::CH + C::swz(brow, k0 + bcol));
      bf[2 * p][0] = r[0];
      bf[2 * p][1] = r[1];
      bf[2 * p + 1][0] = r[2];
      bf[2 * p + 1][1] = r[3];
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      uint32_t af[4];
      ldsm_x4(af, Asl + (size_t)i * 16 * C::CH + C::swz(arow, k0 + acol));
#pragma unroll
      for (int j = 0; j < NS && i + j < ND; ++j) mma_f16_16816(acc[i + j], af, bf[j]);
    }
  }
  if (g < nt) {
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      const int nm = ct * 8 + 2 * c + cc;
      if (nm >= n) continue;
      const int e2 = c_kwexp[nm];
      const double re = assemble<ND>(acc, cc, rowE[g] + e2);
      const double im = assemble<ND>(acc, 2 + cc, rowE[g + 8] + e2);
      cplx* dst = reinterpret_cast<cplx*>(orow(t0 + g)) + (int64_t)sg * n + nm;
      if (first) {
        dst->re = re;
        dst->im = im;
      } else {
        dst->re += re;
        dst->im += im;
      }
    }
  }
}

// Moments as block_moments (the adaptive walk, the smooth-rule and annulus moments):
// I[i][seg][nm] = sum_{q in seg} w_q K(x_i, X_q) J_q K_nm(u_q, v_q) and, when eout is not
// null, eout[i * nseg + seg] = sum_q of the kernel's rounding envelope (FP32 sums), with the
// contraction over the nodes on the tensor cores by the exact slice split (lcq_tc.cuh):
// 8 slices per FP64 operand and the diagonals i + j <= 8 for FP64 kernel values; for the mixed
// form's FP32 kernel values 5 slices and the diagonals i + j <= 4.
// A chunk is a run of pieces (segment sg, its nodes l0 .. l0 + nq - 1), each padded with
// zero columns to a multiple of 16 (the MMA depth), packed while they fit in TcCfg::CH
// columns: the four children of a small rule share one chunk.  Each piece's contribution is
// assembled in FP64 and written (the segment's first part) or added.
// Per chunk: (1) geometry, thread per real node (padding columns are zeroed apart, so no
// lane of the FP64 work idles): X, N w, J w (FP64), and each basis value split into 8 f16
// slices on its column's fixed bound as it is formed (integer work that runs in the shadow
// of the FP64 geometry); (2) per tile of 8 targets: kernel values and envelopes, thread per
// (target, real node); (3) one warp per target splits the Re and Im rows of its kernel
// values on their own power-of-two scales; (4) one warp per n-tile of 8 basis columns
// accumulates the diagonals over each piece's 16-node steps with mma.sync, both operands read
// by ldmatrix, and assembles and stores its 8 x 8 complex block.
// For real k and kinds S, D and CFIE with a real alpha the kernel constants are folded into
// the node data (kernel_eval_fold).  smb: TcCfg<D>::BYTES of shared memory (16-byte aligned).
// form: 0 FP64 kernel values; 1 FP32 ones (the mixed form for eps >= kMixedMinEps); 2
// two-float ones (kernel_eval_ff; the mixed form below that) where the constants fold, else
// FP64.
template <int D, class TA, class OR>
__device__ void block_moments_tc(const double* cf, const double* cfd, const double* __restrict__ ru,
                                 const double* __restrict__ rv, const double* __restrict__ rw,
                                 int Q, const SegMap* segs, int nseg, const TA& ta, int T, OR orow,
                                 const KernelParams& kp, unsigned char* smb, const double* cen,
                                 double R, double* eout, int form) {
  using C = TcCfg<D>;
  constexpr int n = C::n;
  double* Xs = reinterpret_cast<double*>(smb + C::OFF_X);
  double* Ns = reinterpret_cast<double*>(smb + C::OFF_N);
  double* Js = reinterpret_cast<double*>(smb + C::OFF_J);
  double* Ks = reinterpret_cast<double*>(smb + C::OFF_K);
  uint16_t* Bsl = reinterpret_cast<uint16_t*>(smb + C::OFF_BS);
  cplx* Gs = reinterpret_cast<cplx*>(smb + C::OFF_G);
  float2* Gf = reinterpret_cast<float2*>(smb + C::OFF_G);
  uint16_t* Asl = reinterpret_cast<uint16_t*>(smb + C::OFF_G);
  double* rows = reinterpret_cast<double*>(smb + C::OFF_G);
  float* Ef = reinterpret_cast<float*>(smb + C::OFF_EF);
  float* Jf = reinterpret_cast<float*>(smb + C::OFF_JF);
  float* Nf = reinterpret_cast<float*>(smb + C::OFF_NF);
  int* rowE = reinterpret_cast<int*>(smb + C::OFF_ROWE);
  double* tx = reinterpret_cast<double*>(smb + C::OFF_TX);
  double* tn = tx + 3 * C::TT;
  int* colinfo = reinterpret_cast<int*>(smb + C::OFF_CI);  // (piece << 16) | node, 0xffff: pad
  int* pcs = reinterpret_cast<int*>(smb + C::OFF_PC);      // [piece][sg, l0, nq, po, row0, rb, first]
  const KernelParamsF kf = to_f32(kp);
  const float fR = f32_bits(R);
  const bool mixed = form == 1;
  const bool has_ki = kp.ki != 0.0;
  // real k, kinds S, D and CFIE with a real alpha: constants folded into the node data
  const bool fold = !mixed && !has_ki && kp.kind <= 2 && kp.ai == 0.0;
  const bool ffe = fold && form == 2;  // two-float kernel values
  const float escale = mixed ? (float)(kF32Floor / kRoundingFloor)
                             : ffe ? (float)(kTwoFloatFloor / kRoundingFloor) : 1.0f;
  const ff krf = ff_of(kp.kr);
  ff* Nff = reinterpret_cast<ff*>(Ns);  // two-float node data in the FP64 slots
  ff* Jff = reinterpret_cast<ff*>(Js);
  ff* Kff = reinterpret_cast<ff*>(Ks);
  constexpr double kInv4Pi = 0.07957747154594767;
  const double fa_n = (kp.kind == 1 ? 1.0 : kp.ar) * kInv4Pi;
  const double fj_r = (kp.kind == 0 ? 1.0 : kp.br) * kInv4Pi, fj_i = kp.bi * kInv4Pi;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // conical rules: rows of mr nodes sharing v (see block_moments)
  const int mr = (int)lrint(sqrt((double)Q));
  bool by_rows = mr * mr == Q;
  for (int sg = 0; sg < nseg; ++sg) by_rows = by_rows && segs[sg].e1y == 0.0;
  using RW = KwRow<D>;
  constexpr int kRowMax = C::G_BYTES / 8 / RW::size;
  const int nparts = (Q + C::CH - 1) / C::CH;
  const int psize = (Q + nparts - 1) / nparts;
  // the padding columns n .. NP-1 of the basis slices stay zero
  __syncthreads();
  for (int e = threadIdx.x; e < C::NSMAX * (C::NP - n) * C::CH; e += blockDim.x) {
    const int i = e / ((C::NP - n) * C::CH), r = e - i * (C::NP - n) * C::CH;
    const int col = n + r / C::CH, k = r - (col - n) * C::CH;
    Bsl[(size_t)i * C::NP * C::CH + C::swz(col, k)] = 0;
  }
  int sg_next = 0, part_next = 0;
  while (sg_next < nseg) {
    // plan the chunk (uniform across the block); thread 0 records it for indexed lookups
    int np = 0, ncp = 0, nrow = 0, ncr = 0;
    __syncthreads();
    while (sg_next < nseg && np < C::MAXP) {
      const int l0 = part_next * psize, nq = min(psize, Q - l0), pad = (nq + 15) & ~15;
      if (np > 0 && ncp + pad > C::CH) break;
      if (threadIdx.x == 0) {
        int* pc = pcs + 8 * np;
        pc[0] = sg_next;
        pc[1] = l0;
        pc[2] = nq;
        pc[3] = ncp;
        pc[4] = by_rows ? l0 / mr : 0;
        pc[5] = nrow;
        pc[6] = part_next == 0;
        pc[7] = ncr;
      }
      nrow += by_rows ? (l0 + nq - 1) / mr - l0 / mr + 1 : 0;
      ncp += pad;
      ncr += nq;
      ++np;
      if (++part_next == nparts) {
        part_next = 0;
        ++sg_next;
      }
    }
    const bool use_rows = by_rows && nrow <= kRowMax;
    __syncthreads();
    for (int p = threadIdx.x; p < ncp; p += blockDim.x) {
      int k = 0;
      for (int kk = 1; kk < np; ++kk)
        if (pcs[8 * kk + 3] <= p) k = kk;
      const int ql = p - pcs[8 * k + 3];
      colinfo[p] = (k << 16) | (ql < pcs[8 * k + 2] ? ql : 0xffff);
    }
    if (use_rows) {
      // m-major, so that the lanes of a warp share m and with it the loop length
      for (int e = threadIdx.x; e < nrow * (D + 1); e += blockDim.x) {
        const int m = e / nrow, rr = e - m * nrow;
        int k = 0;
        for (int kk = 1; kk < np; ++kk)
          if (pcs[8 * kk + 5] <= rr) k = kk;
        const int* pc = pcs + 8 * k;
        const SegMap& S = segs[pc[0]];
        const int l = (pc[4] + rr - pc[5]) * mr;
        kw_row_factors<D>(S.ay + ru[l] * S.e1y + rv[l] * S.e2y, m, cf, cfd, rows + rr * RW::size);
      }
    }
    __syncthreads();
    // column of the r-th real node of the chunk (the pieces' real columns are contiguous):
    // the FP64 loops run over real nodes only, so that no lane of theirs idles on padding
    auto real_col = [&](int r) {
      int k = 0;
      for (int kk = 1; kk < np; ++kk)
        if (pcs[8 * kk + 7] <= r) k = kk;
      return pcs[8 * k + 3] + (r - pcs[8 * k + 7]);
    };
    // padding columns: zero basis slices
    for (int p = threadIdx.x; p < ncp; p += blockDim.x)
      if ((colinfo[p] & 0xffff) == 0xffff) {
#pragma unroll 1
        for (int idx = 0; idx < n; ++idx)
#pragma unroll
          for (int i = 0; i < 8; ++i) Bsl[(size_t)i * C::NP * C::CH + C::swz(idx, p)] = 0;
      }
    // (1) geometry and basis slices, thread per real node
    for (int rn = threadIdx.x; rn < ncr; rn += blockDim.x) {
      const int p = real_col(rn);
      const int ci = colinfo[p], ql = ci & 0xffff;
      {
        const int* pc = pcs + 8 * (ci >> 16);
        const SegMap& S = segs[pc[0]];
        const int l = pc[1] + ql;
        const double r0 = ru[l], r1 = rv[l];
        const double u = S.ax + r0 * S.e1x + r1 * S.e2x;
        const double w = rw[l] * S.det;
        double X[3], Xu[3], Xv[3], Nn[3];
        if (use_rows) {
          kw_geometry_row_emit<D>(u, rows + (pc[5] + l / mr - pc[4]) * RW::size, X, Xu, Xv,
                                  [&](int idx, double kv) { store_basis_slices<D>(Bsl, idx, p, kv); });
        } else {
          double K[n];
          const double v = S.ay + r0 * S.e1y + r1 * S.e2y;
          kw_geometry_proj<D>(u, v, cf, cfd, X, Xu, Xv, K);
#pragma unroll 1
          for (int idx = 0; idx < n; ++idx) store_basis_slices<D>(Bsl, idx, p, K[idx]);
        }
        cross3(Xu, Xv, Nn);
        const double N2 = fma(Nn[0], Nn[0], fma(Nn[1], Nn[1], Nn[2] * Nn[2]));
        const double Jw = N2 > 0.0 ? N2 * rsqrt_nr(N2) * w : 0.0;
        const double wn = fold ? w * fa_n : w;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Xs[c * C::CH + p] = X[c];
          if (ffe) Nff[c * C::CH + p] = ff_of(Nn[c] * wn);
          else Ns[c * C::CH + p] = Nn[c] * wn;
        }
        if (ffe) {
          Jff[p] = ff_of(Jw * fj_r);
          Kff[p] = ff_of(Jw * fj_i);
        } else {
          Js[p] = fold ? Jw * fj_r : Jw;
          Ks[p] = fold ? Jw * fj_i : 0.0;
        }
        Jf[p] = f32_bits(fold ? Jw * kInv4Pi : Jw);
        if (mixed) {
#pragma unroll
          for (int c = 0; c < 3; ++c) Nf[c * C::CH + p] = (float)(Nn[c] * w);
          Jf[p] = (float)Jw;
        }
      }
    }
    __syncthreads();
    for (int t0 = 0; t0 < T; t0 += C::TT) {
      const int nt = min(C::TT, T - t0);
      if (threadIdx.x < nt) {
        double* xp = tx + 3 * threadIdx.x;
        ta.pos(t0 + threadIdx.x, xp);
        xp[0] -= cen[0];
        xp[1] -= cen[1];
        xp[2] -= cen[2];
        if (kp.kind == 3) ta.nrm(t0 + threadIdx.x, xp, tn + 3 * threadIdx.x);
      }
      __syncthreads();
      // (2) kernel values and envelopes of the real columns; zeros in the padding ones
      for (int e = threadIdx.x; e < nt * ncp; e += blockDim.x) {
        const int i = e / ncp, p = e - i * ncp;
        if ((colinfo[p] & 0xffff) == 0xffff) {
          if (mixed) Gf[i * C::CH + p] = make_float2(0.0f, 0.0f);
          else Gs[i * C::CH + p] = cplx{0.0, 0.0};
          Ef[i * C::CH + p] = 0.0f;
        }
      }
      for (int e = threadIdx.x; e < nt * ncr; e += blockDim.x) {
        const int i = e / ncr, p = real_col(e - i * ncr);
        float ev = 0.0f;
        if (mixed) {
          float2 g = make_float2(0.0f, 0.0f);
          const double d0 = tx[3 * i] - Xs[p], d1 = tx[3 * i + 1] - Xs[C::CH + p],
                       d2 = tx[3 * i + 2] - Xs[2 * C::CH + p];
          const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
          if (r2 > 0.0)
            g = kernel_eval_f32f(kp, kf, d0, d1, d2, r2, Nf[p], Nf[C::CH + p], Nf[2 * C::CH + p],
                                 Jf[p], fR, &ev);
          Gf[i * C::CH + p] = g;
        } else {
          cplx g;
          if (ffe) {
            const ff Np[3] = {Nff[p], Nff[C::CH + p], Nff[2 * C::CH + p]};
            g = kernel_eval_ff(kp.kind, kp.kr, krf, kf, g_sct, g_sctf, tx[3 * i], tx[3 * i + 1],
                               tx[3 * i + 2], Xs[p], Xs[C::CH + p], Xs[2 * C::CH + p], Np,
                               Jff[p], Kff[p], Jf[p], fR, &ev);
          } else if (fold) {
            g = kernel_eval_fold(kp.kind, kp.kr, kf, g_sct, tx[3 * i], tx[3 * i + 1],
                                 tx[3 * i + 2], Xs[p], Xs[C::CH + p], Xs[2 * C::CH + p], Ns[p],
                                 Ns[C::CH + p], Ns[2 * C::CH + p], Js[p], Ks[p], Jf[p], fR, &ev);
          } else {
            g = kernel_eval_tc(kp, kf, g_sct, tx[3 * i], tx[3 * i + 1], tx[3 * i + 2], Xs[p],
                               Xs[C::CH + p], Xs[2 * C::CH + p], Ns[p], Ns[C::CH + p],
                               Ns[2 * C::CH + p], Js[p], Jf[p], fR, &ev, tn + 3 * i, has_ki);
          }
          Gs[i * C::CH + p] = g;
        }
        Ef[i * C::CH + p] = ev;
      }
      __syncthreads();
      // envelope sums, one warp per target, one sum per piece
      if (eout && warp < nt) {
        for (int k = 0; k < np; ++k) {
          const int* pc = pcs + 8 * k;
          float es = 0.0f;
          for (int ql = lane; ql < pc[2]; ql += 32) es += Ef[warp * C::CH + pc[3] + ql];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) es += __shfl_xor_sync(0xffffffffu, es, o);
          if (lane == 0) {
            double* ed = eout + (int64_t)(t0 + warp) * nseg + pc[0];
            const double v = (double)(es * escale);
            *ed = pc[6] ? v : *ed + v;
          }
        }
      }
      // (3) split the kernel rows: warp w owns target w (rows w: Re, w + 8: Im); values are
      // read before the barrier because the slices overwrite them
      constexpr int VPL = C::CH / 32;
      const int q0 = lane * VPL;
      const bool on = warp < nt;
      if (mixed) {
        float re[VPL], im[VPL];
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
          const float2 g = (on && q0 + v < ncp) ? Gf[warp * C::CH + q0 + v] : make_float2(0.0f, 0.0f);
          re[v] = g.x;
          im[v] = g.y;
        }
        __syncthreads();
        if (warp < C::TT) split_row_pair<D, 5, VPL>(re, im, on, Asl, warp, q0, rowE);
      } else {
        double re[VPL], im[VPL];
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
          const cplx g = (on && q0 + v < ncp) ? Gs[warp * C::CH + q0 + v] : cplx{0.0, 0.0};
          re[v] = g.re;
          im[v] = g.im;
        }
        __syncthreads();
        if (warp < C::TT) split_row_pair<D, 8, VPL>(re, im, on, Asl, warp, q0, rowE);
      }
      __syncthreads();
      // (4) tensor-core contraction, one warp per n-tile, piece by piece
      for (int ct = warp; ct < C::NTILE; ct += nwarp) {
        for (int k = 0; k < np; ++k) {
          const int* pc = pcs + 8 * k;
          const int kb = pc[3], ke = pc[3] + ((pc[2] + 15) & ~15);
          if (mixed)
            tc_tile<D, 5, 5>(Bsl, Asl, rowE, ct, kb, ke, nt, t0, pc[0], pc[6] != 0, orow);
          else
            tc_tile<D, 8, 9>(Bsl, Asl, rowE, ct, kb, ke, nt, t0, pc[0], pc[6] != 0, orow);
        }
      }
      __syncthreads();
    }
  }
}

// The moments of the smallest degrees in the FP64 form (n <= 10 basis functions) by the
// plain FP64 engine (16-target tiles, one thread per output): there the contraction is too
// small to pay for the tensor-core pipeline's fixed cost per 8-target tile (barriers, the
// slice split).  Every other case: block_moments_tc.  smb holds either engine's workspace.
constexpr int kFp64MomentsMaxDeg = 3;
template <int D, class TA, class OR>
__device__ __forceinline__ void block_moments_any(
    const double* cf, const double* cfd, const double* __restrict__ ru,
    const double* __restrict__ rv, const double* __restrict__ rw, int Q, const SegMap* segs,
    int nseg, const TA& ta, int T, OR orow, const KernelParams& kp, unsigned char* smb,
    const double* cen, double R, double* eout, int form) {
  if constexpr (D <= kFp64MomentsMaxDeg) {
    if (form == 0) {
      double* sm = reinterpret_cast<double*>(smb);
      if (eout)
        block_moments<D, true>(cf, cfd, ru, rv, rw, Q, segs, nseg, ta, T, orow, Cfg<D>::n, kp, sm,
                               cen, R, eout);
      else
        block_moments<D, false>(cf, cfd, ru, rv, rw, Q, segs, nseg, ta, T, orow, Cfg<D>::n, kp, sm,
                                cen);
      return;
    }
  }
  block_moments_tc<D>(cf, cfd, ru, rv, rw, Q, segs, nseg, ta, T, orow, kp, smb, cen, R, eout,
                      form);
}

// Shared-memory bytes of the moment workspace (either engine's).
template <int D>
constexpr size_t moment_ws_bytes() {
  return D <= kFp64MomentsMaxDeg && sizeof(double) * Cfg<D>::WS > (size_t)TcCfg<D>::BYTES
             ? sizeof(double) * Cfg<D>::WS
             : (size_t)TcCfg<D>::BYTES;
}

template <int D>
__device__ __forceinline__ void load_coef(const double* __restrict__ coef, int64_t off, double* cf) {
  constexpr int n = (D + 1) * (D + 2) / 2;
  for (int e = threadIdx.x; e < 3 * n; e += blockDim.x) cf[e] = coef[off * 3 + e];
}

// Target accessors of block_moments: pos(i, x) the position of target i; nrm(i, xrel, n)
// its unit normal for S' (the caller's normals tn, SoA [3][NT]; for bare test points the
// radial direction from the centroid, xrel being the position relative to it).
__device__ __forceinline__ void read_nrm(const double* tn, int64_t NT, int64_t t, double* n) {
  n[0] = tn[t];
  n[1] = tn[NT + t];
  n[2] = tn[2 * NT + t];
}
struct TgtIdx {  // targets by id list
  const double* tgt;
  int64_t NT;
  const int32_t* ids;
  const double* tn;
  __device__ void pos(int i, double* x) const {
    const int64_t t = ids[i];
    x[0] = tgt[t];
    x[1] = tgt[NT + t];
    x[2] = tgt[2 * NT + t];
  }
  __device__ void nrm(int i, const double*, double* n) const { read_nrm(tn, NT, ids[i], n); }
};
struct TgtPairIdx {  // targets of pair ids
  const double* tgt;
  int64_t NT;
  const int32_t* pair_tgt;
  const int32_t* pairs;
  const double* tn;
  __device__ void pos(int i, double* x) const {
    const int64_t t = pair_tgt[pairs[i]];
    x[0] = tgt[t];
    x[1] = tgt[NT + t];
    x[2] = tgt[2 * NT + t];
  }
  __device__ void nrm(int i, const double*, double* n) const {
    read_nrm(tn, NT, pair_tgt[pairs[i]], n);
  }
};
struct TgtPts {  // explicit points [i][3]
  const double* p;
  __device__ void pos(int i, double* x) const {
    x[0] = p[3 * i];
    x[1] = p[3 * i + 1];
    x[2] = p[3 * i + 2];
  }
  __device__ void nrm(int, const double* xr, double* n) const {
    const double r = sqrt(xr[0] * xr[0] + xr[1] * xr[1] + xr[2] * xr[2]);
    if (r > 0.0) {
      n[0] = xr[0] / r;
      n[1] = xr[1] / r;
      n[2] = xr[2] / r;
    } else {
      n[0] = n[1] = 0.0;
      n[2] = 1.0;
    }
  }
};

struct TgtAdaptive {  // targets of a union-tree node: local ids -> pairs -> targets
  const double* tgt;
  int64_t NT;
  const int32_t* pair_tgt;
  const int32_t* apairs;
  const int* ST;
  const double* tn;
  __device__ void pos(int i, double* x) const {
    const int64_t t = pair_tgt[apairs[ST[i]]];
    x[0] = tgt[t];
    x[1] = tgt[NT + t];
    x[2] = tgt[2 * NT + t];
  }
  __device__ void nrm(int i, const double*, double* n) const {
    read_nrm(tn, NT, pair_tgt[apairs[ST[i]]], n);
  }
};

__device__ __forceinline__ SegMap seg_T0() { return {0.0, 0.0, 1.0, 0.0, 0.0, 1.0, 1.0}; }

// ============================================================================ adjoint
// Gradient moments (adjoint of Sec. 4.2-4.3 rules with the rule frozen): for the nodes of
// a rule pushed onto nseg sub-triangles and T targets with weights wf(i) = conj(g_t)
// (0: skip), accumulates into the thread-private M[3n]
//   dL/dx_nm += sum_nodes K_nm a_X + dK_nm/du (X_v x a_N) + dK_nm/dv (a_N x X_u),
//   a_X = Re(w sigma(u) sum_i wf(i) dK~/dX),  a_N = Re(w sigma(u) sum_i wf(i) dK~/dN),
// where sigma(u) = sum_nm shat_nm K_nm(u) and N = X_u x X_v (so a_N.dN splits into the
// two cross products).  Thread per node; targets staged through shared memory.
// WARP_ACC: M is instead this warp's row of per-warp sums in shared memory; every lane
// takes part (zeros for lanes without a node) and lane 0 adds the warp's sum.
template <int D, bool WARP_ACC = false, class TA, class WF>
__device__ void block_grad(const double* cf, const double* __restrict__ ru,
                           const double* __restrict__ rv, const double* __restrict__ rw, int Q,
                           const SegMap* segs, int nseg, const TA& ta, int T, WF wf,
                           const KernelParams& kp, const cplx* shat, const double* cen,
                           double* M) {
  constexpr int TG = 32;
  __shared__ double gx[TG][3];
  __shared__ cplx gwt[TG];
  const int total = nseg * Q;
  for (int c0 = 0; c0 < total; c0 += blockDim.x) {
    const int q = c0 + threadIdx.x;
    const bool on = q < total;
    double u = 0.0, v = 0.0, w = 0.0, X[3] = {0, 0, 0}, Xu[3] = {0, 0, 0}, Xv[3] = {0, 0, 0};
    double Nn[3] = {0, 0, 0};
    cplx sg = {0.0, 0.0};
    if (on) {
      const int s = q / Q, l = q - s * Q;
      const SegMap& S = segs[s];
      u = S.ax + ru[l] * S.e1x + rv[l] * S.e2x;
      v = S.ay + ru[l] * S.e1y + rv[l] * S.e2y;
      w = rw[l] * S.det;
      kw_geometry<D>(u, v, cf, X, Xu, Xv, nullptr, 1);
      cross3(Xu, Xv, Nn);
      kw_for_each<D>(u, v, [&](int idx, double k0, double, double) {
        sg.re = fma(shat[idx].re, k0, sg.re);
        sg.im = fma(shat[idx].im, k0, sg.im);
      });
    }
    cplx SX[3] = {{0, 0}, {0, 0}, {0, 0}}, SN[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int t0 = 0; t0 < T; t0 += TG) {
      const int nt = min(TG, T - t0);
      __syncthreads();
      if (threadIdx.x < nt) {
        double xp[3];
        ta.pos(t0 + threadIdx.x, xp);
        gx[threadIdx.x][0] = xp[0] - cen[0];
        gx[threadIdx.x][1] = xp[1] - cen[1];
        gx[threadIdx.x][2] = xp[2] - cen[2];
        gwt[threadIdx.x] = wf(t0 + threadIdx.x);
      }
      __syncthreads();
      if (on)
        for (int i = 0; i < nt; ++i) {
          const cplx c = gwt[i];
          if (c.re == 0.0 && c.im == 0.0) continue;
          cplx dX[3], dN[3];
          kernel_grad(kp, gx[i], X, Nn, dX, dN);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const cplx a = cmul(c, dX[k]), b = cmul(c, dN[k]);
            SX[k].re += a.re;
            SX[k].im += a.im;
            SN[k].re += b.re;
            SN[k].im += b.im;
          }
        }
    }
    if (WARP_ACC || on) {
      double aX[3], aN[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        aX[k] = w * (sg.re * SX[k].re - sg.im * SX[k].im);
        aN[k] = w * (sg.re * SN[k].re - sg.im * SN[k].im);
      }
      double bu[3], bv[3];
      cross3(Xv, aN, bu);
      cross3(aN, Xu, bv);
      if constexpr (WARP_ACC) {
        const bool lead = (threadIdx.x & 31) == 0;
        kw_for_each<D>(u, v, [&](int idx, double k0, double ku, double kv) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const double s = warp_sum(k0 * aX[k] + ku * bu[k] + kv * bv[k]);
            if (lead) M[idx * 3 + k] += s;
          }
        });
      } else {
        kw_for_each<D>(u, v, [&](int idx, double k0, double ku, double kv) {
#pragma unroll
          for (int k = 0; k < 3; ++k) M[idx * 3 + k] += k0 * aX[k] + ku * bu[k] + kv * bv[k];
        });
      }
    }
  }
}

// Block sum of the thread-private M[3n] in a fixed order, added to out[3n] (global).
// Uses sm[(blockDim/32) * 3n] doubles of shared memory.
template <int D>
__device__ void block_reduce_M(const double* M, double* sm, double* out) {
  constexpr int n3 = 3 * Cfg<D>::n;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
#pragma unroll 1
  for (int e = 0; e < n3; ++e) {
    const double v = warp_sum(M[e]);
    if (lane == 0) sm[wp * n3 + e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n3; e += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < nw; ++k) acc += sm[k * n3 + e];
    out[e] += acc;
  }
  __syncthreads();
}

// ============================================================================ adaptive
// Adaptive subdivision (Sec. 4.3) for all eta_1-near targets of a patch at once.
// The refinement trees of the targets are walked as one union tree, depth first:
// a node T carries the set S of targets that refine T; the leaf-rule geometry of T's
// four children is evaluated once and contracted with every target in S (the reuse
// of X, K_nm and J across targets of Fig. multipletargpot).  A target accepts the
// children's sum when ||I_T - sum_c I_c||_2 <= max(tol0 4^-L, 2e-13 E), E the summed
// rounding envelope of the kernel over the children's nodes.
constexpr int kMaxTreeNodes = 1 << 16;  // union-tree nodes walked per patch at most

struct AdaptiveWS {
  int64_t stride;   // bytes per block
  int A_max, levels;
};

// Dynamic shared memory of k_adaptive<D>: chart coefficients, the four child maps, scan
// scratch, the walk's stack, alignment, and the tensor-core moment workspace.
template <int D>
constexpr size_t adaptive_smem_bytes() {
  return sizeof(double) * 3 * Cfg<D>::n + sizeof(SegMap) * 4 + 64 * sizeof(int) +
         4 * 32 * sizeof(unsigned long long) + 128 + moment_ws_bytes<D>();
}

// Work items are taken dynamically through the counter *sched, which the caller zeroes
// before the launch.  gofs == nullptr: item b is the patch plist[b] with all its adaptive
// targets.  Otherwise item i is group g of patch plist[b], gofs[b] <= i < gofs[b + 1]
// (an exclusive scan of the groups per listed patch, gofs[count] their total), the group
// being the adaptive targets g gsz .. g gsz + gsz - 1 of the patch: small groups spread one
// patch's walk over several blocks.  Every target's refinement tree, moments and leaf
// count are the same whichever group it walks with (its tests and sums are its own, and a
// depth-first walk of a union tree visits the nodes of each member tree in that tree's own
// depth-first order), so the grouping changes the schedule, not the results.  plist is
// ordered by decreasing number of adaptive targets (longest items first).
template <int D, bool GRAD = false>
__global__ void __launch_bounds__(kThreads, 2) k_adaptive(const int* __restrict__ plist, int count,
                                                       Dev dv, const KernelParams kp, double eps,
                                                       double normV, int leaf_order, int max_depth,
                                                       const cplx* __restrict__ I_smooth,
                                                       cplx* __restrict__ I_near,
                                                       int32_t* __restrict__ leaves_out,
                                                       unsigned char* __restrict__ work,
                                                       AdaptiveWS wsd, int* __restrict__ status,
                                                       int* __restrict__ sched, int form,
                                                       GradArgs ga,
                                                       const int64_t* __restrict__ gofs, int gsz) {
  using C = Cfg<D>;
  constexpr int n = C::n;
  // gradient mode: dL/dx_nm of the accepted leaves, per thread, reduced per patch
  double Mg[GRAD ? 3 * n : 1];
  __shared__ cplx shat[GRAD ? n : 1];
  extern __shared__ double smem[];
  double* cf = smem;
  SegMap* segs = reinterpret_cast<SegMap*>(cf + n * 3);
  int* ism = reinterpret_cast<int*>(segs + 4);  // [64]: scan scratch + misc
  unsigned long long* stk = reinterpret_cast<unsigned long long*>(ism + 64);  // [4 * 32]
  // tensor-core moment workspace, 128-byte aligned (ldmatrix needs 16)
  unsigned char* smb = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(stk + 4 * 32) + 127) & ~static_cast<uintptr_t>(127));
  double* ws = reinterpret_cast<double*>(smb);
  // per-block global workspace
  unsigned char* wb = work + (int64_t)blockIdx.x * wsd.stride;
  const int A_max = wsd.A_max;
  cplx* acc = reinterpret_cast<cplx*>(wb);                          // [A_max][n]
  cplx* tmp = acc + (int64_t)A_max * n;                             // [A_max][4][n]
  cplx* lvlI = tmp + (int64_t)A_max * 4 * n;                        // [levels][A_max][4][n]
  int* lvlT = reinterpret_cast<int*>(lvlI + (int64_t)wsd.levels * A_max * 4 * n);  // [levels][A_max]
  int* flags = lvlT + (int64_t)wsd.levels * A_max;                  // [A_max]
  int* lcnt = flags + A_max;                                        // [A_max]
  int* cnt = lcnt + A_max;                                          // [levels]
  double* tmpE = reinterpret_cast<double*>(                          // [A_max][4], 8-aligned
      (reinterpret_cast<uintptr_t>(cnt + wsd.levels) + 7) & ~static_cast<uintptr_t>(7));
  long long my_tests = 0, my_nodes = 0, my_tree = 0;
  __shared__ int next_b, next_g;
  __shared__ KernelParams kps;
  __shared__ double cfd[2 * 3 * (D * (D + 1) / 2)];  // derivative series of the chart
  const double* cfdp = cfd;

  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const int it = atomicAdd(sched, 1);
      int bb = -1, gg = 0;
      if (gofs == nullptr) {
        if (it < count) bb = it;
      } else if (it < gofs[count]) {
        int lo = 0, hi = count;  // gofs[lo] <= it < gofs[hi]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (gofs[mid] <= it) lo = mid;
          else hi = mid;
        }
        bb = lo;
        gg = it - (int)gofs[lo];
      }
      next_b = bb;
      next_g = gg;
    }
    __syncthreads();
    const int b = next_b;
    if (b < 0) break;
    const int j = plist[b];
    const int64_t ap = dv.ad_ptr[j];
    const int Aall = (int)(dv.ad_ptr[j + 1] - ap);
    const int64_t a0 = gofs ? ap + (int64_t)next_g * gsz : ap;
    const int A = gofs ? min(gsz, Aall - next_g * gsz) : Aall;
    if (A <= 0) continue;
    if (A > A_max) {
      if (threadIdx.x == 0) atomicOr(status, kStCapacity);
      continue;
    }
    const int m = leaf_order > 0 ? leaf_order : dv.q[j];
    const int Q = m * m;
    const double* ru = dv.ru + dv.roff[m];
    const double* rv = dv.rv + dv.roff[m];
    const double* rw = dv.rw + dv.roff[m];
    const double tol0 = (dv.pgroup ? dv.grp[dv.pgroup[j]].eps_ad : eps) * dv.dj[j] / normV;
    const int formj = pair_form(dv, j, form);
    const double Rj = dv.rad[j];
    const int32_t* apairs = dv.ad_pair + a0;
    __syncthreads();
    load_coef<D>(dv.coef, dv.node_off[j], cf);
    if (threadIdx.x == 0) kps = patch_kp(dv, j, kp);  // read after block_moments' barrier
    __syncthreads();
    load_coef_derivs<D>(cf, dv.duv[D], cfd);
    if constexpr (GRAD) {
#pragma unroll
      for (int e = 0; e < 3 * n; ++e) Mg[e] = 0.0;
      const cplx* sh = reinterpret_cast<const cplx*>(ga.shat) + dv.node_off[j];
      for (int e = threadIdx.x; e < n; e += blockDim.x) shat[e] = sh[e];
    }
    // root: level 0 block holds all targets with I_T0 in slot c = 0
    for (int e = threadIdx.x; e < A * n; e += blockDim.x) {
      const int i = e / n, nm = e - i * n;
      acc[e] = {0.0, 0.0};
      if (leaf_order <= 0) lvlI[(int64_t)i * 4 * n + nm] = I_smooth[(int64_t)apairs[i] * dv.ldI + nm];
    }
    for (int i = threadIdx.x; i < A; i += blockDim.x) {
      lvlT[i] = i;
      lcnt[i] = 0;
    }
    if (threadIdx.x == 0) {
      segs[0] = seg_T0();
      cnt[0] = A;
    }
    __syncthreads();
    if (leaf_order > 0) {
      TgtPairIdx ta{dv.tgt, dv.NT, dv.pair_tgt, apairs, dv.tnrm};
      block_moments_any<D>(cf, cfdp, ru, rv, rw, Q, segs, 1, ta, A,
                           [=] __device__(int i) { return lvlI + (int64_t)i * 4 * n; }, kps, smb,
                           dv.cen + 3 * j, Rj, tmpE, formj);
    }
    // DFS stack entries: level (8 bits) | child (2 bits) | path (2 bits per level) << 16
    int sp = 0;
    if (threadIdx.x == 0) stk[0] = 0ull;  // root: level 0, child 0, empty path
    sp = 1;
    int visited = 0;
    while (sp > 0) {
      if (++visited > kMaxTreeNodes) {  // bounded walk: give up on this patch
        if (threadIdx.x == 0) atomicOr(status, kStCapacity);
        break;
      }
      __syncthreads();
      const unsigned long long top = stk[sp - 1];
      --sp;
      const int L = (int)(top & 0xff);
      const int cidx = (int)((top >> 8) & 3);
      const unsigned long long path = top >> 16;  // child digits of T, level 1 at bits 0-1
      const int S = cnt[L];
      const int* ST = lvlT + (int64_t)L * A_max;
      const cplx* IT = lvlI + (int64_t)L * A_max * 4 * n;
      if ((threadIdx.x & 31) == 0 && threadIdx.x < 128) {
        // Every subtriangle of the midpoint tree is T0 scaled by 2^-L, translated and
        // possibly point-reflected: vertex a at (ia, ja) 2^-L, b = a + o (2^-L, 0),
        // c = a + o (0, 2^-L).  The walk down the path runs in integers; the first lane of
        // warp k writes the map of child k (all exact dyadic values).
        const int k = threadIdx.x >> 5;
        long long ia = 0, ja = 0;
        int o = 1;
        for (int l = 0; l < L; ++l) {
          const int dgt = (int)((path >> (2 * l)) & 3);
          ia = 2 * ia + ((dgt & 1) ? o : 0);
          ja = 2 * ja + ((dgt & 2) ? o : 0);
          if (dgt == 3) o = -o;
        }
        const double h = ldexp(1.0, -(L + 1));
        const int ok = k == 3 ? -o : o;
        SegMap sm;
        sm.ax = (double)(2 * ia + ((k & 1) ? o : 0)) * h;
        sm.ay = (double)(2 * ja + ((k & 2) ? o : 0)) * h;
        sm.e1x = ok * h;
        sm.e1y = 0.0;
        sm.e2x = 0.0;
        sm.e2y = ok * h;
        sm.det = h * h;
        segs[k] = sm;
      }
      __syncthreads();
      // children moments of every target in S
      TgtAdaptive ta{dv.tgt, dv.NT, dv.pair_tgt, apairs, ST, dv.tnrm};
      block_moments_any<D>(cf, cfdp, ru, rv, rw, Q, segs, 4, ta, S,
                           [=] __device__(int i) { return tmp + (int64_t)i * 4 * n; }, kps, smb,
                           dv.cen + 3 * j, Rj, tmpE, formj);
      __syncthreads();
      my_tests += S;
      my_nodes += (long long)S * 4 * Q;
      my_tree += 1;
      // decisions: one warp per target
      const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      const double tauL = tol0 * ldexp(1.0, -2 * L);
      for (int s = w; s < S; s += nw) {
        double e2 = 0.0;
        for (int nm = lane; nm < n; nm += 32) {
          const cplx* tc = tmp + (int64_t)s * 4 * n + nm;
          const double sr = tc[0].re + tc[n].re + tc[2 * n].re + tc[3 * n].re;
          const double si = tc[0].im + tc[n].im + tc[2 * n].im + tc[3 * n].im;
          const cplx it = IT[(int64_t)s * 4 * n + (int64_t)cidx * n + nm];
          const double dr = it.re - sr, di = it.im - si;
          e2 += dr * dr + di * di;
        }
        e2 = warp_sum(e2);
        const double err = sqrt(e2);
        const double* ee = tmpE + (int64_t)s * 4;
        const double tau = fmax(tauL, kRoundingFloor * (ee[0] + ee[1] + ee[2] + ee[3]));
        const bool finite = isfinite(err) && isfinite(tau);
        const bool accept = !finite || (err <= tau) || (L + 1 >= max_depth);
        if (lane == 0) {
          if (!finite) atomicOr(status, kStNonFinite);
          else if (err > tau && accept) atomicOr(status, kStMaxDepth);
        }
        const int tl = ST[s];
        if (accept) {
          for (int nm = lane; nm < n; nm += 32) {
            const cplx* tc = tmp + (int64_t)s * 4 * n + nm;
            cplx& a = acc[(int64_t)tl * n + nm];
            a.re += tc[0].re + tc[n].re + tc[2 * n].re + tc[3 * n].re;
            a.im += tc[0].im + tc[n].im + tc[2 * n].im + tc[3 * n].im;
          }
          if (lane == 0) lcnt[tl] += 4;
        }
        if (lane == 0) flags[s] = accept ? 0 : 1;
      }
      __syncthreads();
      if constexpr (GRAD) {
        // kernel gradients on the accepted children (the tree itself is recomputed, not
        // stored): weight conj(g_t) for a target that accepts here, else 0
        const cplx* gt = reinterpret_cast<const cplx*>(ga.g);
        block_grad<D>(cf, ru, rv, rw, Q, segs, 4, ta, S,
                      [&](int i) -> cplx {
                        if (flags[i] != 0) return {0.0, 0.0};
                        const cplx c = gt[dv.pair_tgt[apairs[ST[i]]]];
                        return {c.re, -c.im};
                      },
                      kps, shat, dv.cen + 3 * j, Mg);
      }
      // stable compaction of the refining targets into level L+1
      int base = 0;
      int* DT = lvlT + (int64_t)(L + 1) * A_max;
      cplx* DI = lvlI + (int64_t)(L + 1) * A_max * 4 * n;
      for (int s0 = 0; s0 < S; s0 += blockDim.x) {
        const int s = s0 + threadIdx.x;
        const int f = s < S ? flags[s] : 0;
        int tot;
        const int pos = block_flag_scan(f, ism, &tot);
        if (f) {
          flags[s] = -(base + pos) - 1;  // remember destination
          DT[base + pos] = ST[s];
        }
        base += tot;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < S * 4 * n; e += blockDim.x) {
        const int s = e / (4 * n);
        const int f = flags[s];
        if (f < 0) DI[(int64_t)(-f - 1) * 4 * n + (e - s * 4 * n)] = tmp[e];
      }
      if (threadIdx.x == 0) cnt[L + 1] = base;
      __syncthreads();
      if (base > 0) {
        if (sp + 4 > 4 * 32) {
          if (threadIdx.x == 0) atomicOr(status, kStCapacity);
        } else {
          const unsigned long long np = (L == 0) ? 0ull : path;
          if (threadIdx.x == 0) {
            for (int c = 3; c >= 0; --c)
              stk[sp + (3 - c)] = (unsigned long long)(L + 1) | ((unsigned long long)c << 8) |
                                  ((np | ((unsigned long long)c << (2 * L))) << 16);
          }
          sp += 4;
        }
      }
      (void)cidx;
    }
    __syncthreads();
    // results of the patch
    for (int e = threadIdx.x; e < A * n; e += blockDim.x) {
      const int i = e / n, nm = e - i * n;
      I_near[(int64_t)apairs[i] * dv.ldI + nm] = acc[e];
    }
    for (int i = threadIdx.x; i < A; i += blockDim.x) leaves_out[apairs[i]] = lcnt[i];
    if constexpr (GRAD) block_reduce_M<D>(Mg, ws, ga.M + dv.node_off[j] * 3);
  }
  if (threadIdx.x == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(dv.counters + 0), (unsigned long long)my_tests);
    atomicAdd(reinterpret_cast<unsigned long long*>(dv.counters + 1), (unsigned long long)my_nodes);
    atomicAdd(reinterpret_cast<unsigned long long*>(dv.counters + 4), (unsigned long long)my_tree);
  }
}

}  // namespace lcq
