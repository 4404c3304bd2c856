// Pipe-throughput microbenchmarks: the measured denominators of the roofline fractions the
// benchmark reports (FP64 FMA for the FP64 correction kernels, FP32 FMA and the special
// function unit for the mixed form, the integer pipe and the warp-level tensor-core MMA
// forms for split-precision contractions).  No counterpart in the paper.
//
// Every kernel runs U independent dependency chains per thread over a grid of 4 blocks of
// 256 threads per SM, long enough (about 20 ms, calibrated by a first short run) for the
// launch overhead to vanish; time by CUDA events on a private stream.  Operands are runtime
// values so nothing folds; one result per block is stored behind a never-true test so the
// chains stay live.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lcq.h"

namespace lcq {
namespace {

constexpr int kPeakThreads = 256;

// FP64 FMA chains (the FP64 pipe's peak).
template <int U>
__global__ void k_peak_dfma(double* sink, int iters, double a, double b) {
  double x[U];
#pragma unroll
  for (int i = 0; i < U; ++i) x[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < U; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < U; ++i) s += x[i];
  if (s == -1.2345) sink[blockIdx.x] = s;
}

// FP32 FMA chains (the FP32 pipe's peak).
template <int U>
__global__ void k_peak_ffma(float* sink, int iters, float a, float b) {
  float x[U];
#pragma unroll
  for (int i = 0; i < U; ++i) x[i] = threadIdx.x * 1e-3f + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < U; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < U; ++i) s += x[i];
  if (s == -1.2345f) sink[blockIdx.x] = s;
}

// special function unit: sin.approx.f32 chains
template <int U>
__global__ void k_peak_mufu(float* sink, int iters, float a) {
  float x[U];
#pragma unroll
  for (int i = 0; i < U; ++i) x[i] = threadIdx.x * 1e-3f + i * a;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < U; ++i) asm volatile("sin.approx.f32 %0, %0;" : "+f"(x[i]));
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < U; ++i) s += x[i];
  if (s == -1.2345f) sink[blockIdx.x] = s;
}

// integer pipe: xor-add chains (LOP3 / IADD3)
template <int U>
__global__ void k_peak_int(unsigned* sink, int iters, unsigned a, unsigned b) {
  unsigned x[U];
#pragma unroll
  for (int i = 0; i < U; ++i) x[i] = threadIdx.x * 7u + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < U; ++i) x[i] = (x[i] ^ a) + b;
  }
  unsigned s = 0;
#pragma unroll
  for (int i = 0; i < U; ++i) s += x[i];
  if (s == 0x9e3779b9u) sink[blockIdx.x] = s;
}

// mma.sync m8n8k4 f64: 512 FLOP per warp instruction
template <int U>
__global__ void k_peak_dmma(double* sink, int iters, double a, double b) {
  double c0[U], c1[U];
#pragma unroll
  for (int i = 0; i < U; ++i) c0[i] = c1[i] = 1e-3 * i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < U; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c0[i]), "+d"(c1[i])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < U; ++i) s += c0[i] + c1[i];
  if (s == -1.2345) sink[blockIdx.x] = s;
}

// mma.sync m16n8k16 f16 or bf16 inputs, f32 accumulators: 4096 FLOP per warp instruction
template <int U, bool BF16>
__global__ void k_peak_hmma(float* sink, int iters, unsigned a, unsigned b) {
  float c[U][4];
#pragma unroll
  for (int i = 0; i < U; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.0f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < U; ++i) {
      if (BF16)
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
            "{%8,%9}, {%0,%1,%2,%3};"
            : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
            : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
      else
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
            "{%8,%9}, {%0,%1,%2,%3};"
            : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
            : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < U; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  if (s == -1.2345f) sink[blockIdx.x] = s;
}

// mma.sync m16n8k8 tf32 inputs, f32 accumulators: 2048 FLOP per warp instruction
template <int U>
__global__ void k_peak_tf32(float* sink, int iters, unsigned a, unsigned b) {
  float c[U][4];
#pragma unroll
  for (int i = 0; i < U; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.0f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < U; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
          "{%8,%9}, {%0,%1,%2,%3};"
          : "+f"(c[i][0]), "+f"(c[i][1]), "+f"(c[i][2]), "+f"(c[i][3])
          : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < U; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  if (s == -1.2345f) sink[blockIdx.x] = s;
}

// Runs launch(iters) once short to calibrate, then for about 20 ms; returns units/s with
// `units` counted per (thread, iteration) of the whole grid (or < 0 on a CUDA error).
template <class L>
double time_rate(cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int grid, double units_per_thread_iter,
                 L launch) {
  int iters = 256;
  float ms = 0.0f;
  for (int pass = 0; pass < 3; ++pass) {
    if (cudaEventRecord(e0, st) != cudaSuccess) return -1.0;
    launch(iters);
    if (cudaEventRecord(e1, st) != cudaSuccess) return -1.0;
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0;
    if (pass < 2) {
      const double scale = ms > 0.0f ? 20.0 / ms : 64.0;
      double next = iters * (scale > 64.0 ? 64.0 : scale);
      if (next > 2.0e8) next = 2.0e8;
      if (next < 16) next = 16;
      iters = (int)next;
    }
  }
  const double units = (double)grid * kPeakThreads * (double)iters * units_per_thread_iter;
  return units / (ms * 1e-3);
}

}  // namespace
}  // namespace lcq

using namespace lcq;

extern "C" lcq_status lcq_pipe_peaks(int device, double* out, int n_out) {
  if (!out || n_out < 1) return LCQ_ERR_ARG;
  for (int i = 0; i < n_out; ++i) out[i] = 0.0;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return LCQ_ERR_CUDA;
  }
  int sms = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* sink = nullptr;
  lcq_status status = LCQ_OK;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMalloc(&sink, 4096 * 8) != cudaSuccess) {
    status = LCQ_ERR_CUDA;
  }
  if (status == LCQ_OK) {
    const int grid = sms * 4;
    double* sd = static_cast<double*>(sink);
    float* sf = static_cast<float*>(sink);
    unsigned* su = static_cast<unsigned*>(sink);
    const unsigned h2 = 0x3c003c00u;   // two f16 ones
    const unsigned b2 = 0x3f803f80u;   // two bf16 ones
    const unsigned t1 = 0x3f800000u;   // tf32 one
    // [0] FP64 FMA TFLOP/s  [1] FP32 FMA TFLOP/s  [2] MUFU sin Top/s  [3] INT32 xor+add Top/s
    // [4] f64 mma.sync TFLOP/s  [5] f16 mma.sync TFLOP/s  [6] bf16 mma.sync TFLOP/s
    // [7] tf32 mma.sync TFLOP/s
    double r[8];
    r[0] = time_rate(st, e0, e1, grid, 2.0 * 8, [&](int it) {
      k_peak_dfma<8><<<grid, kPeakThreads, 0, st>>>(sd, it, 0.999999, 1e-7);
    });
    r[1] = time_rate(st, e0, e1, grid, 2.0 * 8, [&](int it) {
      k_peak_ffma<8><<<grid, kPeakThreads, 0, st>>>(sf, it, 0.999999f, 1e-7f);
    });
    r[2] = time_rate(st, e0, e1, grid, 8, [&](int it) {
      k_peak_mufu<8><<<grid, kPeakThreads, 0, st>>>(sf, it, 0.25f);
    });
    r[3] = time_rate(st, e0, e1, grid, 2.0 * 8, [&](int it) {
      k_peak_int<8><<<grid, kPeakThreads, 0, st>>>(su, it, 0x5bd1e995u, 0x27d4eb2fu);
    });
    // MMA forms: per thread and iteration U warp instructions / 32 threads
    r[4] = time_rate(st, e0, e1, grid, 4 * 512.0 / 32, [&](int it) {
      k_peak_dmma<4><<<grid, kPeakThreads, 0, st>>>(sd, it, 1.0, 1e-9);
    });
    r[5] = time_rate(st, e0, e1, grid, 4 * 4096.0 / 32, [&](int it) {
      k_peak_hmma<4, false><<<grid, kPeakThreads, 0, st>>>(sf, it, h2, 0u);
    });
    r[6] = time_rate(st, e0, e1, grid, 4 * 4096.0 / 32, [&](int it) {
      k_peak_hmma<4, true><<<grid, kPeakThreads, 0, st>>>(sf, it, b2, 0u);
    });
    r[7] = time_rate(st, e0, e1, grid, 4 * 2048.0 / 32, [&](int it) {
      k_peak_tf32<4><<<grid, kPeakThreads, 0, st>>>(sf, it, t1, 0u);
    });
    for (int i = 0; i < 8 && i < n_out; ++i) {
      if (r[i] < 0.0) status = LCQ_ERR_CUDA;
      out[i] = r[i] > 0.0 ? r[i] * 1e-12 : 0.0;
    }
  }
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaGetLastError();
  cudaSetDevice(prev);
  return status;
}
