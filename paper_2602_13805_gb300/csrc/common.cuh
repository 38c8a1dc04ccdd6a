// Shared device helpers: complex arithmetic on float2/double2, block reductions,
// the FFT plan description, and launch-error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pdf.h"

#define PDF_MAX_RADICES 16
#define PDF_MAX_P 512           // largest padded FFT length (2 * 256)

// ---------------------------------------------------------------------------
// programmatic dependent launch: the solve loop's kernels are launched with programmatic stream
// serialisation and start with pdl_wait(), which returns once the previous kernel in the stream has
// completed and its memory is visible (a no-op under a plain launch).  No kernel triggers its
// dependents early, so a dependent grid is scheduled only after every block of the previous one has
// exited; what the attribute saves is the launch latency between consecutive kernels.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... P, typename... A>
static inline void launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename T> struct cvec;
template <> struct cvec<float> { typedef float2 type; };
template <> struct cvec<double> { typedef double2 type; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// acc + a b and acc + a conj(b) as four FMAs: the accumulation is fused into the products (a plain
// acc + cmul(a, b) costs two multiplies, two FMAs and two adds)
__host__ __device__ __forceinline__ float2 cmac(float2 acc, float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
__host__ __device__ __forceinline__ float2 cmacc(float2 acc, float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.y, b.x, fmaf(-a.x, b.y, acc.y)));
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ float2 to_f(double2 a) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__host__ __device__ __forceinline__ float2 cdivf(float2 a, float2 b) {
  float d = b.x * b.x + b.y * b.y;
  return make_float2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// ---------------------------------------------------------------------------
// reductions (double accumulation).  blockDim.x must be a multiple of 32, <= 1024.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; result valid in thread 0.  `scratch` needs 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  double r = 0.0;
  if (wid == 0) {
    r = lane < nw ? scratch[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// ---------------------------------------------------------------------------
// float-float ("double-single") accumulation: value = hi + lo with |lo| <= ulp(hi)/2, built from
// error-free TwoSum steps.  Carries ~44 significant bits at FP32 speed; used instead of FP64,
// whose throughput and latency on this part make even small FP64 reductions dominate a kernel.
// ---------------------------------------------------------------------------
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_make(float a) { return FF{a, 0.f}; }
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float hi = s + e;
  return FF{hi, e - (hi - s)};
}
__device__ __forceinline__ FF ff_add(FF a, float b) { return ff_add(a, FF{b, 0.f}); }
__device__ __forceinline__ double ff_to_d(FF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ FF ff_shfl_xor(FF a, int m) {
  return FF{__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
}
__device__ __forceinline__ FF ff_warp_sum(FF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = ff_add(v, ff_shfl_xor(v, o));
  return v;
}
// Sum over the block; valid in thread 0.  `scratch` needs 32 FF of shared memory.
__device__ __forceinline__ FF ff_block_sum(FF v, FF* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = ff_warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  FF r = FF{0.f, 0.f};
  if (wid == 0) {
    r = lane < nw ? scratch[lane] : FF{0.f, 0.f};
    r = ff_warp_sum(r);
  }
  return r;
}

// N sums over the block in one pass (valid in thread 0).  `scratch` needs 32 N FF of shared memory.
template <int N>
__device__ __forceinline__ void ff_block_sum_multi(FF (&v)[N], FF* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int s = 0; s < N; ++s) v[s] = ff_add(v[s], ff_shfl_xor(v[s], o));
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int s = 0; s < N; ++s) scratch[s * 32 + wid] = v[s];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int s = 0; s < N; ++s) v[s] = lane < nw ? scratch[s * 32 + lane] : FF{0.f, 0.f};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int s = 0; s < N; ++s) v[s] = ff_add(v[s], ff_shfl_xor(v[s], o));
  }
}

// ---------------------------------------------------------------------------
// FFT plan: P = product of radices (each 2, 3 or 4), Stockham ordering
// ---------------------------------------------------------------------------
struct FFTPlan {
  int P;
  int nst;
  int radix[PDF_MAX_RADICES];
};

// host-side launch accounting
extern "C++" void pdf_count_launch(uint64_t n);
