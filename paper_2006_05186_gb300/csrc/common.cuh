// Shared device/host helpers of libcqmbem: complex arithmetic on double2,
// warp and block reductions, status plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "cqm_bem.h"

namespace cqm {

// ---------------------------------------------------------------- status ----
void set_last_error(const std::string& msg);

struct Status {
  int code = CQM_OK;
  bool ok() const { return code == CQM_OK; }
};

#define CQM_CUDA_TRY(expr)                                                        \
  do {                                                                            \
    cudaError_t _e = (expr);                                                      \
    if (_e != cudaSuccess) {                                                      \
      ::cqm::set_last_error(std::string(#expr) + ": " + cudaGetErrorString(_e) +  \
                            " (" + __FILE__ + ":" + std::to_string(__LINE__) + ")"); \
      return (_e == cudaErrorMemoryAllocation) ? CQM_ENOMEM : CQM_ECUDA;          \
    }                                                                             \
  } while (0)

#define CQM_TRY(expr)                 \
  do {                                \
    int _s = (expr);                  \
    if (_s != CQM_OK) return _s;      \
  } while (0)

#define CQM_CHECK_LAUNCH() CQM_CUDA_TRY(cudaGetLastError())

// --------------------------------------------------------------- complex ----
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) {
  return make_double2(a.x * s, a.y * s);
}
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
// a += b * c
__device__ __forceinline__ void cfma(double2& a, double2 b, double2 c) {
  a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
  a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}

// float2 versions (storage and arithmetic of the FP32 inner operator)
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ void cfma(float2& a, float2 b, float2 c) {
  a.x = fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x));
  a.y = fmaf(b.x, c.y, fmaf(b.y, c.x, a.y));
}

// Complex type of a real type.
template <class R> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };

template <class T> __device__ __forceinline__ T cz();
template <> __device__ __forceinline__ double2 cz<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 cz<float2>() { return make_float2(0.f, 0.f); }

__device__ __forceinline__ double2 to_c(double2 v, double2*) { return v; }
__device__ __forceinline__ float2 to_c(double2 v, float2*) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_d(double2 v) { return v; }
__device__ __forceinline__ double2 to_d(float2 v) { return make_double2(v.x, v.y); }

// ------------------------------------------------------------ reductions ----
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 warp_sum2(double2 v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}

// Block-wide sum; `sh` holds at least 32 doubles. Result valid in all threads.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (warp == 0) {
    t = warp_sum(t);
    if (lane == 0) sh[0] = t;
  }
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------- allocator ----
struct Allocator {
  const cqm_allocator* user = nullptr;
  cudaStream_t stream = nullptr;
  int64_t bytes_held = 0;

  int alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return CQM_OK;
    bytes = (bytes + 255) & ~size_t(255);
    if (user && user->alloc) {
      *p = user->alloc(bytes, (void*)stream, user->ctx);
      if (!*p) {
        set_last_error("allocator callback failed for " + std::to_string(bytes) + " bytes");
        return CQM_ENOMEM;
      }
    } else {
      cudaError_t e = cudaMallocAsync(p, bytes, stream);
      if (e != cudaSuccess) {
        cudaGetLastError();
        set_last_error(std::string("cudaMallocAsync: ") + cudaGetErrorString(e) + " (" +
                       std::to_string(bytes) + " bytes)");
        return e == cudaErrorMemoryAllocation ? CQM_ENOMEM : CQM_ECUDA;
      }
    }
    bytes_held += (int64_t)bytes;
    return CQM_OK;
  }
  void release(void* p, size_t bytes) {
    if (!p) return;
    bytes = (bytes + 255) & ~size_t(255);
    if (user && user->free) user->free(p, bytes, (void*)stream, user->ctx);
    else cudaFreeAsync(p, stream);
    bytes_held -= (int64_t)bytes;
  }
};

// A typed device array owned by a handle.
template <class T>
struct DArray {
  T* p = nullptr;
  size_t n = 0;
  int allocate(Allocator& a, size_t count) {
    free(a);
    n = count;
    void* q = nullptr;
    int s = a.alloc(&q, count * sizeof(T));
    p = (T*)q;
    if (s != CQM_OK) n = 0;
    return s;
  }
  void free(Allocator& a) {
    if (p) a.release(p, n * sizeof(T));
    p = nullptr;
    n = 0;
  }
};

inline int grid_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace cqm
