// Cluster tree for callers that cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc: code that runs inside
// another runtime which has reserved the device memory up front (a serving
// process with a fixed arena), code on a path where an allocation, which can
// synchronise the device, is not allowed, or code whose memory is partitioned
// at start-up.  cqm_cluster_tree_noalloc gives them the cluster tree of a mesh
// that is already on the device, writing into buffers they own, with the
// kernel's scratch taken from a fixed array that this file reserves on every
// GPU that loads the library (held until the process exits).
#include <mutex>
#include <string>

#include "handle.cuh"

namespace cqm {

constexpr int kTreeNoallocMax = CQM_TREE_NOALLOC_MAX_TRIANGLES;

// Scratch layout: centroids (3 M doubles), partition buffer (M ints),
// per-node split counts (2 M ints), counters (4 ints).
constexpr size_t kCenBytes = sizeof(double) * 3 * (size_t)kTreeNoallocMax;
constexpr size_t kTmpBytes = sizeof(int) * (size_t)kTreeNoallocMax;
constexpr size_t kSplitBytes = sizeof(int) * 2 * (size_t)kTreeNoallocMax;
constexpr size_t kCounterBytes = 256;
constexpr size_t kScratchBytes = kCenBytes + kTmpBytes + kSplitBytes + kCounterBytes;

static __device__ __align__(256) unsigned char g_tree_scratch[kScratchBytes];

// Device address of the scratch array on the current device, looked up once
// per device (the array's name is not a device address in host code).
static std::mutex g_scratch_mu;
static void* g_scratch_addr[128] = {};

static int scratch_on_current_device(unsigned char** out) {
  int dev = 0;
  CQM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) {
    set_last_error("device ordinal out of range");
    return CQM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_tree_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error(std::string("cudaGetSymbolAddress(tree scratch): ") + cudaGetErrorString(e));
      return CQM_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return CQM_OK;
}

// Centroids ((P0 + P1) + P2) / 3, as in the geometry kernel; flags vertex
// indices outside [0, nv) instead of reading through them.
__global__ void k_noalloc_centroids(int M, int nv, const double* __restrict__ xyz,
                                    const int* __restrict__ tri, double* cen, int* counters) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M) return;
  int v[3];
  for (int k = 0; k < 3; ++k) {
    v[k] = tri[3 * t + k];
    if (v[k] < 0 || v[k] >= nv) {
      atomicOr(&counters[2], 1);
      return;
    }
  }
  for (int d = 0; d < 3; ++d)
    cen[3 * t + d] = __ddiv_rn(__dadd_rn(__dadd_rn(xyz[3 * v[0] + d], xyz[3 * v[1] + d]),
                                         xyz[3 * v[2] + d]), 3.0);
}

}  // namespace cqm

using namespace cqm;

extern "C" int cqm_cluster_tree_noalloc(const double* xyz, int32_t nv, const int32_t* tri,
                                        int32_t nt, int32_t n_min, int32_t* perm, int32_t* begin,
                                        int32_t* end, int32_t* son0, int32_t* son1,
                                        int32_t* parent, int32_t* level, double* lo, double* hi,
                                        int32_t* n_nodes, void* cuda_stream) {
  set_last_error("");
  if (!xyz || !tri || !perm || !begin || !end || !son0 || !son1 || !parent || !level || !lo ||
      !hi || !n_nodes) {
    set_last_error("cqm_cluster_tree_noalloc: NULL argument");
    return CQM_EINVAL;
  }
  if (nt < 1 || nv < 3 || n_min < 1) {
    set_last_error("cqm_cluster_tree_noalloc: need nt >= 1, nv >= 3, n_min >= 1");
    return CQM_EINVAL;
  }
  if (nt > kTreeNoallocMax) {
    set_last_error("cqm_cluster_tree_noalloc: " + std::to_string(nt) +
                   " triangles exceed the fixed scratch of " + std::to_string(kTreeNoallocMax));
    return CQM_EINVAL;
  }
  unsigned char* base = nullptr;
  CQM_TRY(scratch_on_current_device(&base));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* cen = (double*)base;
  int* tmp = (int*)(base + kCenBytes);
  int* split = (int*)(base + kCenBytes + kTmpBytes);
  int* counters = (int*)(base + kCenBytes + kTmpBytes + kSplitBytes);
  // the array keeps the previous call's contents: clear the counters
  CQM_CUDA_TRY(cudaMemsetAsync(counters, 0, kCounterBytes, s));
  k_noalloc_centroids<<<grid_for(nt, 256), 256, 0, s>>>(nt, nv, xyz, tri, cen, counters);
  CQM_CHECK_LAUNCH();
  int hc[4] = {0, 0, 0, 0};
  CQM_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, s));
  CQM_CUDA_TRY(cudaStreamSynchronize(s));
  if (hc[2]) {
    set_last_error("cqm_cluster_tree_noalloc: vertex index out of range");
    return CQM_EINVAL;
  }
  const int cap = 2 * nt - 1;
  CQM_TRY(launch_tree_kernel(nt, n_min, cap, xyz, tri, cen, perm, tmp, begin, end, son0, son1,
                             parent, level, lo, hi, split, counters, s));
  CQM_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, s));
  CQM_CUDA_TRY(cudaStreamSynchronize(s));
  *n_nodes = hc[0];
  return CQM_OK;
}
