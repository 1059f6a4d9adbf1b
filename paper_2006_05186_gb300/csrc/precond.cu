// Block-diagonal (leaf) preconditioner for the batched GMRES.  The paper
// suggests replacing the direct solver by an iterative one with a
// preconditioner (Sec. 6.2, before Table 1); the preconditioner is the inverse
// of the near-field diagonal blocks V_l[r, r] of every leaf cluster r, built
// from their MACA factors (eq. lrfinal) for every solved frequency and
// applied as right preconditioning, so that GMRES still minimises the true
// residual ghat_l - V_l qhat_l.
// Layout: P[leaf k][i][j][l] (frequency fastest) for coalesced application.
#include <algorithm>
#include <vector>

#include "handle.cuh"

namespace cqm {

constexpr int PB = 32;  // maximum leaf size

// One block per (leaf k, frequency l): B = sum_t D[t][l] C_t, Gauss-Jordan
// inversion with partial pivoting in shared memory.
__global__ void __launch_bounds__(256) k_precond_build(int Ls, int cap, const int* __restrict__ leaves,
                                                       const int* __restrict__ diag_block,
                                                       const int* __restrict__ begin,
                                                       const int* __restrict__ end,
                                                       const int* __restrict__ rank,
                                                       const int64_t* __restrict__ off,
                                                       const double2* __restrict__ Cn,
                                                       const double2* __restrict__ Dn,
                                                       double2* __restrict__ P, int* flag) {
  __shared__ double2 A[PB][2 * PB + 1];
  __shared__ int s_piv;
  const int k = blockIdx.x, l = blockIdx.y;
  const int r = leaves[k];
  const int n = end[r] - begin[r];
  const int b = diag_block[k];
  const int rk = rank[b];
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    double2 v = make_double2(0.0, 0.0);
    for (int t = 0; t < rk; ++t) cfma(v, Cn[off[b] + (size_t)t * n * n + e], Dn[((size_t)b * cap + t) * Ls + l]);
    A[i][j] = v;
    A[i][n + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = c;
      for (int i = c + threadIdx.x; i < n; i += 32) {
        const double a = cabs2(A[i][c]);
        if (a > best) { best = a; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        s_piv = bi;
        if (!(best > 0.0)) atomicOr(flag, 1);
      }
    }
    __syncthreads();
    const int pr = s_piv;
    if (pr != c)
      for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) {
        const double2 t = A[c][j];
        A[c][j] = A[pr][j];
        A[pr][j] = t;
      }
    __syncthreads();
    const double2 pv = A[c][c];
    const double2 inv = cdiv(make_double2(1.0, 0.0), pv);
    __syncthreads();
    for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) A[c][j] = cmul(A[c][j], inv);
    __syncthreads();
    for (int e = threadIdx.x; e < n * 2 * n; e += blockDim.x) {
      const int i = e / (2 * n), j = e - i * 2 * n;
      if (i != c) {
        const double2 f = A[i][c];
        if (j != c) A[i][j] = csub(A[i][j], cmul(f, A[c][j]));
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (i != c) A[i][c] = make_double2(0.0, 0.0);
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    P[(((size_t)k * PB + i) * PB + j) * Ls + l] = A[i][n + j];
  }
}

// z[l][perm[rb + i]] = sum_j P[k][i][j][l] v[l][perm[rb + j]]
__global__ void __launch_bounds__(256) k_precond_apply(int M, int Ls, const int* __restrict__ leaves,
                                                       const int* __restrict__ begin,
                                                       const int* __restrict__ end,
                                                       const int* __restrict__ perm,
                                                       const double2* __restrict__ P,
                                                       const double2* __restrict__ v,
                                                       double2* __restrict__ z,
                                                       const int* __restrict__ act) {
  __shared__ double2 vs[PB][32];
  const int k = blockIdx.x;
  const int r = leaves[k];
  const int rb = begin[r], n = end[r] - rb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int l = blockIdx.y * 32 + lane;
  // act (may be null): frequencies still iterating; the others are skipped
  const bool on = l < Ls && (!act || act[l]);
  if (!__syncthreads_or(on)) return;
  for (int j = w; j < n; j += 8) vs[j][lane] = on ? v[(size_t)l * M + perm[rb + j]] : make_double2(0.0, 0.0);
  __syncthreads();
  if (!on) return;
  for (int i = w; i < n; i += 8) {
    double2 acc = make_double2(0.0, 0.0);
    const double2* Pi = P + ((size_t)k * PB + i) * PB * Ls + l;
    for (int j = 0; j < n; ++j) cfma(acc, Pi[(size_t)j * Ls], vs[j][lane]);
    z[(size_t)l * M + perm[rb + i]] = acc;
  }
}

int build_precond(cqm_handle* h) {
  const int nl = (int)h->h_leaves.size();
  std::vector<int> diag(nl, -1);
  for (int k = 0; k < nl; ++k) {
    const int r = h->h_leaves[k];
    for (int b = 0; b < h->n_near; ++b)
      if (h->h_near[b].x == r && h->h_near[b].y == r) { diag[k] = b; break; }
    if (diag[k] < 0) {
      set_last_error("leaf without a diagonal near block");
      return CQM_EINVAL;
    }
  }
  CQM_TRY(h->Pinv.allocate(h->alloc, (size_t)nl * PB * PB * h->Ls));
  DArray<int> d_diag;
  CQM_TRY(d_diag.allocate(h->alloc, nl));
  CQM_CUDA_TRY(cudaMemcpyAsync(d_diag.p, diag.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, h->stream));
  CQM_CUDA_TRY(cudaMemsetAsync(h->flag.p, 0, sizeof(int), h->stream));
  {
    ProfScope ps_(h, CQM_K_PRECOND);
    k_precond_build<<<dim3(nl, h->Ls), 256, 0, h->stream>>>(
        h->Ls, h->rank_cap, h->d_leaves.p, d_diag.p, h->node_begin.p, h->node_end.p, h->near_rank.p,
        h->near_off.p, h->nearC.p, h->nearD.p, h->Pinv.p, h->flag.p);
  }
  cudaError_t e = cudaGetLastError();
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, h->flag.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  d_diag.free(h->alloc);
  if (e != cudaSuccess) {
    set_last_error(std::string("precond: ") + cudaGetErrorString(e));
    return CQM_ECUDA;
  }
  if (flag) {
    set_last_error("singular diagonal block in the preconditioner");
    return CQM_EINVAL;
  }
  h->use_precond = true;
  return CQM_OK;
}

int apply_precond(cqm_handle* h, const double2* v, double2* z, const int* act) {
  const int nl = (int)h->h_leaves.size();
  {
    ProfScope ps_(h, CQM_K_PRECOND);
    k_precond_apply<<<dim3(nl, (h->Ls + 31) / 32), 256, 0, h->stream>>>(
        h->M, h->Ls, h->d_leaves.p, h->node_begin.p, h->node_end.p, h->perm.p, h->Pinv.p, v, z, act);
  }
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

}  // namespace cqm
