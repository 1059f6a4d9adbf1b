// Batched restarted GMRES over the solved CQM frequencies: for every l < Ls,
// V_l qhat_l = ghat_l (Remark in Sec. 6.2; the paper factorises instead and
// names iterative solvers as the way to avoid the O(M^2) factorisation).
// All frequencies advance in lockstep; a frequency whose residual estimate
// meets the tolerance stops contributing to the cycle, and every restart
// recomputes the true FP64 residual b - V x.
// Orthogonalisation: classical Gram-Schmidt applied twice (CGS2).
// Layouts: vectors Ls x M complex (row l); basis (m+1) x Ls x M.
#include <algorithm>
#include <vector>

#include "handle.cuh"

namespace cqm {

struct GmresWork {
  int m = 0;
  DArray<double2> Vb, r, H, sn, g, y, Z, p1, p2;  // p1, p2: partial dot products
  DArray<double> cs, bnorm, beta, thr, nrm;
  DArray<int> active, kdim, converged, counters, need;
  DArray<unsigned long long> work;  // [0] basis vectors, [1] frequency steps of the Arnoldi steps
  int* h_counters = nullptr;  // pinned
};

// r = b - y (y = V x) or r = b when y == nullptr; beta_l = ||r_l||,
// bnorm_l = ||b_l|| on the first call; sets active/converged, v0 = r/beta,
// g = (beta, 0, ...).
__global__ void k_restart(int M, int m, const double2* __restrict__ b, const double2* y,
                          double2* __restrict__ r, double2* __restrict__ V0, double* bnorm,
                          double* beta, int* active, int* converged, double2* g, double tol,
                          double rtol, double* thr, int first, int* counters) {
  __shared__ double sh[32];
  const int l = blockIdx.x;
  // converged at an earlier restart: the solution has not changed since, and
  // y (not computed for it) is not read; the residual and state stay
  if (!first && converged[l]) {
    if (threadIdx.x == 0) {
      active[l] = 0;
      for (int k = 0; k <= m; ++k) g[(size_t)l * (m + 1) + k] = make_double2(0.0, 0.0);
    }
    return;
  }
  const double2* bl = b + (size_t)l * M;
  double2* rl = r + (size_t)l * M;
  double s = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    double2 v = bl[i];
    if (y) v = csub(v, y[(size_t)l * M + i]);
    rl[i] = v;
    s += cabs2(v);
    if (first) sb += cabs2(bl[i]);
  }
  s = block_sum(s, sh);
  if (first) {
    sb = block_sum(sb, sh);
    if (threadIdx.x == 0) bnorm[l] = sqrt(sb);
    __syncthreads();
  }
  const double bt = sqrt(s);
  const double bn = bnorm[l];
  const bool done = !(bt > tol * bn) || bn == 0.0;
  if (threadIdx.x == 0) {
    beta[l] = bt;
    // this cycle stops at thr; convergence is decided on the FP64 residual at the
    // next restart, so the cycle aims below tol to land under it in one go
    thr[l] = fmax(0.25 * tol * bn, rtol * bt);
    converged[l] = done ? 1 : 0;
    active[l] = done ? 0 : 1;
    if (!done) atomicAdd(&counters[0], 1);
    g[(size_t)l * (m + 1)] = make_double2(done ? 0.0 : bt, 0.0);
    for (int k = 1; k <= m; ++k) g[(size_t)l * (m + 1) + k] = make_double2(0.0, 0.0);
  }
  if (done) return;
  const double inv = 1.0 / bt;
  double2* v0 = V0 + (size_t)l * M;
  for (int i = threadIdx.x; i < M; i += blockDim.x) v0[i] = cscale(rl[i], inv);
}

// need[l] = !converged[l]; *count += the number of such l
__global__ void k_not(int n, const int* __restrict__ a, int* __restrict__ b, unsigned long long* count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = i < n && !a[i];
  if (i < n) b[i] = v;
  const int c = __popc(__ballot_sync(0xffffffffu, v));
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

// Reference norms of the convergence test: bnorm_l <- max(bnorm_l, floor *
// max_k bnorm_k).  Every frequency enters the time steps with the same weight
// (inverse transform), so a frequency whose data lie far below the largest
// (the rounding floor of smooth data at high l) needs only that absolute
// accuracy; its own relative target could sit below what FP64 residuals
// resolve.  One CTA.
__global__ void k_bnorm_floor(int Ls, double* bnorm, double floor_rel) {
  __shared__ double sh[32];
  double mx = 0.0;
  for (int l = threadIdx.x; l < Ls; l += blockDim.x) mx = fmax(mx, bnorm[l]);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, sh[w]);
    sh[0] = mx;
  }
  __syncthreads();
  mx = sh[0];
  for (int l = threadIdx.x; l < Ls; l += blockDim.x) bnorm[l] = fmax(bnorm[l], floor_rel * mx);
}

// One Arnoldi step j for every active frequency: w = basis slot j+1 (already
// holds V v_j) is orthogonalised against v_0..v_j by classical Gram-Schmidt
// applied twice (CGS2), normalised, and the new Hessenberg column is reduced
// by the Givens rotations.  Each frequency's rows are split into nch chunks,
// one block per (chunk, frequency), so that the whole GPU streams the basis;
// the partial sums of a pass are reduced in chunk order by the next kernel
// (no atomics: the result does not depend on the schedule).
//   k_gs_dots:   part[l][ch][k] = sum over the chunk of conj(v_k) w
//   k_gs_update: h = sum_ch part; w -= sum_k h_k v_k on the chunk; the first
//                pass writes H[:, j] = h and the partial dots of the second
//                pass, the second adds h to H[:, j] and writes ||w||^2 partials
//   k_gs_finish: normalise the chunk; chunk 0 applies the rotations.
__device__ __forceinline__ void chunk_rows(int M, int nch, int ch, int& i0, int& i1) {
  const int CH = (M + nch - 1) / nch;
  i0 = ch * CH;
  i1 = min(M, i0 + CH);
}

template <int KB>
__device__ __forceinline__ void chunk_dots(int i0, int i1, int j, size_t stride, const double2* __restrict__ v,
                                           const double2* __restrict__ w, double2* __restrict__ out,
                                           double* sh) {
  for (int k0 = 0; k0 <= j; k0 += KB) {
    double2 acc[KB];
#pragma unroll
    for (int t = 0; t < KB; ++t) acc[t] = make_double2(0.0, 0.0);
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const double2 wi = w[i];
#pragma unroll
      for (int t = 0; t < KB; ++t)
        if (k0 + t <= j) {
          const double2 vk = v[(size_t)(k0 + t) * stride + i];
          acc[t].x += vk.x * wi.x + vk.y * wi.y;
          acc[t].y += vk.x * wi.y - vk.y * wi.x;
        }
    }
    // the KB sums at once: warp sums, then the eight warps' partials added in
    // warp order by one thread per sum (one barrier pair per KB vectors)
    __shared__ double2 red[8][KB];  // blockDim.x = 256
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < KB; ++t) {
      acc[t].x = warp_sum(acc[t].x);
      acc[t].y = warp_sum(acc[t].y);
      if (lane == 0) red[warp][t] = acc[t];
    }
    __syncthreads();
    if (threadIdx.x < KB && k0 + (int)threadIdx.x <= j) {
      double2 a = red[0][threadIdx.x];
      for (int v2 = 1; v2 < 8; ++v2) a = cadd(a, red[v2][threadIdx.x]);
      out[k0 + threadIdx.x] = a;
    }
    __syncthreads();
  }
  (void)sh;
}

template <int KB>
__global__ void __launch_bounds__(256) k_gs_dots(int M, int Ls, int m, int j, int nch,
                                                 const double2* __restrict__ Vb,
                                                 const int* __restrict__ active,
                                                 double2* __restrict__ part) {
  __shared__ double sh[32];
  const int ch = blockIdx.x, l = blockIdx.y;
  if (!active[l]) return;
  int i0, i1;
  chunk_rows(M, nch, ch, i0, i1);
  const size_t stride = (size_t)Ls * M;
  chunk_dots<KB>(i0, i1, j, stride, Vb + (size_t)l * M, Vb + (size_t)(j + 1) * stride + (size_t)l * M,
                 part + ((size_t)l * nch + ch) * (m + 1), sh);
}

template <int KB>
__global__ void __launch_bounds__(256) k_gs_update(int M, int Ls, int m, int j, int nch, int pass,
                                                   double2* __restrict__ Vb, double2* __restrict__ H,
                                                   const int* __restrict__ active,
                                                   const double2* __restrict__ part_in,
                                                   double2* __restrict__ part_out,
                                                   double* __restrict__ nrm) {
  __shared__ double sh[32];
  __shared__ double2 h[64];
  const int ch = blockIdx.x, l = blockIdx.y;
  if (!active[l]) return;
  for (int k = threadIdx.x; k <= j; k += blockDim.x) {
    double2 a = make_double2(0.0, 0.0);
    for (int c = 0; c < nch; ++c) a = cadd(a, part_in[((size_t)l * nch + c) * (m + 1) + k]);
    h[k] = a;
    if (ch == 0) {
      double2* Hc = H + (size_t)l * (m + 1) * m + (size_t)j * (m + 1);
      Hc[k] = pass == 0 ? a : cadd(Hc[k], a);
    }
  }
  __syncthreads();
  int i0, i1;
  chunk_rows(M, nch, ch, i0, i1);
  const size_t stride = (size_t)Ls * M;
  const double2* v = Vb + (size_t)l * M;
  double2* w = Vb + (size_t)(j + 1) * stride + (size_t)l * M;
  double s2 = 0.0;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    double2 wi = w[i];
    for (int k = 0; k <= j; ++k) {
      const double2 vk = v[(size_t)k * stride + i];
      const double2 hk = h[k];
      wi.x -= hk.x * vk.x - hk.y * vk.y;
      wi.y -= hk.x * vk.y + hk.y * vk.x;
    }
    w[i] = wi;
    s2 += cabs2(wi);
  }
  if (pass == 0) {
    __syncthreads();  // this block's rows of w are final before the dots read them
    chunk_dots<KB>(i0, i1, j, stride, v, w, part_out + ((size_t)l * nch + ch) * (m + 1), sh);
  } else {
    s2 = block_sum(s2, sh);
    if (threadIdx.x == 0) nrm[(size_t)l * nch + ch] = s2;
  }
}

// Normalise w; chunk 0 of each frequency closes the Hessenberg column with
// the Givens rotations and decides whether the frequency stays active.
__global__ void __launch_bounds__(256) k_gs_finish(int M, int Ls, int m, int j, int nch,
                                                   double2* __restrict__ Vb, double2* __restrict__ H,
                                                   double* __restrict__ cs, double2* __restrict__ sn,
                                                   double2* __restrict__ g, const double* __restrict__ thr,
                                                   const double* __restrict__ nrm, int* active, int* kdim,
                                                   int* counters, unsigned long long* work) {
  const int ch = blockIdx.x, l = blockIdx.y;
  if (!active[l]) return;
  if (ch == 0 && threadIdx.x == 0) {
    atomicAdd(&work[0], (unsigned long long)(j + 1));
    atomicAdd(&work[1], 1ull);
  }
  double s2 = 0.0;
  for (int c = 0; c < nch; ++c) s2 += nrm[(size_t)l * nch + c];
  const double hn = sqrt(s2);
  int i0, i1;
  chunk_rows(M, nch, ch, i0, i1);
  double2* w = Vb + (size_t)(j + 1) * Ls * M + (size_t)l * M;
  if (hn > 0.0) {
    const double inv = 1.0 / hn;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) w[i] = cscale(w[i], inv);
  }
  if (ch != 0 || threadIdx.x != 0) return;
  double2* col = H + (size_t)l * (m + 1) * m + (size_t)j * (m + 1);
  col[j + 1] = make_double2(hn, 0.0);
  double* csl = cs + (size_t)l * m;
  double2* snl = sn + (size_t)l * m;
  for (int k = 0; k < j; ++k) {  // previous rotations
    const double2 a = col[k], b = col[k + 1];
    col[k] = cadd(cscale(a, csl[k]), cmul(snl[k], b));
    col[k + 1] = csub(cscale(b, csl[k]), cmulc(snl[k], a));  // -conj(s) a + c b
  }
  const double2 a = col[j], b = col[j + 1];
  const double aa = sqrt(cabs2(a)), bb = sqrt(cabs2(b));
  double c;
  double2 s;
  if (bb == 0.0) {
    c = 1.0;
    s = make_double2(0.0, 0.0);
  } else if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
  } else {
    const double t = hypot(aa, bb);
    c = aa / t;
    const double2 ph = cscale(a, 1.0 / aa);
    s = cscale(cmul(ph, make_double2(b.x, -b.y)), 1.0 / t);
  }
  csl[j] = c;
  snl[j] = s;
  col[j] = cadd(cscale(a, c), cmul(s, b));
  col[j + 1] = make_double2(0.0, 0.0);
  double2* gl = g + (size_t)l * (m + 1);
  const double2 gj = gl[j];
  gl[j] = cscale(gj, c);
  gl[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));  // -conj(s) g_j
  kdim[l] = j + 1;
  const double res = sqrt(cabs2(gl[j + 1]));
  if (!(res > thr[l]) || hn == 0.0) {
    active[l] = 0;
    atomicSub(&counters[0], 1);
  }
}

// Back substitution R y = g (k = kdim[l]); then x_l += V y (add = 1) or
// x_l = V y (add = 0, zero for frequencies without an update); one block per l.
__global__ void k_update_x(int M, int Ls, int m, const double2* __restrict__ Vb,
                           const double2* __restrict__ H, const double2* __restrict__ g,
                           const int* __restrict__ kdim, const int* __restrict__ converged,
                           double2* __restrict__ y, double2* __restrict__ x, int add) {
  const int l = blockIdx.x;
  const int k = kdim[l];
  if (converged[l] || k == 0) {
    if (!add)
      for (int i = threadIdx.x; i < M; i += blockDim.x) x[(size_t)l * M + i] = make_double2(0.0, 0.0);
    return;
  }
  const double2* Hl = H + (size_t)l * (m + 1) * m;
  double2* yl = y + (size_t)l * m;
  if (threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double2 acc = g[(size_t)l * (m + 1) + i];
      for (int c = i + 1; c < k; ++c) acc = csub(acc, cmul(Hl[(size_t)c * (m + 1) + i], yl[c]));
      yl[i] = cdiv(acc, Hl[(size_t)i * (m + 1) + i]);
    }
  }
  __syncthreads();
  const size_t stride = (size_t)Ls * M;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    double2 xi = add ? x[(size_t)l * M + i] : make_double2(0.0, 0.0);
    for (int c = 0; c < k; ++c) cfma(xi, yl[c], Vb[(size_t)c * stride + (size_t)l * M + i]);
    x[(size_t)l * M + i] = xi;
  }
}

__global__ void k_axpy(int64_t n, const double2* __restrict__ z, double2* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = cadd(x[i], z[i]);
}

int gmres_solve(cqm_handle* h, const double2* d_b, double2* d_x, cqm_solve_info* info) {
  const int M = h->M, Ls = h->Ls;
  const int m = std::max(1, std::min(h->params.gmres_restart, 64));
  const double tol = h->params.gmres_tol;
  // a cycle with an inexact (FP32) inner operator can only gain about that
  // many digits; the FP64 residual of the next restart continues from there
  const double rtol = h->use_f32 ? h->params.inner_rtol : 0.0;
  Allocator& A = h->alloc;
  GmresWork W;
  int st = CQM_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    e0 = e1 = nullptr;
    W.Vb.free(A); W.r.free(A); W.Z.free(A); W.H.free(A); W.sn.free(A); W.g.free(A); W.y.free(A);
    W.p1.free(A); W.p2.free(A); W.nrm.free(A);
    W.cs.free(A); W.bnorm.free(A); W.beta.free(A); W.thr.free(A); W.active.free(A); W.kdim.free(A);
    W.converged.free(A); W.counters.free(A); W.work.free(A); W.need.free(A);
    if (W.h_counters) cudaFreeHost(W.h_counters);
  };
#define GM_TRY(e) do { st = (e); if (st != CQM_OK) { cleanup(); return st; } } while (0)
  GM_TRY(W.Vb.allocate(A, (size_t)(m + 1) * Ls * M));
  GM_TRY(W.r.allocate(A, (size_t)Ls * M));
  const bool pre = h->use_precond;
  if (pre) GM_TRY(W.Z.allocate(A, (size_t)Ls * M));
  GM_TRY(W.H.allocate(A, (size_t)Ls * (m + 1) * m));
  GM_TRY(W.sn.allocate(A, (size_t)Ls * m));
  GM_TRY(W.g.allocate(A, (size_t)Ls * (m + 1)));
  GM_TRY(W.y.allocate(A, (size_t)Ls * m));
  GM_TRY(W.cs.allocate(A, (size_t)Ls * m));
  GM_TRY(W.bnorm.allocate(A, Ls));
  GM_TRY(W.beta.allocate(A, Ls));
  GM_TRY(W.thr.allocate(A, Ls));
  GM_TRY(W.active.allocate(A, Ls));
  GM_TRY(W.kdim.allocate(A, Ls));
  GM_TRY(W.converged.allocate(A, Ls));
  GM_TRY(W.counters.allocate(A, 4));
  GM_TRY(W.work.allocate(A, 3));
  GM_TRY(W.need.allocate(A, Ls));
  // row chunks per frequency for the Arnoldi kernels: about 4 blocks per SM in
  // all, at least 256 rows per chunk
  const int nch = std::max(1, std::min((M + 255) / 256, (4 * 152 + Ls - 1) / Ls));
  GM_TRY(W.p1.allocate(A, (size_t)Ls * nch * (m + 1)));
  GM_TRY(W.p2.allocate(A, (size_t)Ls * nch * (m + 1)));
  GM_TRY(W.nrm.allocate(A, (size_t)Ls * nch));
  if (cudaMallocHost(&W.h_counters, 4 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    W.h_counters = nullptr;
    cleanup();
    set_last_error("cudaMallocHost failed");
    return CQM_ENOMEM;
  }
  cudaStream_t S = h->stream;
  auto cu = [&](cudaError_t e) -> int {
    if (e != cudaSuccess) {
      set_last_error(std::string("gmres: ") + cudaGetErrorString(e));
      return CQM_ECUDA;
    }
    return CQM_OK;
  };
  GM_TRY(cu(cudaMemsetAsync(d_x, 0, sizeof(double2) * Ls * M, S)));
  GM_TRY(cu(cudaMemsetAsync(W.work.p, 0, 3 * sizeof(unsigned long long), S)));
  GM_TRY(clear_wait_flag(h));
  GM_TRY(cu(cudaEventCreate(&e0)));
  GM_TRY(cu(cudaEventCreate(&e1)));
  cudaEventRecord(e0, S);
  int iters = 0, restarts = 0;
  bool first = true, timed_out = false;
  const int maxit = std::max(1, h->params.gmres_max_iter);
  int status = CQM_OK;
  while (true) {
    double2* Ax = W.Vb.p + (size_t)1 * Ls * M;  // scratch: basis slot 1
    if (!first) {
      // the residual only of the frequencies not converged at an earlier restart
      k_not<<<grid_for(Ls, 256), 256, 0, S>>>(Ls, W.converged.p, W.need.p, W.work.p + 2);
      h->exact_active = W.need.p;
      const int ast = apply_operator(h, d_x, Ax);
      h->exact_active = nullptr;
      GM_TRY(ast);
    }
    GM_TRY(cu(cudaMemsetAsync(W.counters.p, 0, 4 * sizeof(int), S)));
    {
      ProfScope ps_(h, CQM_K_GMRES_OTHER);
      k_restart<<<Ls, 256, 0, S>>>(M, m, d_b, first ? nullptr : Ax, W.r.p, W.Vb.p, W.bnorm.p,
                                   W.beta.p, W.active.p, W.converged.p, W.g.p, tol, rtol, W.thr.p,
                                   first ? 1 : 0, W.counters.p);
      if (first) k_bnorm_floor<<<1, 256, 0, S>>>(Ls, W.bnorm.p, 1e-6);
    }
    GM_TRY(cu(cudaGetLastError()));
    GM_TRY(cu(cudaMemsetAsync(W.kdim.p, 0, sizeof(int) * Ls, S)));
    first = false;
    GM_TRY(cu(cudaMemcpyAsync(W.h_counters, W.counters.p, sizeof(int), cudaMemcpyDeviceToHost, S)));
    GM_TRY(cu(cudaStreamSynchronize(S)));
    if (W.h_counters[0] == 0) break;
    if (iters >= maxit) {
      status = CQM_ENOCONV;
      break;
    }
    for (int j = 0; j < m && iters < maxit; ++j) {
      // the converged frequencies' new basis vectors are never read: the
      // inner apply and the preconditioner skip them
      h->inner_active = W.active.p;
      int ast;
      if (pre) {
        ast = apply_precond(h, W.Vb.p + (size_t)j * Ls * M, W.Z.p, W.active.p);
        if (ast == CQM_OK) ast = apply_operator_inner(h, W.Z.p, W.Vb.p + (size_t)(j + 1) * Ls * M);
      } else {
        ast = apply_operator_inner(h, W.Vb.p + (size_t)j * Ls * M, W.Vb.p + (size_t)(j + 1) * Ls * M);
      }
      h->inner_active = nullptr;
      GM_TRY(ast);
      {
        ProfScope ps_(h, CQM_K_ARNOLDI);
        const dim3 grid((unsigned)nch, (unsigned)Ls);
        k_gs_dots<8><<<grid, 256, 0, S>>>(M, Ls, m, j, nch, W.Vb.p, W.active.p, W.p1.p);
        k_gs_update<8><<<grid, 256, 0, S>>>(M, Ls, m, j, nch, 0, W.Vb.p, W.H.p, W.active.p, W.p1.p,
                                            W.p2.p, W.nrm.p);
        k_gs_update<8><<<grid, 256, 0, S>>>(M, Ls, m, j, nch, 1, W.Vb.p, W.H.p, W.active.p, W.p2.p,
                                            W.p1.p, W.nrm.p);
        k_gs_finish<<<grid, 256, 0, S>>>(M, Ls, m, j, nch, W.Vb.p, W.H.p, W.cs.p, W.sn.p, W.g.p,
                                         W.thr.p, W.nrm.p, W.active.p, W.kdim.p, W.counters.p, W.work.p);
      }
      GM_TRY(cu(cudaGetLastError()));
      ++iters;
      if ((j % 4) == 3 || j == m - 1) {
        GM_TRY(cu(cudaMemcpyAsync(W.h_counters, W.counters.p, sizeof(int), cudaMemcpyDeviceToHost, S)));
        // a bounded wait that ran out leaves the inner products unusable: stop
        GM_TRY(cu(cudaMemcpyAsync(W.h_counters + 1, h->flag.p + 1, sizeof(int), cudaMemcpyDeviceToHost, S)));
        GM_TRY(cu(cudaStreamSynchronize(S)));
        if (W.h_counters[1] != 0) {
          timed_out = true;
          break;
        }
        if (W.h_counters[0] == 0) break;
      }
    }
    if (timed_out) break;
    {
      ProfScope ps_(h, CQM_K_GMRES_OTHER);
      k_update_x<<<Ls, 256, 0, S>>>(M, Ls, m, W.Vb.p, W.H.p, W.g.p, W.kdim.p, W.converged.p, W.y.p,
                                    pre ? W.r.p : d_x, pre ? 0 : 1);
    }
    if (pre) {
      GM_TRY(apply_precond(h, W.r.p, W.Z.p));
      ProfScope ps_(h, CQM_K_GMRES_OTHER);
      k_axpy<<<grid_for((int64_t)Ls * M, 256), 256, 0, S>>>((int64_t)Ls * M, W.Z.p, d_x);
    }
    GM_TRY(cu(cudaGetLastError()));
    ++restarts;
  }
  cudaEventRecord(e1, S);
  // every exit follows a restart, which computed the true FP64 residual
  // beta_l = ||ghat_l - V_l qhat_l|| at the returned solution
  std::vector<double> rel(Ls), bn(Ls);
  std::vector<int> conv(Ls);
  unsigned long long work[3] = {0, 0, 0};
  GM_TRY(cu(cudaMemcpyAsync(work, W.work.p, sizeof(work), cudaMemcpyDeviceToHost, S)));
  GM_TRY(cu(cudaMemcpyAsync(rel.data(), W.beta.p, sizeof(double) * Ls, cudaMemcpyDeviceToHost, S)));
  GM_TRY(cu(cudaMemcpyAsync(bn.data(), W.bnorm.p, sizeof(double) * Ls, cudaMemcpyDeviceToHost, S)));
  GM_TRY(cu(cudaMemcpyAsync(conv.data(), W.converged.p, sizeof(int) * Ls, cudaMemcpyDeviceToHost, S)));
  GM_TRY(cu(cudaStreamSynchronize(S)));
  GM_TRY(check_wait_flag(h));
  for (int l = 0; l < Ls; ++l) rel[l] = bn[l] > 0.0 ? rel[l] / bn[l] : 0.0;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  if (info) {
    info->iterations = iters;
    info->restarts = restarts;
    info->Ls = Ls;
    int c = 0;
    double mx = 0.0;
    for (int l = 0; l < Ls; ++l) {
      c += conv[l];
      mx = std::max(mx, rel[l]);
    }
    info->converged = c;
    info->max_rel_residual = mx;
    info->t_gmres_ms = ms;
    info->arnoldi_vectors = (int64_t)work[0];
    info->arnoldi_freq_steps = (int64_t)work[1];
    info->restart_freq_applies = (int64_t)work[2];
  }
  cleanup();
#undef GM_TRY
  return status;
}

}  // namespace cqm
