// Mixed boundary conditions (Sec. 2.3 eq. wavegalform; Sec. 3.2 eq.
// cqmgalapx, here decoupled in frequency like the single-layer solve), dense:
// Gamma_D is a set of triangles, Gamma_N the rest.  Unknowns per solved
// frequency: the Neumann data qhat on Gamma_D (P0) and the Dirichlet data
// uhat in the hats of the vertices that touch no Gamma_D triangle (so u
// vanishes on Gamma_D).  With the data gD (P1, on the vertices of Gamma_D's
// triangles) and gN (P0, on Gamma_N's triangles) transformed by the R-scaled
// DFT,
//
//   [ V_DD   -K1_DN ] [qhat]   [ (-1/2 I + K1)_D: gDhat - V_D: gNhat   ]
//   [ Kp_ND   D_NN  ] [uhat] = [ (-1/2 I' - Kp)_N: gNhat - D_N: gDhat  ]
//
// with I[m][v] = |t_m| / 3 for the vertices v of t_m (P0 x P1 mass) and
// I' = I^T; one dense system per frequency solved by Gaussian elimination with
// partial pivoting (one CTA per frequency), then the inverse transform.  V
// from the dense mode's matrices, K1, Kp and D from p1_matrices.  FP64.
#include <vector>

#include "handle.cuh"

namespace cqm {

namespace {

// rows of the system: r < nD -> test triangle ED[r]; else test vertex VN[r - nD]
__global__ void k_mixed_system(int M, int nv, int Ls, int nD, int nN, const int* __restrict__ ED,
                               const int* __restrict__ VN, const double2* __restrict__ V,
                               const double2* __restrict__ K1, const double2* __restrict__ Kp,
                               const double2* __restrict__ Dm, double2* __restrict__ A) {
  const int n = nD + nN;
  const int r = blockIdx.x, l = blockIdx.y;
  double2* Ar = A + ((size_t)l * n + r) * n;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double2 v;
    if (r < nD) {
      const size_t row = (size_t)l * M + ED[r];
      if (c < nD) {
        v = V[row * M + ED[c]];
      } else {
        const double2 k = K1[row * nv + VN[c - nD]];
        v = make_double2(-k.x, -k.y);
      }
    } else {
      const size_t row = (size_t)l * nv + VN[r - nD];
      v = c < nD ? Kp[row * M + ED[c]] : Dm[row * nv + VN[c - nD]];
    }
    Ar[c] = v;
  }
}

// right-hand side: one warp per row; Im: P0 x P1 mass (M x nv, real)
__global__ void k_mixed_rhs(int M, int nv, int Ls, int nD, int nN, const int* __restrict__ ED,
                            const int* __restrict__ VN, const double2* __restrict__ V,
                            const double2* __restrict__ K1, const double2* __restrict__ Kp,
                            const double2* __restrict__ Dm, const double* __restrict__ Im,
                            const double2* __restrict__ gDh, const double2* __restrict__ gNh,
                            double2* __restrict__ f) {
  const int n = nD + nN;
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), l = blockIdx.y;
  if (row >= n) return;
  const double2* gd = gDh + (size_t)l * nv;
  const double2* gn = gNh + (size_t)l * M;
  double2 acc = make_double2(0.0, 0.0);
  if (row < nD) {
    const int m = ED[row];
    const double2* k1 = K1 + ((size_t)l * M + m) * nv;
    const double2* vr = V + ((size_t)l * M + m) * M;
    for (int v = lane; v < nv; v += 32) {  // (-1/2 I + K1) gD
      const double2 a = make_double2(k1[v].x - 0.5 * Im[(size_t)m * nv + v], k1[v].y);
      acc = cadd(acc, cmul(a, gd[v]));
    }
    for (int i = lane; i < M; i += 32) {   // - V gN
      const double2 t = cmul(vr[i], gn[i]);
      acc = make_double2(acc.x - t.x, acc.y - t.y);
    }
  } else {
    const int u = VN[row - nD];
    const double2* kp = Kp + ((size_t)l * nv + u) * M;
    const double2* dr = Dm + ((size_t)l * nv + u) * nv;
    for (int i = lane; i < M; i += 32) {   // (-1/2 I' - Kp) gN
      const double2 a = make_double2(-0.5 * Im[(size_t)i * nv + u] - kp[i].x, -kp[i].y);
      acc = cadd(acc, cmul(a, gn[i]));
    }
    for (int v = lane; v < nv; v += 32) {  // - D gD
      const double2 t = cmul(dr[v], gd[v]);
      acc = make_double2(acc.x - t.x, acc.y - t.y);
    }
  }
  acc.x = warp_sum(acc.x);
  acc.y = warp_sum(acc.y);
  if (lane == 0) f[(size_t)l * n + row] = acc;
}

// Gaussian elimination with partial pivoting of A_l x = f_l, in place; the
// solution overwrites f_l.  One CTA of 256 threads per frequency.
__global__ void __launch_bounds__(256) k_mixed_lu(int n, double2* __restrict__ A, double2* __restrict__ f) {
  __shared__ double s_best[8];
  __shared__ int s_idx[8];
  __shared__ int s_piv;
  const int l = blockIdx.x;
  double2* Al = A + (size_t)l * n * n;
  double2* fl = f + (size_t)l * n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < n; ++k) {
    // pivot: the largest |A[i][k]|, i >= k (smallest index on ties)
    double best = -1.0;
    int bi = n;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
      const double2 a = Al[(size_t)i * n + k];
      const double m = a.x * a.x + a.y * a.y;
      if (m > best) { best = m; bi = i; }
    }
    for (int o = 16; o; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { s_best[w] = best; s_idx[w] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = s_best[0];
      int p = s_idx[0];
      for (int v = 1; v < 8; ++v)
        if (s_best[v] > b || (s_best[v] == b && s_idx[v] < p)) { b = s_best[v]; p = s_idx[v]; }
      s_piv = p < n ? p : k;
    }
    __syncthreads();
    const int p = s_piv;
    if (p != k) {
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double2 t = Al[(size_t)k * n + j];
        Al[(size_t)k * n + j] = Al[(size_t)p * n + j];
        Al[(size_t)p * n + j] = t;
      }
      if (threadIdx.x == 0) {
        const double2 t = fl[k];
        fl[k] = fl[p];
        fl[p] = t;
      }
    }
    __syncthreads();
    const double2 akk = Al[(size_t)k * n + k];
    const double den = akk.x * akk.x + akk.y * akk.y;
    const double2 inv = make_double2(akk.x / den, -akk.y / den);
    const double2 fk = fl[k];
    // eliminate below the pivot: one warp per row
    for (int i = k + 1 + w; i < n; i += 8) {
      const double2 fac = cmul(Al[(size_t)i * n + k], inv);
      for (int j = k + 1 + lane; j < n; j += 32) {
        const double2 t = cmul(fac, Al[(size_t)k * n + j]);
        Al[(size_t)i * n + j].x -= t.x;
        Al[(size_t)i * n + j].y -= t.y;
      }
      if (lane == 0) {
        const double2 t = cmul(fac, fk);
        fl[i].x -= t.x;
        fl[i].y -= t.y;
      }
    }
    __syncthreads();
  }
  // back substitution (one thread; n is small in this dense mode)
  if (threadIdx.x == 0) {
    for (int k = n - 1; k >= 0; --k) {
      double2 acc = fl[k];
      for (int j = k + 1; j < n; ++j) {
        const double2 t = cmul(Al[(size_t)k * n + j], fl[j]);
        acc.x -= t.x;
        acc.y -= t.y;
      }
      const double2 akk = Al[(size_t)k * n + k];
      const double den = akk.x * akk.x + akk.y * akk.y;
      fl[k] = cmul(acc, make_double2(akk.x / den, -akk.y / den));
    }
  }
}

// qhat[l][ED[r]] = x[l][r], uhat[l][VN[r]] = x[l][nD + r] (zeroed outside)
__global__ void k_mixed_scatter(int M, int nv, int Ls, int nD, int nN, const int* __restrict__ ED,
                                const int* __restrict__ VN, const double2* __restrict__ x,
                                double2* __restrict__ qh, double2* __restrict__ uh) {
  const int n = nD + nN, l = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double2 v = x[(size_t)l * n + r];
  if (r < nD) qh[(size_t)l * M + ED[r]] = v;
  else uh[(size_t)l * nv + VN[r - nD]] = v;
}

// data outside their parts set to zero: gD on vertices not in keep, gN on Gamma_D's triangles
__global__ void k_mixed_mask(int64_t n, int ncol, const int* __restrict__ keep, const double* __restrict__ a,
                             double* __restrict__ b) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  b[k] = keep[k % ncol] ? a[k] : 0.0;
}

__global__ void k_mass_p0p1(int M, int nv, const int* __restrict__ tri, const double* __restrict__ area,
                            double* __restrict__ Im) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  for (int a = 0; a < 3; ++a) Im[(size_t)m * nv + tri[3 * m + a]] = area[m] / 3.0;
}

}  // namespace

int mixed_solve(cqm_handle* h, const int* dmask, const double* gD, const double* gN, double* q, double* u) {
  if (!h->Vd.p) {
    set_last_error("mixed solve: needs the dense mode's matrices (CQM_MODE_DENSE)");
    return CQM_EINVAL;
  }
  const int M = h->M, nv = h->nv, Ls = h->Ls, L = h->L;
  // spaces from the triangle list (host)
  std::vector<int> tri((size_t)3 * M);
  CQM_CUDA_TRY(cudaMemcpyAsync(tri.data(), h->tri.p, sizeof(int) * 3 * M, cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  std::vector<int> ED, VN, keepD(nv, 0), keepN(M, 1), used(nv, 0);
  for (int m = 0; m < M; ++m) {
    for (int a = 0; a < 3; ++a) used[tri[3 * m + a]] = 1;
    if (dmask[m]) {
      ED.push_back(m);
      keepN[m] = 0;
      for (int a = 0; a < 3; ++a) keepD[tri[3 * m + a]] = 1;
    }
  }
  for (int v = 0; v < nv; ++v)
    if (used[v] && !keepD[v]) VN.push_back(v);
  const int nD = (int)ED.size(), nN = (int)VN.size(), n = nD + nN;
  if (n == 0) {
    set_last_error("mixed solve: no unknowns");
    return CQM_EINVAL;
  }
  Allocator& A = h->alloc;
  DArray<int> dED, dVN, dkeepD, dkeepN;
  DArray<double2> K1, Kp, Dm, Asys, f, gDh, gNh, qh, uh;
  DArray<double> Im, gDm, gNm;
  auto release = [&]() {
    dED.free(A); dVN.free(A); dkeepD.free(A); dkeepN.free(A); K1.free(A); Kp.free(A); Dm.free(A);
    Asys.free(A); f.free(A); gDh.free(A); gNh.free(A); qh.free(A); uh.free(A); Im.free(A); gDm.free(A);
    gNm.free(A);
  };
  int st = CQM_OK;
#define MX_TRY(e) do { st = (e); if (st != CQM_OK) { release(); return st; } } while (0)
#define MX_CU(e) do { if ((e) != cudaSuccess) { set_last_error("mixed solve: CUDA error"); release(); return CQM_ECUDA; } } while (0)
  MX_TRY(dED.allocate(A, std::max(1, nD)));
  MX_TRY(dVN.allocate(A, std::max(1, nN)));
  MX_TRY(dkeepD.allocate(A, nv));
  MX_TRY(dkeepN.allocate(A, M));
  MX_TRY(K1.allocate(A, (size_t)Ls * M * nv));
  MX_TRY(Kp.allocate(A, (size_t)Ls * nv * M));
  MX_TRY(Dm.allocate(A, (size_t)Ls * nv * nv));
  MX_TRY(Asys.allocate(A, (size_t)Ls * n * n));
  MX_TRY(f.allocate(A, (size_t)Ls * n));
  MX_TRY(gDh.allocate(A, (size_t)Ls * nv));
  MX_TRY(gNh.allocate(A, (size_t)Ls * M));
  MX_TRY(qh.allocate(A, (size_t)Ls * M));
  MX_TRY(uh.allocate(A, (size_t)Ls * nv));
  MX_TRY(Im.allocate(A, (size_t)M * nv));
  MX_TRY(gDm.allocate(A, (size_t)L * nv));
  MX_TRY(gNm.allocate(A, (size_t)L * M));
  cudaStream_t S = h->stream;
  if (nD) MX_CU(cudaMemcpyAsync(dED.p, ED.data(), sizeof(int) * nD, cudaMemcpyHostToDevice, S));
  if (nN) MX_CU(cudaMemcpyAsync(dVN.p, VN.data(), sizeof(int) * nN, cudaMemcpyHostToDevice, S));
  MX_CU(cudaMemcpyAsync(dkeepD.p, keepD.data(), sizeof(int) * nv, cudaMemcpyHostToDevice, S));
  MX_CU(cudaMemcpyAsync(dkeepN.p, keepN.data(), sizeof(int) * M, cudaMemcpyHostToDevice, S));
  MX_CU(cudaMemsetAsync(Im.p, 0, sizeof(double) * M * nv, S));
  MX_CU(cudaMemsetAsync(qh.p, 0, sizeof(double2) * Ls * M, S));
  MX_CU(cudaMemsetAsync(uh.p, 0, sizeof(double2) * Ls * nv, S));
  k_mass_p0p1<<<grid_for(M, 128), 128, 0, S>>>(M, nv, h->tri.p, h->area.p, Im.p);
  k_mixed_mask<<<grid_for((int64_t)L * nv, 256), 256, 0, S>>>((int64_t)L * nv, nv, dkeepD.p, gD, gDm.p);
  k_mixed_mask<<<grid_for((int64_t)L * M, 256), 256, 0, S>>>((int64_t)L * M, M, dkeepN.p, gN, gNm.p);
  MX_CU(cudaGetLastError());
  MX_TRY(p1_matrices(h, K1.p, Kp.p, Dm.p));
  MX_TRY(forward_transform_cols(h, nv, gDm.p, gDh.p));
  MX_TRY(forward_transform_cols(h, M, gNm.p, gNh.p));
  k_mixed_system<<<dim3((unsigned)n, (unsigned)Ls), 128, 0, S>>>(M, nv, Ls, nD, nN, dED.p, dVN.p, h->Vd.p, K1.p,
                                                               Kp.p, Dm.p, Asys.p);
  k_mixed_rhs<<<dim3((unsigned)grid_for(n, 8), (unsigned)Ls), 256, 0, S>>>(M, nv, Ls, nD, nN, dED.p, dVN.p,
                                                                         h->Vd.p, K1.p, Kp.p, Dm.p, Im.p, gDh.p,
                                                                         gNh.p, f.p);
  k_mixed_lu<<<Ls, 256, 0, S>>>(n, Asys.p, f.p);
  k_mixed_scatter<<<dim3((unsigned)grid_for(n, 128), (unsigned)Ls), 128, 0, S>>>(M, nv, Ls, nD, nN, dED.p,
                                                                               dVN.p, f.p, qh.p, uh.p);
  MX_CU(cudaGetLastError());
  MX_TRY(inverse_transform_cols(h, M, qh.p, q));
  MX_TRY(inverse_transform_cols(h, nv, uh.p, u));
  MX_CU(cudaStreamSynchronize(S));
#undef MX_TRY
#undef MX_CU
  release();
  return CQM_OK;
}

}  // namespace cqm
