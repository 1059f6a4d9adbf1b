// Chebyshev-interpolation cluster bases (Sec. 4, eqs. degexp/uniformlr, Def. 5,
// Alg. 1) and the application of the compressed tensor (eq. lrfinal):
//   near block b = r x c:  V_l[b] = sum_t D_b[l,t] C_{b,t}
//   far block  b = r x c:  V_l[b] = U_r (sum_t D_b[l,t] C_{b,t}) U_c^T
// applied to all solved frequencies at once (X: Ls x M complex, row l).
// Far field: leaf forward xhat_c = U_c^T x_c, up-sweep with transfers
// E_{c',c}^T, coupling yhat_r += sum_t D[l,t] C_t xhat_c, down-sweep with
// E_{r',r}, leaf backward y_r += U_r yhat_r.
// Interpolation nodes: m first-kind Chebyshev points per axis on the cluster
// box, mu = ix + m (iy + m iz); E_{r',r}[lambda, mu] = L_{r,mu}(xi_{r',lambda})
// is the Kronecker product of three 1-D m x m factors.
#include <algorithm>
#include <vector>

#include "handle.cuh"

namespace cqm {

constexpr int MAXM = 4;
constexpr int MAXP = MAXM * MAXM * MAXM;

__global__ void k_cheb_nodes(int n_nodes, int m, const double* __restrict__ lo,
                             const double* __restrict__ hi, double* cheb) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_nodes * 3 * m) return;
  const int node = t / (3 * m), rem = t - node * 3 * m, ax = rem / m, k = rem - ax * m;
  const double* l = lo + 3 * node;
  const double* u = hi + 3 * node;
  const double mid = (l[ax] + u[ax]) * 0.5;
  double half = (u[ax] - l[ax]) * 0.5;
  if (!(half > 0.0)) {
    const double dx = u[0] - l[0], dy = u[1] - l[1], dz = u[2] - l[2];
    half = 0.5e-8 * sqrt(dx * dx + dy * dy + dz * dz);
  }
  cheb[t] = mid + half * cospi((2.0 * k + 1.0) / (2.0 * m));
}

// l_k(x) on the m nodes of one axis
__device__ __forceinline__ double lagrange1(const double* nodes, int m, int k, double x) {
  double v = 1.0;
  for (int j = 0; j < m; ++j)
    if (j != k) v *= (x - nodes[j]) / (nodes[k] - nodes[j]);
  return v;
}

// Leaf bases: U[pos][mu] = |tau| sum_q w_q L_{r,mu}(x_q) for the triangle at
// position pos of leaf r (Radon rule).
__global__ void k_leaf_basis(int M, int m, int p, const int* __restrict__ leaf_of,
                             const int* __restrict__ perm, const double* __restrict__ P,
                             const double* __restrict__ area, const double* __restrict__ cheb,
                             double* U) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M * p) return;
  const int pos = t / p, mu = t - pos * p;
  const int r = leaf_of[pos];
  const int tri = perm[pos];
  const double* v = P + 9 * tri;
  const double* nd = cheb + (size_t)r * 3 * m;
  const int ix = mu % m, iy = (mu / m) % m, iz = mu / (m * m);
  double acc = 0.0;
  for (int q = 0; q < 7; ++q) {
    double l0, l1, l2, w;
    radon7(q, l0, l1, l2, w);
    const double x = l0 * v[0] + l1 * v[3] + l2 * v[6];
    const double y = l0 * v[1] + l1 * v[4] + l2 * v[7];
    const double z = l0 * v[2] + l1 * v[5] + l2 * v[8];
    acc += w * lagrange1(nd, m, ix, x) * lagrange1(nd + m, m, iy, y) * lagrange1(nd + 2 * m, m, iz, z);
  }
  U[t] = area[tri] * acc;
}

// 1-D transfer factors of node s (parent r): Etr[s][ax][a][b] = l^{(r)}_b(xi^{(s)}_{ax,a}).
__global__ void k_transfer(int n_nodes, int m, const int* __restrict__ parent,
                           const double* __restrict__ cheb, double* Etr) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_nodes * 3 * m * m) return;
  const int s = t / (3 * m * m), rem = t - s * 3 * m * m, ax = rem / (m * m);
  const int a = (rem / m) % m, b = rem % m;
  const int r = parent[s];
  if (r < 0) {
    Etr[t] = 0.0;
    return;
  }
  Etr[t] = lagrange1(cheb + ((size_t)r * 3 + ax) * m, m, b, cheb[((size_t)s * 3 + ax) * m + a]);
}

__global__ void k_leaf_of(int n_leaves, const int* __restrict__ leaves, const int* __restrict__ begin,
                          const int* __restrict__ end, int* leaf_of) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_leaves) return;
  const int r = leaves[k];
  for (int pos = begin[r]; pos < end[r]; ++pos) leaf_of[pos] = r;
}

int make_apply_plan(cqm_handle* h);

int build_bases(cqm_handle* h) {
  const int n = h->n_nodes, m = h->m, p = h->p, M = h->M;
  CQM_TRY(h->cheb.allocate(h->alloc, (size_t)n * 3 * m));
  CQM_TRY(h->Uleaf.allocate(h->alloc, (size_t)M * p));
  CQM_TRY(h->Etr.allocate(h->alloc, (size_t)n * 3 * m * m));
  std::vector<int> leaves;
  for (int r = 0; r < n; ++r)
    if (h->h_son0[r] < 0) leaves.push_back(r);
  DArray<int> dleaves, leaf_of;
  int st = dleaves.allocate(h->alloc, leaves.size());
  if (st == CQM_OK) st = leaf_of.allocate(h->alloc, M);
  if (st == CQM_OK) {
    cudaMemcpyAsync(dleaves.p, leaves.data(), sizeof(int) * leaves.size(), cudaMemcpyHostToDevice, h->stream);
    {
      ProfScope ps_(h, CQM_K_BASES);
      k_cheb_nodes<<<grid_for(n * 3 * m, 256), 256, 0, h->stream>>>(n, m, h->node_lo.p, h->node_hi.p, h->cheb.p);
    }
    {
      ProfScope ps_(h, CQM_K_BASES);
      k_leaf_of<<<grid_for(leaves.size(), 128), 128, 0, h->stream>>>((int)leaves.size(), dleaves.p,
                                                                    h->node_begin.p, h->node_end.p, leaf_of.p);
    }
    {
      ProfScope ps_(h, CQM_K_BASES);
      k_leaf_basis<<<grid_for((int64_t)M * p, 256), 256, 0, h->stream>>>(
          M, m, p, leaf_of.p, h->perm.p, h->P.p, h->area.p, h->cheb.p, h->Uleaf.p);
    }
    {
      ProfScope ps_(h, CQM_K_BASES);
      k_transfer<<<grid_for(n * 3 * m * m, 256), 256, 0, h->stream>>>(n, m, h->node_parent.p, h->cheb.p, h->Etr.p);
    }
    if (cudaGetLastError() != cudaSuccess) st = CQM_ECUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) st = CQM_ECUDA;
  }
  dleaves.free(h->alloc);
  leaf_of.free(h->alloc);
  if (st == CQM_ECUDA) set_last_error("build_bases failed");
  CQM_TRY(st);
  CQM_TRY(h->xhat.allocate(h->alloc, (size_t)n * p * h->Ls));
  CQM_TRY(h->yhat.allocate(h->alloc, (size_t)n * p * h->Ls));
  return make_apply_plan(h);
}

// ------------------------------------------------------------------ apply ---
constexpr int LC = 32;  // frequencies per chunk (one warp width)

// Near field: one block per leaf row cluster r; y_r = sum over near blocks.
__global__ void __launch_bounds__(256) k_near_apply(
    int M, int Ls, int cap, const int* __restrict__ leaves, const int* __restrict__ rowptr,
    const int2* __restrict__ blocks, const int* __restrict__ rank, const int64_t* __restrict__ off,
    const double2* __restrict__ Cn, const double2* __restrict__ Dn, const int* __restrict__ begin,
    const int* __restrict__ end, const int* __restrict__ perm, const double2* __restrict__ X,
    double2* __restrict__ Y) {
  __shared__ double2 Xs[32][LC];
  __shared__ double2 Cs[32 * 32];
  __shared__ double2 Ds[LC];
  const int r = leaves[blockIdx.x];
  const int rb = begin[r], nr = end[r] - rb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // 8 warps: rows w, w+8, w+16, w+24
  for (int l0 = 0; l0 < Ls; l0 += LC) {
    double2 acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = make_double2(0.0, 0.0);
    for (int bi = rowptr[r]; bi < rowptr[r + 1]; ++bi) {
      const int c = blocks[bi].y;
      const int cb = begin[c], nc = end[c] - cb;
      __syncthreads();
      for (int t = threadIdx.x; t < nc * LC; t += blockDim.x) {
        const int j = t / LC, l = t - j * LC;
        Xs[j][l] = (l0 + l < Ls) ? X[(size_t)(l0 + l) * M + perm[cb + j]] : make_double2(0.0, 0.0);
      }
      const int rk = rank[bi];
      for (int tt = 0; tt < rk; ++tt) {
        __syncthreads();
        const double2* Ct = Cn + off[bi] + (size_t)tt * nr * nc;
        for (int t = threadIdx.x; t < nr * nc; t += blockDim.x) Cs[t] = Ct[t];
        if (threadIdx.x < LC)
          Ds[threadIdx.x] = (l0 + threadIdx.x < Ls) ? Dn[((size_t)bi * cap + tt) * Ls + l0 + threadIdx.x]
                                                    : make_double2(0.0, 0.0);
        __syncthreads();
        const double2 d = Ds[lane];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int i = w + 8 * k;
          if (i < nr) {
            double2 z = make_double2(0.0, 0.0);
            for (int j = 0; j < nc; ++j) cfma(z, Cs[i * nc + j], Xs[j][lane]);
            cfma(acc[k], d, z);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = w + 8 * k;
      if (i < nr && l0 + lane < Ls) Y[(size_t)(l0 + lane) * M + perm[rb + i]] = acc[k];
    }
  }
}

// xhat_c[mu][l] = sum_j U[cb + j][mu] x[l][perm[cb + j]] for leaf c.
__global__ void __launch_bounds__(256) k_leaf_forward(int M, int Ls, int p,
                                                      const int* __restrict__ leaves,
                                                      const int* __restrict__ begin,
                                                      const int* __restrict__ end,
                                                      const int* __restrict__ perm,
                                                      const double* __restrict__ U,
                                                      const double2* __restrict__ X,
                                                      double2* __restrict__ xhat) {
  __shared__ double2 Xs[32][LC];
  __shared__ double Us[32 * MAXP];
  const int c = leaves[blockIdx.x];
  const int cb = begin[c], nc = end[c] - cb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < nc * p; t += blockDim.x) Us[t] = U[(size_t)cb * p + t];
  for (int l0 = 0; l0 < Ls; l0 += LC) {
    __syncthreads();
    for (int t = threadIdx.x; t < nc * LC; t += blockDim.x) {
      const int j = t / LC, l = t - j * LC;
      Xs[j][l] = (l0 + l < Ls) ? X[(size_t)(l0 + l) * M + perm[cb + j]] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int mu = w; mu < p; mu += 8) {
      double2 z = make_double2(0.0, 0.0);
      for (int j = 0; j < nc; ++j) {
        const double u = Us[j * p + mu];
        z.x += u * Xs[j][lane].x;
        z.y += u * Xs[j][lane].y;
      }
      if (l0 + lane < Ls) xhat[((size_t)c * p + mu) * Ls + l0 + lane] = z;
    }
  }
}

// E[lambda][mu] of node s from its 1-D factors into shared memory.
__device__ void expand_transfer(const double* __restrict__ Etr, int s, int m, int p, double* E) {
  const double* f = Etr + (size_t)s * 3 * m * m;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int lam = t / p, mu = t - lam * p;
    const int lx = lam % m, ly = (lam / m) % m, lz = lam / (m * m);
    const int mx = mu % m, my = (mu / m) % m, mz = mu / (m * m);
    E[t] = f[lx * m + mx] * f[m * m + ly * m + my] * f[2 * m * m + lz * m + mz];
  }
}

// Up-sweep for one level: xhat_r = sum_{s in sons(r)} E_{s,r}^T xhat_s.
__global__ void __launch_bounds__(256) k_upsweep(int node0, int Ls, int m, int p,
                                                 const int* __restrict__ son0,
                                                 const int* __restrict__ son1,
                                                 const double* __restrict__ Etr,
                                                 double2* __restrict__ xhat) {
  extern __shared__ double sm[];
  double* E = sm;  // p x p
  const int r = node0 + blockIdx.x;
  if (son0[r] < 0) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int l0 = 0; l0 < Ls; l0 += LC) {
    double2 acc[MAXP / 8];
    const int nmu = (p + 7) / 8;
    for (int k = 0; k < nmu; ++k) acc[k] = make_double2(0.0, 0.0);
    for (int si = 0; si < 2; ++si) {
      const int s = si == 0 ? son0[r] : son1[r];
      __syncthreads();
      expand_transfer(Etr, s, m, p, E);
      __syncthreads();
      if (l0 + lane < Ls) {
        for (int lam = 0; lam < p; ++lam) {
          const double2 xv = xhat[((size_t)s * p + lam) * Ls + l0 + lane];
          for (int k = 0; k < nmu; ++k) {
            const int mu = w + 8 * k;
            if (mu < p) {
              const double e = E[lam * p + mu];
              acc[k].x += e * xv.x;
              acc[k].y += e * xv.y;
            }
          }
        }
      }
    }
    if (l0 + lane < Ls)
      for (int k = 0; k < nmu; ++k) {
        const int mu = w + 8 * k;
        if (mu < p) xhat[((size_t)r * p + mu) * Ls + l0 + lane] = acc[k];
      }
  }
}

// Coupling: yhat_r[mu][l] += sum_{b=(r,c)} sum_t D_b[t][l] sum_nu C_{b,t}[mu][nu] xhat_c[nu][l].
__global__ void __launch_bounds__(256) k_far_coupling(int Ls, int p, int cap,
                                                      const int* __restrict__ rows,
                                                      const int* __restrict__ rowptr,
                                                      const int2* __restrict__ blocks,
                                                      const int* __restrict__ rank,
                                                      const double2* __restrict__ Cf,
                                                      const double2* __restrict__ Df,
                                                      const double2* __restrict__ xhat,
                                                      double2* __restrict__ yhat) {
  extern __shared__ double2 sm2[];
  double2* Xs = sm2;                 // p x LC
  double2* Cs = sm2 + MAXP * LC;     // p x p
  __shared__ double2 Ds[LC];
  const int r = rows[blockIdx.x];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int l0 = 0; l0 < Ls; l0 += LC) {
    double2 acc[MAXP / 8];
    const int nmu = (p + 7) / 8;
    for (int k = 0; k < nmu; ++k) acc[k] = make_double2(0.0, 0.0);
    for (int bi = rowptr[r]; bi < rowptr[r + 1]; ++bi) {
      const int c = blocks[bi].y;
      __syncthreads();
      for (int t = threadIdx.x; t < p * LC; t += blockDim.x) {
        const int nu = t / LC, l = t - nu * LC;
        Xs[t] = (l0 + l < Ls) ? xhat[((size_t)c * p + nu) * Ls + l0 + l] : make_double2(0.0, 0.0);
      }
      const int rk = rank[bi];
      for (int tt = 0; tt < rk; ++tt) {
        __syncthreads();
        const double2* Ct = Cf + ((size_t)bi * cap + tt) * p * p;
        for (int t = threadIdx.x; t < p * p; t += blockDim.x) Cs[t] = Ct[t];
        if (threadIdx.x < LC)
          Ds[threadIdx.x] = (l0 + threadIdx.x < Ls) ? Df[((size_t)bi * cap + tt) * Ls + l0 + threadIdx.x]
                                                    : make_double2(0.0, 0.0);
        __syncthreads();
        const double2 d = Ds[lane];
        for (int k = 0; k < nmu; ++k) {
          const int mu = w + 8 * k;
          if (mu < p) {
            double2 z = make_double2(0.0, 0.0);
            for (int nu = 0; nu < p; ++nu) cfma(z, Cs[mu * p + nu], Xs[nu * LC + lane]);
            cfma(acc[k], d, z);
          }
        }
      }
    }
    if (l0 + lane < Ls)
      for (int k = 0; k < nmu; ++k) {
        const int mu = w + 8 * k;
        if (mu < p) {
          double2* o = yhat + ((size_t)r * p + mu) * Ls + l0 + lane;
          *o = cadd(*o, acc[k]);
        }
      }
  }
}

// Down-sweep for one level: yhat_s += E_{s,r} yhat_r for every node s of the level.
__global__ void __launch_bounds__(256) k_downsweep(int node0, int Ls, int m, int p,
                                                   const int* __restrict__ parent,
                                                   const double* __restrict__ Etr,
                                                   double2* __restrict__ yhat) {
  extern __shared__ double sm[];
  double* E = sm;
  const int s = node0 + blockIdx.x;
  const int r = parent[s];
  if (r < 0) return;
  expand_transfer(Etr, s, m, p, E);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int l0 = 0; l0 < Ls; l0 += LC) {
    if (l0 + lane >= Ls) continue;
    for (int lam = w; lam < p; lam += 8) {
      double2 z = make_double2(0.0, 0.0);
      for (int mu = 0; mu < p; ++mu) {
        const double e = E[lam * p + mu];
        const double2 yv = yhat[((size_t)r * p + mu) * Ls + l0 + lane];
        z.x += e * yv.x;
        z.y += e * yv.y;
      }
      double2* o = yhat + ((size_t)s * p + lam) * Ls + l0 + lane;
      *o = cadd(*o, z);
    }
  }
}

// y[l][perm[rb + i]] += sum_mu U[rb + i][mu] yhat_r[mu][l] for leaf r.
__global__ void __launch_bounds__(256) k_leaf_backward(int M, int Ls, int p,
                                                       const int* __restrict__ leaves,
                                                       const int* __restrict__ begin,
                                                       const int* __restrict__ end,
                                                       const int* __restrict__ perm,
                                                       const double* __restrict__ U,
                                                       const double2* __restrict__ yhat,
                                                       double2* __restrict__ Y) {
  __shared__ double Us[32 * MAXP];
  const int r = leaves[blockIdx.x];
  const int rb = begin[r], nr = end[r] - rb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < nr * p; t += blockDim.x) Us[t] = U[(size_t)rb * p + t];
  __syncthreads();
  for (int l0 = 0; l0 < Ls; l0 += LC) {
    if (l0 + lane >= Ls) continue;
    for (int i = w; i < nr; i += 8) {
      double2 z = make_double2(0.0, 0.0);
      for (int mu = 0; mu < p; ++mu) {
        const double u = Us[i * p + mu];
        const double2 yv = yhat[((size_t)r * p + mu) * Ls + l0 + lane];
        z.x += u * yv.x;
        z.y += u * yv.y;
      }
      double2* o = Y + (size_t)(l0 + lane) * M + perm[rb + i];
      *o = cadd(*o, z);
    }
  }
}

int make_apply_plan(cqm_handle* h) {
  h->h_leaves.clear();
  h->h_far_rows.clear();
  for (int r = 0; r < h->n_nodes; ++r)
    if (h->h_son0[r] < 0) h->h_leaves.push_back(r);
  std::vector<int> hasfar(h->n_nodes, 0);
  for (auto& b : h->h_far) hasfar[b.x] = 1;
  for (int r = 0; r < h->n_nodes; ++r)
    if (hasfar[r]) h->h_far_rows.push_back(r);
  CQM_TRY(h->d_leaves.allocate(h->alloc, std::max<size_t>(1, h->h_leaves.size())));
  CQM_TRY(h->d_far_rows.allocate(h->alloc, std::max<size_t>(1, h->h_far_rows.size())));
  CQM_CUDA_TRY(cudaMemcpyAsync(h->d_leaves.p, h->h_leaves.data(), sizeof(int) * h->h_leaves.size(),
                               cudaMemcpyHostToDevice, h->stream));
  if (!h->h_far_rows.empty())
    CQM_CUDA_TRY(cudaMemcpyAsync(h->d_far_rows.p, h->h_far_rows.data(),
                                 sizeof(int) * h->h_far_rows.size(), cudaMemcpyHostToDevice, h->stream));
  const size_t shC = sizeof(double2) * (MAXP * LC + (size_t)h->p * h->p);
  CQM_CUDA_TRY(cudaFuncSetAttribute(k_far_coupling, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shC));
  return CQM_OK;
}

int apply_compressed(cqm_handle* h, const double2* x, double2* y) {
  const int nleaf = (int)h->h_leaves.size(), nfr = (int)h->h_far_rows.size();
  const int M = h->M, Ls = h->Ls, p = h->p, m = h->m;
  cudaStream_t S = h->stream;
  int st = CQM_OK;
  do {
    {
      ProfScope ps_(h, CQM_K_NEAR_APPLY);
      k_near_apply<<<(unsigned)nleaf, 256, 0, S>>>(
          M, Ls, h->rank_cap, h->d_leaves.p, h->near_rowptr.p, h->near_rc.p, h->near_rank.p,
          h->near_off.p, h->nearC.p, h->nearD.p, h->node_begin.p, h->node_end.p, h->perm.p, x, y);
    }
    if (h->n_far == 0) break;
    {
      ProfScope ps_(h, CQM_K_LEAF_FORWARD);
      k_leaf_forward<<<(unsigned)nleaf, 256, 0, S>>>(M, Ls, p, h->d_leaves.p, h->node_begin.p,
                                                              h->node_end.p, h->perm.p, h->Uleaf.p, x,
                                                              h->xhat.p);
    }
    const size_t shE = sizeof(double) * p * p;
    for (int lv = h->depth - 1; lv >= 0; --lv) {
      const int n0 = h->level_begin[lv], n1 = h->level_begin[lv + 1];
      if (n1 > n0)
        {
          ProfScope ps_(h, CQM_K_UPSWEEP);
          k_upsweep<<<n1 - n0, 256, shE, S>>>(n0, Ls, m, p, h->node_son0.p, h->node_son1.p, h->Etr.p,
                                              h->xhat.p);
        }
    }
    cudaMemsetAsync(h->yhat.p, 0, sizeof(double2) * (size_t)h->n_nodes * p * Ls, S);
    const size_t shC = sizeof(double2) * (MAXP * LC + (size_t)p * p);
    {
      ProfScope ps_(h, CQM_K_FAR_COUPLING);
      k_far_coupling<<<(unsigned)nfr, 256, shC, S>>>(
          Ls, p, h->rank_cap, h->d_far_rows.p, h->far_rowptr.p, h->far_rc.p, h->far_rank.p, h->farC.p,
          h->farD.p, h->xhat.p, h->yhat.p);
    }
    for (int lv = 1; lv <= h->depth; ++lv) {
      const int n0 = h->level_begin[lv], n1 = h->level_begin[lv + 1];
      if (n1 > n0)
        {
          ProfScope ps_(h, CQM_K_DOWNSWEEP);
          k_downsweep<<<n1 - n0, 256, shE, S>>>(n0, Ls, m, p, h->node_parent.p, h->Etr.p, h->yhat.p);
        }
    }
    {
      ProfScope ps_(h, CQM_K_LEAF_BACKWARD);
      k_leaf_backward<<<(unsigned)nleaf, 256, 0, S>>>(M, Ls, p, h->d_leaves.p, h->node_begin.p,
                                                               h->node_end.p, h->perm.p, h->Uleaf.p,
                                                               h->yhat.p, y);
    }
  } while (0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("apply_compressed: ") + cudaGetErrorString(e));
    st = CQM_ECUDA;
  }
  return st;
}

}  // namespace cqm
