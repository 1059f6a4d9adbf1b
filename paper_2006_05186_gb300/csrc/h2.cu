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
#include <type_traits>
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
// The kernels below are templated on the storage/arithmetic real type R of
// the operator (double: the FP64 operator; float: its FP32 copy used by the
// inner GMRES iterations).  Input and output vectors are always FP64.
constexpr int LC = 32;  // frequencies per chunk (one warp width)

// Whether any frequency of the chunk [l0, l0 + LC) is still iterating (act
// may be null: all are); a barrier, called by every thread of the block.
__device__ __forceinline__ bool chunk_active(const int* __restrict__ act, int l0, int Ls) {
  if (!act) return true;
  return __syncthreads_or(threadIdx.x < LC && l0 + (int)threadIdx.x < Ls && act[l0 + threadIdx.x]) != 0;
}


// Near field: one block per leaf row cluster r; y_r = sum over near blocks.
template <class R>
__global__ void __launch_bounds__(256) k_near_apply(
    int M, int Ls, int cap, const int* __restrict__ leaves, const int* __restrict__ rowptr,
    const int2* __restrict__ blocks, const int* __restrict__ rank, const int64_t* __restrict__ off,
    const typename Cplx<R>::type* __restrict__ Cn, const typename Cplx<R>::type* __restrict__ Dn,
    const int* __restrict__ begin, const int* __restrict__ end, const int* __restrict__ perm,
    const double2* __restrict__ X, double2* __restrict__ Y) {
  using C = typename Cplx<R>::type;
  __shared__ C Xs[32][LC];
  __shared__ C Cs[32 * 32];
  __shared__ C Ds[LC];
  const int r = leaves[blockIdx.x];
  const int rb = begin[r], nr = end[r] - rb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // 8 warps: rows w, w+8, w+16, w+24
  for (int l0 = 0; l0 < Ls; l0 += LC) {
    C acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = cz<C>();
    for (int bi = rowptr[r]; bi < rowptr[r + 1]; ++bi) {
      const int c = blocks[bi].y;
      const int cb = begin[c], nc = end[c] - cb;
      __syncthreads();
      for (int t = threadIdx.x; t < nc * LC; t += blockDim.x) {
        const int j = t / LC, l = t - j * LC;
        Xs[j][l] = (l0 + l < Ls) ? to_c(X[(size_t)(l0 + l) * M + perm[cb + j]], (C*)0) : cz<C>();
      }
      const int rk = rank[bi];
      for (int tt = 0; tt < rk; ++tt) {
        __syncthreads();
        const C* Ct = Cn + off[bi] + (size_t)tt * nr * nc;
        for (int t = threadIdx.x; t < nr * nc; t += blockDim.x) Cs[t] = Ct[t];
        if (threadIdx.x < LC)
          Ds[threadIdx.x] = (l0 + threadIdx.x < Ls) ? Dn[((size_t)bi * cap + tt) * Ls + l0 + threadIdx.x]
                                                    : cz<C>();
        __syncthreads();
        const C d = Ds[lane];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int i = w + 8 * k;
          if (i < nr) {
            C z = cz<C>();
            for (int j = 0; j < nc; ++j) cfma(z, Cs[i * nc + j], Xs[j][lane]);
            cfma(acc[k], d, z);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = w + 8 * k;
      if (i < nr && l0 + lane < Ls) Y[(size_t)(l0 + lane) * M + perm[rb + i]] = to_d(acc[k]);
    }
  }
}

// xhat_c[mu][l] = sum_j U[cb + j][mu] x[l][perm[cb + j]] for leaf c.
template <class R>
__global__ void __launch_bounds__(256) k_leaf_forward(int M, int Ls, int p,
                                                      const int* __restrict__ leaves,
                                                      const int* __restrict__ begin,
                                                      const int* __restrict__ end,
                                                      const int* __restrict__ perm,
                                                      const R* __restrict__ U,
                                                      const double2* __restrict__ X,
                                                      typename Cplx<R>::type* __restrict__ xhat,
                                                      const int* __restrict__ act) {
  using C = typename Cplx<R>::type;
  __shared__ C Xs[32][LC];
  __shared__ R Us[32 * MAXP];
  const int c = leaves[blockIdx.x];
  const int cb = begin[c], nc = end[c] - cb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < nc * p; t += blockDim.x) Us[t] = U[(size_t)cb * p + t];
  for (int l0 = 0; l0 < Ls; l0 += LC) {
    if (!chunk_active(act, l0, Ls)) continue;
    __syncthreads();
    for (int t = threadIdx.x; t < nc * LC; t += blockDim.x) {
      const int j = t / LC, l = t - j * LC;
      Xs[j][l] = (l0 + l < Ls) ? to_c(X[(size_t)(l0 + l) * M + perm[cb + j]], (C*)0) : cz<C>();
    }
    __syncthreads();
    for (int mu = w; mu < p; mu += 8) {
      C z = cz<C>();
      for (int j = 0; j < nc; ++j) {
        const R u = Us[j * p + mu];
        z.x += u * Xs[j][lane].x;
        z.y += u * Xs[j][lane].y;
      }
      if (l0 + lane < Ls) xhat[((size_t)c * p + mu) * Ls + l0 + lane] = z;
    }
  }
}

// E[lambda][mu] of node s from its 1-D factors into shared memory.
template <class R>
__device__ void expand_transfer(const R* __restrict__ Etr, int s, int m, int p, R* E) {
  const R* f = Etr + (size_t)s * 3 * m * m;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int lam = t / p, mu = t - lam * p;
    const int lx = lam % m, ly = (lam / m) % m, lz = lam / (m * m);
    const int mx = mu % m, my = (mu / m) % m, mz = mu / (m * m);
    E[t] = f[lx * m + mx] * f[m * m + ly * m + my] * f[2 * m * m + lz * m + mz];
  }
}

// Up-sweep for one level: xhat_r = sum_{s in sons(r)} E_{s,r}^T xhat_s.
// One block per (node, chunk of LC frequencies), so that the top levels with
// few nodes still fill the GPU; both transfer matrices are expanded per
// block and each son's p x LC tile is staged in shared memory by one
// coalesced load.
template <class R>
__global__ void __launch_bounds__(256) k_upsweep(int node0, int Ls, int m, int p,
                                                 const int* __restrict__ son0,
                                                 const int* __restrict__ son1,
                                                 const R* __restrict__ Etr,
                                                 typename Cplx<R>::type* __restrict__ xhat,
                                                 const int* __restrict__ act) {
  using C = typename Cplx<R>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* E = (R*)smraw;                        // 2 x p x p
  C* Xs = (C*)(E + 2 * MAXP * MAXP);       // p x LC
  const int r = node0 + blockIdx.x;
  if (son0[r] < 0) return;
  if (!chunk_active(act, blockIdx.y * LC, Ls)) return;
  const int sons[2] = {son0[r], son1[r]};
  expand_transfer<R>(Etr, sons[0], m, p, E);
  expand_transfer<R>(Etr, sons[1], m, p, E + MAXP * MAXP);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  {
    const int l0 = blockIdx.y * LC;
    C acc[MAXP / 8];
#pragma unroll
    for (int k = 0; k < MAXP / 8; ++k) acc[k] = cz<C>();
    for (int si = 0; si < 2; ++si) {
      const C* xs = xhat + (size_t)sons[si] * p * Ls + l0;
      __syncthreads();
      for (int t = threadIdx.x; t < p * LC; t += blockDim.x) {
        const int lam = t / LC, l = t - lam * LC;
        Xs[t] = (l0 + l < Ls) ? xs[(size_t)lam * Ls + l] : cz<C>();
      }
      __syncthreads();
      const R* Es = E + si * MAXP * MAXP;
      for (int lam = 0; lam < p; ++lam) {
        const C xv = Xs[lam * LC + lane];
#pragma unroll
        for (int k = 0; k < (int)(sizeof(acc) / sizeof(acc[0])); ++k) {
          const int mu = w + 8 * k;
          if (mu < p) {
            const R e = Es[lam * p + mu];
            acc[k].x += e * xv.x;
            acc[k].y += e * xv.y;
          }
        }
      }
    }
    if (l0 + lane < Ls)
#pragma unroll
      for (int k = 0; k < (int)(sizeof(acc) / sizeof(acc[0])); ++k) {
        const int mu = w + 8 * k;
        if (mu < p) xhat[((size_t)r * p + mu) * Ls + l0 + lane] = acc[k];
      }
  }
}

// Coupling: yhat_r[mu][l] += sum_{b=(r,c)} sum_t D_b[t][l] sum_nu C_{b,t}[mu][nu] xhat_c[nu][l].
template <class R>
__global__ void __launch_bounds__(256) k_far_coupling(int Ls, int p, int cap,
                                                      const int* __restrict__ rows,
                                                      const int* __restrict__ rowptr,
                                                      const int2* __restrict__ blocks,
                                                      const int* __restrict__ rank,
                                                      const typename Cplx<R>::type* __restrict__ Cf,
                                                      const typename Cplx<R>::type* __restrict__ Df,
                                                      const typename Cplx<R>::type* __restrict__ xhat,
                                                      typename Cplx<R>::type* __restrict__ yhat) {
  using C = typename Cplx<R>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* Xs = (C*)smraw;               // p x LC
  C* Cs = Xs + MAXP * LC;          // p x p
  __shared__ C Ds[LC];
  const int r = rows[blockIdx.x];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int l0 = 0; l0 < Ls; l0 += LC) {
    C acc[MAXP / 8];
#pragma unroll
    for (int k = 0; k < MAXP / 8; ++k) acc[k] = cz<C>();
    for (int bi = rowptr[r]; bi < rowptr[r + 1]; ++bi) {
      const int c = blocks[bi].y;
      __syncthreads();
      for (int t = threadIdx.x; t < p * LC; t += blockDim.x) {
        const int nu = t / LC, l = t - nu * LC;
        Xs[t] = (l0 + l < Ls) ? xhat[((size_t)c * p + nu) * Ls + l0 + l] : cz<C>();
      }
      const int rk = rank[bi];
      for (int tt = 0; tt < rk; ++tt) {
        __syncthreads();
        const C* Ct = Cf + ((size_t)bi * cap + tt) * p * p;
        for (int t = threadIdx.x; t < p * p; t += blockDim.x) Cs[t] = Ct[t];
        if (threadIdx.x < LC)
          Ds[threadIdx.x] = (l0 + threadIdx.x < Ls) ? Df[((size_t)bi * cap + tt) * Ls + l0 + threadIdx.x]
                                                    : cz<C>();
        __syncthreads();
        const C d = Ds[lane];
#pragma unroll
        for (int k = 0; k < (int)(sizeof(acc) / sizeof(acc[0])); ++k) {
          const int mu = w + 8 * k;
          if (mu < p) {
            C z = cz<C>();
            for (int nu = 0; nu < p; ++nu) cfma(z, Cs[mu * p + nu], Xs[nu * LC + lane]);
            cfma(acc[k], d, z);
          }
        }
      }
    }
    if (l0 + lane < Ls)
#pragma unroll
      for (int k = 0; k < (int)(sizeof(acc) / sizeof(acc[0])); ++k) {
        const int mu = w + 8 * k;
        if (mu < p) {
          C* o = yhat + ((size_t)r * p + mu) * Ls + l0 + lane;
          *o = cadd(*o, acc[k]);
        }
      }
  }
}

// Down-sweep for one level: yhat_s += E_{s,r} yhat_r for every node s of the
// level; one block per (node, chunk of LC frequencies), the parent's p x LC
// tile staged in shared memory.
template <class R>
__global__ void __launch_bounds__(256) k_downsweep(int node0, int Ls, int m, int p,
                                                   const int* __restrict__ parent,
                                                   const R* __restrict__ Etr,
                                                   typename Cplx<R>::type* __restrict__ yhat,
                                                   const int* __restrict__ act) {
  using C = typename Cplx<R>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* E = (R*)smraw;                  // p x p
  C* Ys = (C*)(E + MAXP * MAXP);     // p x LC
  const int s = node0 + blockIdx.x;
  const int r = parent[s];
  if (r < 0) return;
  if (!chunk_active(act, blockIdx.y * LC, Ls)) return;
  expand_transfer<R>(Etr, s, m, p, E);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const C* yr = yhat + (size_t)r * p * Ls;
  {
    const int l0 = blockIdx.y * LC;
    __syncthreads();
    for (int t = threadIdx.x; t < p * LC; t += blockDim.x) {
      const int mu = t / LC, l = t - mu * LC;
      Ys[t] = (l0 + l < Ls) ? yr[(size_t)mu * Ls + l0 + l] : cz<C>();
    }
    __syncthreads();
    if (l0 + lane >= Ls) return;
    for (int lam = w; lam < p; lam += 8) {
      C z = cz<C>();
      for (int mu = 0; mu < p; ++mu) {
        const R e = E[lam * p + mu];
        const C yv = Ys[mu * LC + lane];
        z.x += e * yv.x;
        z.y += e * yv.y;
      }
      C* o = yhat + ((size_t)s * p + lam) * Ls + l0 + lane;
      *o = cadd(*o, z);
    }
  }
}

// y[l][perm[rb + i]] += sum_mu U[rb + i][mu] yhat_r[mu][l] for leaf r; the
// leaf's tile of p x LC coefficients is staged in shared memory.
template <class R>
__global__ void __launch_bounds__(256) k_leaf_backward(int M, int Ls, int p,
                                                       const int* __restrict__ leaves,
                                                       const int* __restrict__ begin,
                                                       const int* __restrict__ end,
                                                       const int* __restrict__ perm,
                                                       const R* __restrict__ U,
                                                       const typename Cplx<R>::type* __restrict__ yhat,
                                                       double2* __restrict__ Y,
                                                       const int* __restrict__ act) {
  using C = typename Cplx<R>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* Us = (R*)smraw;                 // 32 x p
  C* Ys = (C*)(Us + 32 * MAXP);      // p x LC
  const int r = leaves[blockIdx.x];
  const int rb = begin[r], nr = end[r] - rb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < nr * p; t += blockDim.x) Us[t] = U[(size_t)rb * p + t];
  const C* yr = yhat + (size_t)r * p * Ls;
  for (int l0 = 0; l0 < Ls; l0 += LC) {
    if (!chunk_active(act, l0, Ls)) continue;
    __syncthreads();
    for (int t = threadIdx.x; t < p * LC; t += blockDim.x) {
      const int mu = t / LC, l = t - mu * LC;
      Ys[t] = (l0 + l < Ls) ? yr[(size_t)mu * Ls + l0 + l] : cz<C>();
    }
    __syncthreads();
    if (l0 + lane >= Ls) continue;
    for (int i = w; i < nr; i += 8) {
      C z = cz<C>();
      for (int mu = 0; mu < p; ++mu) {
        const R u = Us[i * p + mu];
        const C yv = Ys[mu * LC + lane];
        z.x += u * yv.x;
        z.y += u * yv.y;
      }
      double2* o = Y + (size_t)(l0 + lane) * M + perm[rb + i];
      *o = cadd(*o, to_d(z));
    }
  }
}

template <class R>
static size_t upsweep_smem() {
  return sizeof(R) * 2 * MAXP * MAXP + sizeof(typename Cplx<R>::type) * MAXP * LC;
}
template <class R>
static size_t downsweep_smem() {
  return sizeof(R) * MAXP * MAXP + sizeof(typename Cplx<R>::type) * MAXP * LC;
}
template <class R>
static size_t leaf_backward_smem() {
  return sizeof(R) * 32 * MAXP + sizeof(typename Cplx<R>::type) * MAXP * LC;
}

template <class R>
static size_t coupling_smem(int p) {
  return sizeof(typename Cplx<R>::type) * (MAXP * LC + (size_t)p * p);
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
  CQM_CUDA_TRY(cudaFuncSetAttribute(k_far_coupling<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)coupling_smem<double>(h->p)));
  CQM_CUDA_TRY(cudaFuncSetAttribute(k_far_coupling<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)coupling_smem<float>(h->p)));
#define SWEEP_ATTR(K, F)                                                                          \
  CQM_CUDA_TRY(cudaFuncSetAttribute(K<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                    (int)F<double>()));                                          \
  CQM_CUDA_TRY(cudaFuncSetAttribute(K<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                    (int)F<float>()));
  SWEEP_ATTR(k_upsweep, upsweep_smem)
  SWEEP_ATTR(k_downsweep, downsweep_smem)
  SWEEP_ATTR(k_leaf_backward, leaf_backward_smem)
#undef SWEEP_ATTR
  CQM_TRY(setup_f32_kernels(h));
  return setup_ff(h);
}

// Operator factors in one precision.
template <class R>
struct OpView {
  using C = typename Cplx<R>::type;
  const C *nearC, *nearD, *farC, *farD;
  const R *U, *Etr;
  C *xhat, *yhat;
  const R* Ucol = nullptr;  // column basis of the leaf forward transform (U when null)
};

template <class R>
static int apply_t(cqm_handle* h, const OpView<R>& V, const double2* x, double2* y, bool ff = false,
                   bool far_only = false) {
  using C = typename Cplx<R>::type;
  const int nleaf = (int)h->h_leaves.size(), nfr = (int)h->h_far_rows.size();
  const int M = h->M, Ls = h->Ls, p = h->p, m = h->m;
  cudaStream_t S = h->stream;
  // inside GMRES the inner (FP32) apply skips converged frequencies, and the
  // restart's FP64-accurate apply those whose residual is already final
  const int* act = std::is_same<R, float>::value ? h->inner_active : h->exact_active;
  if (far_only) {
    // the caller has written y
  } else if (ff) {
    CQM_TRY(near_apply_ff(h, x, y));
  } else if (std::is_same<R, float>::value) {
    CQM_TRY(near_apply_f32(h, x, y));
  } else {
    ProfScope ps_(h, (std::is_same<R, double>::value && h->use_f32) ? CQM_K_NEAR_EXACT : CQM_K_NEAR_APPLY);
    k_near_apply<R><<<(unsigned)nleaf, 256, 0, S>>>(
        M, Ls, h->rank_cap, h->d_leaves.p, h->near_rowptr.p, h->near_rc.p, h->near_rank.p,
        h->near_off.p, V.nearC, V.nearD, h->node_begin.p, h->node_end.p, h->perm.p, x, y);
  }
  if (h->n_far > 0) {
    {
      ProfScope ps_(h, CQM_K_LEAF_FORWARD);
      k_leaf_forward<R><<<(unsigned)nleaf, 256, 0, S>>>(M, Ls, p, h->d_leaves.p, h->node_begin.p,
                                                        h->node_end.p, h->perm.p, V.Ucol ? V.Ucol : V.U,
                                                        x, V.xhat, act);
    }
    for (int lv = h->depth - 1; lv >= 0; --lv) {
      const int n0 = h->level_begin[lv], n1 = h->level_begin[lv + 1];
      if (n1 > n0) {
        ProfScope ps_(h, CQM_K_UPSWEEP);
        k_upsweep<R><<<dim3((unsigned)(n1 - n0), (unsigned)((Ls + LC - 1) / LC)), 256, upsweep_smem<R>(), S>>>(n0, Ls, m, p, h->node_son0.p, h->node_son1.p, V.Etr, V.xhat, act);
      }
    }
    cudaMemsetAsync(V.yhat, 0, sizeof(C) * (size_t)h->n_nodes * p * Ls, S);
    if (ff) {
      CQM_TRY(far_coupling_ff(h));
    } else if (std::is_same<R, float>::value) {
      CQM_TRY(far_coupling_f32(h));
    } else {
      ProfScope ps_(h, (std::is_same<R, double>::value && h->use_f32) ? CQM_K_FAR_EXACT : CQM_K_FAR_COUPLING);
      k_far_coupling<R><<<(unsigned)nfr, 256, coupling_smem<R>(p), S>>>(
          Ls, p, h->rank_cap, h->d_far_rows.p, h->far_rowptr.p, h->far_rc.p, h->far_rank.p, V.farC,
          V.farD, V.xhat, V.yhat);
    }
    for (int lv = 1; lv <= h->depth; ++lv) {
      const int n0 = h->level_begin[lv], n1 = h->level_begin[lv + 1];
      if (n1 > n0) {
        ProfScope ps_(h, CQM_K_DOWNSWEEP);
        k_downsweep<R><<<dim3((unsigned)(n1 - n0), (unsigned)((Ls + LC - 1) / LC)), 256, downsweep_smem<R>(), S>>>(n0, Ls, m, p, h->node_parent.p, V.Etr, V.yhat, act);
      }
    }
    {
      ProfScope ps_(h, CQM_K_LEAF_BACKWARD);
      k_leaf_backward<R><<<(unsigned)nleaf, 256, leaf_backward_smem<R>(), S>>>(M, Ls, p, h->d_leaves.p, h->node_begin.p,
                                                         h->node_end.p, h->perm.p, V.U, V.yhat, y, act);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("apply_compressed: ") + cudaGetErrorString(e));
    return CQM_ECUDA;
  }
  return CQM_OK;
}

int far_coupling_generic_f32(cqm_handle* h) {
  ProfScope ps_(h, CQM_K_FAR_COUPLING);
  k_far_coupling<float><<<(unsigned)h->h_far_rows.size(), 256, coupling_smem<float>(h->p), h->stream>>>(
      h->Ls, h->p, h->rank_cap, h->d_far_rows.p, h->far_rowptr.p, h->far_rc.p, h->far_rank.p,
      h->farC_f.p, h->farD_f.p, h->xhat_f.p, h->yhat_f.p);
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

int apply_compressed(cqm_handle* h, const double2* x, double2* y) {
  OpView<double> V{h->nearC.p, h->nearD.p, h->farC.p, h->farD.p, h->Uleaf.p, h->Etr.p,
                   h->xhat.p, h->yhat.p};
  return apply_t<double>(h, V, x, y, h->params.exact_ff != 0);
}

// y += U (S_b) W^T x over the far blocks, the FP64-accurate couplings of the
// handle with the column basis W in place of U (the double layer's far field).
int apply_far_columns(cqm_handle* h, const double* Wleaf, const double2* x, double2* y) {
  OpView<double> V{h->nearC.p, h->nearD.p, h->farC.p, h->farD.p, h->Uleaf.p, h->Etr.p,
                   h->xhat.p, h->yhat.p, Wleaf};
  return apply_t<double>(h, V, x, y, h->params.exact_ff != 0 && h->factors_ff, true);
}

int apply_compressed_f32(cqm_handle* h, const double2* x, double2* y) {
  OpView<float> V{h->nearC_f.p, h->nearD_f.p, h->farC_f.p, h->farD_f.p, h->Uleaf_f.p, h->Etr_f.p,
                  h->xhat_f.p, h->yhat_f.p};
  return apply_t<float>(h, V, x, y);
}

__global__ void k_to_f32c(int64_t n, const double2* __restrict__ a, float2* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void k_to_f32r(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// FP32 copy of 64 x 64 coupling factors, each stored transposed (nu-major):
// dst[tile][nu][mu] = src[tile][mu][nu].  One block per tile.
__global__ void __launch_bounds__(256) k_to_f32c_t64(const double2* __restrict__ src,
                                                     float2* __restrict__ dst) {
  __shared__ float2 T[64][65];
  const size_t base = (size_t)blockIdx.x * 4096;
  for (int e = threadIdx.x; e < 4096; e += blockDim.x) {
    const double2 v = src[base + e];
    T[e & 63][e >> 6] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 4096; e += blockDim.x) dst[base + e] = T[e >> 6][e & 63];
}

// FP32 copy of the operator factors (the inner operator of mixed precision).
// With the tensor-core coupling (m = 4) the far C factors are stored
// transposed, so the coupling kernel reads each row of C coalesced.
int build_f32_copy(cqm_handle* h) {
  auto cc = [&](DArray<double2>& a, DArray<float2>& b) -> int {
    CQM_TRY(b.allocate(h->alloc, std::max<size_t>(1, a.n)));
    if (a.n) {
      ProfScope ps_(h, CQM_K_BASES);
      k_to_f32c<<<grid_for((int64_t)a.n, 256), 256, 0, h->stream>>>((int64_t)a.n, a.p, b.p);
    }
    return CQM_OK;
  };
  auto cr = [&](DArray<double>& a, DArray<float>& b) -> int {
    CQM_TRY(b.allocate(h->alloc, std::max<size_t>(1, a.n)));
    if (a.n) {
      ProfScope ps_(h, CQM_K_BASES);
      k_to_f32r<<<grid_for((int64_t)a.n, 256), 256, 0, h->stream>>>((int64_t)a.n, a.p, b.p);
    }
    return CQM_OK;
  };
  if (!h->expand_near_ok) {  // the expanded near field replaces the factored FP32 near field
    CQM_TRY(cc(h->nearC, h->nearC_f));
    CQM_TRY(cc(h->nearD, h->nearD_f));
  }
  h->farC_f_transposed = h->params.tensor_cores == 2 && h->p == 64;
  if (h->params.tensor_cores == 1 && h->p == 64) {
    CQM_TRY(build_tc2(h));  // bf16 images of the far factors replace their FP32 copy
  } else if (h->farC_f_transposed) {
    CQM_TRY(h->farC_f.allocate(h->alloc, std::max<size_t>(1, h->farC.n)));
    if (h->farC.n >= 4096) {
      ProfScope ps_(h, CQM_K_BASES);
      k_to_f32c_t64<<<(unsigned)(h->farC.n / 4096), 256, 0, h->stream>>>(h->farC.p, h->farC_f.p);
    }
  } else {
    CQM_TRY(cc(h->farC, h->farC_f));
  }
  CQM_TRY(cc(h->farD, h->farD_f));
  CQM_TRY(cr(h->Uleaf, h->Uleaf_f));
  CQM_TRY(cr(h->Etr, h->Etr_f));
  CQM_TRY(h->xhat_f.allocate(h->alloc, (size_t)h->n_nodes * h->p * h->Ls));
  CQM_TRY(h->yhat_f.allocate(h->alloc, (size_t)h->n_nodes * h->p * h->Ls));
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

}  // namespace cqm
