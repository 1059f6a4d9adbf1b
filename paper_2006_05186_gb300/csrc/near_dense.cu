// Expanded near field: after the MACA of the near blocks (Alg. 3, NEAR), every
// near block is expanded per solved frequency, V_l[i][j] = sum_t C_t[i][j] d_t[l]
// (eq. lrfinal), with an FP32 copy.  This file holds the FP64 expansion and
// apply (used without exact_ff) and the FP32 apply of the inner operator; with
// exact_ff the table is formed and applied in float-float (ff.cu).  This is the same
// operator as the factored form (up to rounding); the applies then stream it
// once per product instead of recontracting every rank term, which on this
// GPU turns a compute-bound contraction into an HBM-bound one with Ls / rank
// times fewer operations, and gives the FP32 inner operator entries rounded
// once from FP64 (no cancellation among the rank terms).
//
// Layout: block b holds Ls column-major #r x #c slabs, entry (l, i, j) at
// voff[b] + (l #c + j) #r + i, so that a warp whose lanes are the rows reads
// each column of a block with one coalesced load.
#include <algorithm>
#include <vector>

#include "handle.cuh"

namespace cqm {

namespace {
constexpr int EXP_NF = 8;  // frequencies per expansion block
}

// One block per (near block, chunk of EXP_NF frequencies); a thread per entry.
__global__ void __launch_bounds__(256) k_near_expand(int Ls, int cap, const int2* __restrict__ rc,
                                                     const int* __restrict__ begin,
                                                     const int* __restrict__ end,
                                                     const int64_t* __restrict__ coff,
                                                     const int* __restrict__ rank,
                                                     const double2* __restrict__ C,
                                                     const double2* __restrict__ D,
                                                     const int64_t* __restrict__ voff,
                                                     double2* __restrict__ V, float2* __restrict__ Vf) {
  __shared__ double2 Ds[64][EXP_NF];  // rank <= rank_cap <= 64
  const int nch = (Ls + EXP_NF - 1) / EXP_NF;  // block-major one-dimensional grid
  const int b = (int)(blockIdx.x / nch), l0 = (int)(blockIdx.x - (unsigned)b * nch) * EXP_NF;
  const int2 c2 = rc[b];
  const int nr = end[c2.x] - begin[c2.x], nc = end[c2.y] - begin[c2.y];
  const int rk = rank[b], nf = min(EXP_NF, Ls - l0);
  for (int t = threadIdx.x; t < rk * EXP_NF; t += blockDim.x) {
    const int tt = t / EXP_NF, f = t - tt * EXP_NF;
    Ds[tt][f] = f < nf ? D[((size_t)b * cap + tt) * Ls + l0 + f] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
    const int i = e / nc, j = e - i * nc;
    double2 acc[EXP_NF];
#pragma unroll
    for (int f = 0; f < EXP_NF; ++f) acc[f] = make_double2(0.0, 0.0);
    for (int tt = 0; tt < rk; ++tt) {
      const double2 c = C[coff[b] + (size_t)tt * nr * nc + e];
#pragma unroll
      for (int f = 0; f < EXP_NF; ++f) acc[f] = cadd(acc[f], cmul(c, Ds[tt][f]));
    }
    for (int f = 0; f < nf; ++f) {
      const size_t o = voff[b] + ((size_t)(l0 + f) * nc + j) * nr + i;
      V[o] = acc[f];
      Vf[o] = make_float2((float)acc[f].x, (float)acc[f].y);
    }
  }
}

// y_l[perm[rb + i]] = sum over the near blocks (r, c) of leaf row r of
// sum_j V_l[i][j] x_l[perm[cb + j]]: one warp per (leaf row, frequency), lanes
// over the rows i, blocks in their stored order, each block's sum added to an
// FP64 total (the FP64 table; the double layer's table).  Overwrites y on the
// rows.
template <class VT>
__global__ void __launch_bounds__(256) k_near_dense(int M, int Ls, const int* __restrict__ leaves,
                                                    const int* __restrict__ rowptr,
                                                    const int2* __restrict__ rc,
                                                    const int* __restrict__ begin,
                                                    const int* __restrict__ end,
                                                    const int* __restrict__ perm,
                                                    const int64_t* __restrict__ voff,
                                                    const VT* __restrict__ V,
                                                    const double2* __restrict__ x,
                                                    double2* __restrict__ y) {
  using C = VT;  // float2 (FP32 accumulation) or double2 (FP64)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int l = blockIdx.x * 8 + w;
  if (l >= Ls) return;
  const int r = leaves[blockIdx.y];
  const int rb = begin[r], nr = end[r] - rb;
  const double2* xl = x + (size_t)l * M;
  double2 acc = make_double2(0.0, 0.0);
  for (int bi = rowptr[r]; bi < rowptr[r + 1]; ++bi) {
    const int c = rc[bi].y;
    const int cb = begin[c], nc = end[c] - cb;
    // lane j fetches x_l at column j of the block; broadcast below
    const C xj = lane < nc ? to_c(xl[perm[cb + lane]], (C*)0) : cz<C>();
    const VT* Vb = V + voff[bi] + (size_t)l * nc * nr;
    C bacc = cz<C>();
    // columns in groups of 8: the group's loads are issued together
    for (int j0 = 0; j0 < nc; j0 += 8) {
      C v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = (lane < nr && j0 + u < nc) ? Vb[(size_t)(j0 + u) * nr + lane] : cz<C>();
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        C xv;
        xv.x = __shfl_sync(0xffffffffu, xj.x, (j0 + u) & 31);
        xv.y = __shfl_sync(0xffffffffu, xj.y, (j0 + u) & 31);
        bacc.x = fma(v[u].x, xv.x, fma(-v[u].y, xv.y, bacc.x));
        bacc.y = fma(v[u].x, xv.y, fma(v[u].y, xv.x, bacc.y));
      }
    }
    acc = cadd(acc, to_d(bacc));
  }
  if (lane < nr) y[(size_t)l * M + perm[rb + lane]] = acc;
}

// The same for the FP32 table with an FP32 copy of x (converted once per
// apply, not once per block that reads it): each block's sum in FP32, the
// row's total over the blocks in compensated FP32 (TwoSum, ~48 bits, the
// accuracy of the FP64 total of the kernel above without its FP64
// instructions).  Overwrites y on the rows.
__global__ void __launch_bounds__(256) k_near_dense_f32x(int M, int Ls, const int* __restrict__ leaves,
                                                         const int* __restrict__ rowptr,
                                                         const int2* __restrict__ rc,
                                                         const int* __restrict__ begin,
                                                         const int* __restrict__ end,
                                                         const int* __restrict__ perm,
                                                         const int64_t* __restrict__ voff,
                                                         const float2* __restrict__ V,
                                                         const float2* __restrict__ x,
                                                         double2* __restrict__ y,
                                                         const int* __restrict__ act) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int l = blockIdx.x * 8 + w;
  if (l >= Ls || (act && !act[l])) return;  // act: frequencies still iterating (may be null)
  const int r = leaves[blockIdx.y];
  const int rb = begin[r], nr = end[r] - rb;
  const float2* xl = x + (size_t)l * M;
  float hr = 0.f, lr = 0.f, hi = 0.f, li = 0.f;  // compensated totals (re, im)
  for (int bi = rowptr[r]; bi < rowptr[r + 1]; ++bi) {
    const int c = rc[bi].y;
    const int cb = begin[c], nc = end[c] - cb;
    const float2 xj = lane < nc ? xl[perm[cb + lane]] : make_float2(0.f, 0.f);
    const float2* Vb = V + voff[bi] + (size_t)l * nc * nr;
    float2 bacc = make_float2(0.f, 0.f);
    for (int j0 = 0; j0 < nc; j0 += 8) {
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = (lane < nr && j0 + u < nc) ? Vb[(size_t)(j0 + u) * nr + lane] : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        float2 xv;
        xv.x = __shfl_sync(0xffffffffu, xj.x, (j0 + u) & 31);
        xv.y = __shfl_sync(0xffffffffu, xj.y, (j0 + u) & 31);
        bacc.x = fmaf(v[u].x, xv.x, fmaf(-v[u].y, xv.y, bacc.x));
        bacc.y = fmaf(v[u].x, xv.y, fmaf(v[u].y, xv.x, bacc.y));
      }
    }
    float s, e;
    s = __fadd_rn(hr, bacc.x);  // TwoSum
    e = __fadd_rn(__fsub_rn(hr, __fsub_rn(s, __fsub_rn(s, hr))), __fsub_rn(bacc.x, __fsub_rn(s, hr)));
    hr = s;
    lr = __fadd_rn(lr, e);
    s = __fadd_rn(hi, bacc.y);
    e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, __fsub_rn(s, hi))), __fsub_rn(bacc.y, __fsub_rn(s, hi)));
    hi = s;
    li = __fadd_rn(li, e);
  }
  if (lane < nr)
    y[(size_t)l * M + perm[rb + lane]] = make_double2((double)hr + (double)lr, (double)hi + (double)li);
}

__global__ void k_x_to_f32(int64_t n, const double2* __restrict__ a, float2* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

int build_near_expanded(cqm_handle* h) {
  const int nb = h->n_near;
  h->h_nearV_off.assign(nb + 1, 0);
  for (int b = 0; b < nb; ++b) {
    const int2 rc = h->h_near[b];
    h->h_nearV_off[b + 1] = h->h_nearV_off[b] + (int64_t)h->Ls * (h->h_end[rc.x] - h->h_begin[rc.x]) *
                                                     (h->h_end[rc.y] - h->h_begin[rc.y]);
  }
  const size_t n = (size_t)std::max<int64_t>(1, h->h_nearV_off[nb]);
  CQM_TRY(h->nearV_off.allocate(h->alloc, nb + 1));
  CQM_TRY(h->nearV.allocate(h->alloc, n));
  CQM_TRY(h->nearV_f.allocate(h->alloc, n));
  CQM_CUDA_TRY(cudaMemcpyAsync(h->nearV_off.p, h->h_nearV_off.data(), sizeof(int64_t) * (nb + 1),
                               cudaMemcpyHostToDevice, h->stream));
  if (nb > 0) {
    ProfScope ps_(h, CQM_K_EXPAND);
    const unsigned g = (unsigned)((h->Ls + EXP_NF - 1) / EXP_NF) * (unsigned)nb;
    k_near_expand<<<g, 256, 0, h->stream>>>(h->Ls, h->rank_cap, h->near_rc.p, h->node_begin.p,
                                            h->node_end.p, h->near_off.p, h->near_rank.p, h->nearC.p,
                                            h->nearD.p, h->nearV_off.p, h->nearV.p, h->nearV_f.p);
  }
  CQM_CHECK_LAUNCH();
  h->near_expanded = true;
  return CQM_OK;
}

// y = (table) x over the near field for a table of the layout above (the
// double layer's near field), FP64.
int near_apply_table(cqm_handle* h, const double2* T, const int64_t* off, const double2* x, double2* y) {
  const int nleaf = (int)h->h_leaves.size();
  if (nleaf == 0) return CQM_OK;
  dim3 g((unsigned)((h->Ls + 7) / 8), (unsigned)nleaf);
  k_near_dense<double2><<<g, 256, 0, h->stream>>>(h->M, h->Ls, h->d_leaves.p, h->near_rowptr.p,
                                                  h->near_rc.p, h->node_begin.p, h->node_end.p,
                                                  h->perm.p, off, T, x, y);
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

int near_apply_expanded(cqm_handle* h, const double2* x, double2* y, bool fp64) {
  const int nleaf = (int)h->h_leaves.size();
  if (nleaf == 0) return CQM_OK;
  dim3 g((unsigned)((h->Ls + 7) / 8), (unsigned)nleaf);
  if (!fp64) {
    const int64_t n = (int64_t)h->Ls * h->M;
    if (h->x32.n < (size_t)n) CQM_TRY(h->x32.allocate(h->alloc, (size_t)n));
    k_x_to_f32<<<grid_for(n, 256), 256, 0, h->stream>>>(n, x, h->x32.p);
    k_near_dense_f32x<<<g, 256, 0, h->stream>>>(h->M, h->Ls, h->d_leaves.p, h->near_rowptr.p, h->near_rc.p,
                                                h->node_begin.p, h->node_end.p, h->perm.p, h->nearV_off.p,
                                                h->nearV_f.p, h->x32.p, y, h->inner_active);
    CQM_CHECK_LAUNCH();
    return CQM_OK;
  }
  k_near_dense<double2><<<g, 256, 0, h->stream>>>(h->M, h->Ls, h->d_leaves.p, h->near_rowptr.p,
                                                  h->near_rc.p, h->node_begin.p, h->node_end.p,
                                                  h->perm.p, h->nearV_off.p, h->nearV.p, x, y);
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

}  // namespace cqm
