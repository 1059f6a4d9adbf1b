// FP64-accurate application of the compressed operator in float-float
// arithmetic on the FP32 pipes (GB300 runs FP32 about 60x faster than FP64).
// A float-float number is an unevaluated sum hi + lo of two floats; products
// use the FMA-based exact product (the error of hi*hi is fma(a, b, -a*b)) and
// sums Knuth's error-free TwoSum, which together keep about 48 significant
// bits.  The near-field and far-field coupling contractions (the bulk of the
// flops of eq. lrfinal) run this way; the H^2 transforms, which are cheap,
// stay in FP64.  Inputs and outputs are FP64.  The C factors are converted to
// float-float pairs once at setup (factors_to_ff).  This file also forms the
// expanded near field and far couplings in float-float (V_l = sum_t C_t d_t(l)
// per block and frequency) and streams them in the FP64-accurate apply; the
// factored contractions remain for tables that are not expanded.
#include <algorithm>
#include <vector>

#include "handle.cuh"

namespace cqm {

struct ffc {  // complex float-float: (re_hi, im_hi, re_lo, im_lo)
  float rh, ih, rl, il;
};

__device__ __forceinline__ ffc ffc_zero() { return {0.f, 0.f, 0.f, 0.f}; }

__device__ __forceinline__ ffc ffc_from(double2 v) {
  const float rh = (float)v.x, ih = (float)v.y;
  return {rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih)};
}

__device__ __forceinline__ double2 ffc_to(const ffc& a) {
  return make_double2((double)a.rh + (double)a.rl, (double)a.ih + (double)a.il);
}

// (sh, sl) += (ah, al) * (bh, bl)
__device__ __forceinline__ void ff_mac(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);  // exact low part of ah*bh
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float t = __fadd_rn(sh, p);  // TwoSum(sh, p)
  const float bb = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  sl = __fadd_rn(sl, __fadd_rn(err, e));
  sh = t;
}

// z += a * b (complex)
__device__ __forceinline__ void ffc_mac(ffc& z, const ffc& a, const ffc& b) {
  ff_mac(z.rh, z.rl, a.rh, a.rl, b.rh, b.rl);
  ff_mac(z.rh, z.rl, -a.ih, -a.il, b.ih, b.il);
  ff_mac(z.ih, z.il, a.rh, a.rl, b.ih, b.il);
  ff_mac(z.ih, z.il, a.ih, a.il, b.rh, b.rl);
}

// keep |lo| below half an ulp of hi (FastTwoSum)
__device__ __forceinline__ void ffc_renorm(ffc& z) {
  float t = __fadd_rn(z.rh, z.rl);
  z.rl = __fsub_rn(z.rl, __fsub_rn(t, z.rh));
  z.rh = t;
  t = __fadd_rn(z.ih, z.il);
  z.il = __fsub_rn(z.il, __fsub_rn(t, z.ih));
  z.ih = t;
}

constexpr int LCF = 32;
constexpr int PMAX = 64;

// Near field in float-float: one block per leaf row cluster.
__global__ void __launch_bounds__(256) k_near_apply_ff(
    int M, int Ls, int cap, const int4* __restrict__ items, const int2* __restrict__ blocks,
    const int* __restrict__ rank, const int64_t* __restrict__ off, const ffc* __restrict__ Cn,
    const double2* __restrict__ Dn, const int* __restrict__ begin, const int* __restrict__ end,
    const int* __restrict__ perm, const double2* __restrict__ X, double2* __restrict__ part) {
  __shared__ ffc Xs[32][LCF];
  __shared__ ffc Cs[32 * 32];
  __shared__ ffc Ds[LCF];
  const int4 itm = items[blockIdx.x];  // (leaf row, first block, end block, -)
  const int r = itm.x;
  const int rb = begin[r], nr = end[r] - rb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int l0 = 0; l0 < Ls; l0 += LCF) {
    ffc acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = ffc_zero();
    for (int bi = itm.y; bi < itm.z; ++bi) {
      const int c = blocks[bi].y;
      const int cb = begin[c], nc = end[c] - cb;
      __syncthreads();
      for (int t = threadIdx.x; t < nc * LCF; t += blockDim.x) {
        const int j = t / LCF, l = t - j * LCF;
        Xs[j][l] = (l0 + l < Ls) ? ffc_from(X[(size_t)(l0 + l) * M + perm[cb + j]]) : ffc_zero();
      }
      const int rk = rank[bi];
      for (int tt = 0; tt < rk; ++tt) {
        __syncthreads();
        const ffc* Ct = Cn + off[bi] + (size_t)tt * nr * nc;
        for (int t = threadIdx.x; t < nr * nc; t += blockDim.x) Cs[t] = Ct[t];
        if (threadIdx.x < LCF)
          Ds[threadIdx.x] = (l0 + threadIdx.x < Ls)
                                ? ffc_from(Dn[((size_t)bi * cap + tt) * Ls + l0 + threadIdx.x])
                                : ffc_zero();
        __syncthreads();
        const ffc d = Ds[lane];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int i = w + 8 * k;
          if (i < nr) {
            ffc z = ffc_zero();
            for (int j = 0; j < nc; ++j) ffc_mac(z, Cs[i * nc + j], Xs[j][lane]);
            ffc_renorm(z);
            ffc_mac(acc[k], d, z);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) ffc_renorm(acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = w + 8 * k;
      if (i < nr && l0 + lane < Ls) part[((size_t)blockIdx.x * 32 + i) * Ls + l0 + lane] = ffc_to(acc[k]);
    }
  }
}

// Y[l][perm[rb + i]] = sum of leaf row k's item tiles, in item order (FP64).
__global__ void k_near_reduce_d(int M, int Ls, const int* __restrict__ leaves,
                                const int* __restrict__ item_ptr, const int* __restrict__ begin,
                                const int* __restrict__ end, const int* __restrict__ perm,
                                const double2* __restrict__ part, double2* __restrict__ Y) {
  const int k = blockIdx.x;
  const int r = leaves[k];
  const int rb = begin[r], nr = end[r] - rb;
  for (int e = threadIdx.x; e < nr * Ls; e += blockDim.x) {
    const int i = e / Ls, l = e - i * Ls;
    double2 a = make_double2(0.0, 0.0);
    for (int it = item_ptr[k]; it < item_ptr[k + 1]; ++it) a = cadd(a, part[((size_t)it * 32 + i) * Ls + l]);
    Y[(size_t)l * M + perm[rb + i]] = a;
  }
}

// yhat_r += sum of row k's item tiles, in item order (FP64).
__global__ void k_far_reduce_d(int Ls, int p, const int* __restrict__ rows,
                               const int* __restrict__ item_ptr, const double2* __restrict__ part,
                               double2* __restrict__ yhat) {
  const int k = blockIdx.x;
  const int r = rows[k];
  for (int e = threadIdx.x; e < p * Ls; e += blockDim.x) {
    double2 a = make_double2(0.0, 0.0);
    for (int it = item_ptr[k]; it < item_ptr[k + 1]; ++it) a = cadd(a, part[(size_t)it * p * Ls + e]);
    double2* o = yhat + (size_t)r * p * Ls + e;
    *o = cadd(*o, a);
  }
}

// Far coupling in float-float, one block per work item (a row cluster and a
// run of its far blocks): part = sum_b sum_t d_t (.) (C_{b,t} xhat_c).
// Full passes of LCF frequency columns give each lane one column and each
// warp every 8th row; the Ls mod LCF remaining columns are done in one tail
// pass that gives each thread whole (row, column) outputs instead, so the
// ragged end costs a fraction of a pass.  Every output is summed in the same
// order either way.  The staged C has row stride p + 1, which keeps the tail's
// per-lane rows in distinct banks.
__global__ void __launch_bounds__(256) k_far_coupling_ff(int Ls, int p, int cap,
                                                         const int4* __restrict__ items,
                                                         const int2* __restrict__ blocks,
                                                         const int* __restrict__ rank,
                                                         const ffc* __restrict__ Cf,
                                                         const double2* __restrict__ Df,
                                                         const double2* __restrict__ xhat,
                                                         double2* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  ffc* Xs = (ffc*)smraw;        // p x LCF
  ffc* Cs = Xs + PMAX * LCF;    // p x (p + 1)
  __shared__ ffc Ds[LCF];
  const int cs = p + 1;
  const int4 itm = items[blockIdx.x];  // (row, first block, end block, -)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nfull = Ls / LCF, rem = Ls - nfull * LCF;
  auto stage_c = [&](int bi, int tt, int l0, int ncol) {
    const ffc* Ct = Cf + ((size_t)bi * cap + tt) * p * p;
    for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
      const int mu = t / p;
      Cs[t + mu] = Ct[t];
    }
    if (threadIdx.x < ncol) Ds[threadIdx.x] = ffc_from(Df[((size_t)bi * cap + tt) * Ls + l0 + threadIdx.x]);
  };
  for (int pass = 0; pass < nfull; ++pass) {
    const int l0 = pass * LCF;
    ffc acc[PMAX / 8];
#pragma unroll
    for (int k = 0; k < PMAX / 8; ++k) acc[k] = ffc_zero();
    for (int bi = itm.y; bi < itm.z; ++bi) {
      const int c = blocks[bi].y;
      __syncthreads();
      for (int t = threadIdx.x; t < p * LCF; t += blockDim.x) {
        const int nu = t / LCF, l = t - nu * LCF;
        Xs[t] = ffc_from(xhat[((size_t)c * p + nu) * Ls + l0 + l]);
      }
      const int rk = rank[bi];
      for (int tt = 0; tt < rk; ++tt) {
        __syncthreads();
        stage_c(bi, tt, l0, LCF);
        __syncthreads();
        const ffc d = Ds[lane];
#pragma unroll
        for (int k = 0; k < (int)(sizeof(acc) / sizeof(acc[0])); ++k) {
          const int mu = w + 8 * k;
          if (mu < p) {
            ffc z = ffc_zero();
            for (int nu = 0; nu < p; ++nu) ffc_mac(z, Cs[mu * cs + nu], Xs[nu * LCF + lane]);
            ffc_renorm(z);
            ffc_mac(acc[k], d, z);
            ffc_renorm(acc[k]);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < (int)(sizeof(acc) / sizeof(acc[0])); ++k) {
      const int mu = w + 8 * k;
      if (mu < p) part[((size_t)blockIdx.x * p + mu) * Ls + l0 + lane] = ffc_to(acc[k]);
    }
  }
  if (rem > 0) {
    // tail: output o = mu * rem + j (column l0 + j), outputs tid + 256 k
    constexpr int KT = PMAX * LCF / 256;
    const int l0 = nfull * LCF, nout = p * rem;
    ffc acc[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) acc[k] = ffc_zero();
    for (int bi = itm.y; bi < itm.z; ++bi) {
      const int c = blocks[bi].y;
      __syncthreads();
      for (int t = threadIdx.x; t < p * rem; t += blockDim.x) {
        const int nu = t / rem, l = t - nu * rem;
        Xs[nu * LCF + l] = ffc_from(xhat[((size_t)c * p + nu) * Ls + l0 + l]);
      }
      const int rk = rank[bi];
      for (int tt = 0; tt < rk; ++tt) {
        __syncthreads();
        stage_c(bi, tt, l0, rem);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KT; ++k) {
          const int o = threadIdx.x + 256 * k;
          if (o < nout) {
            const int mu = o / rem, j = o - mu * rem;
            ffc z = ffc_zero();
            for (int nu = 0; nu < p; ++nu) ffc_mac(z, Cs[mu * cs + nu], Xs[nu * LCF + j]);
            ffc_renorm(z);
            ffc_mac(acc[k], Ds[j], z);
            ffc_renorm(acc[k]);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KT; ++k) {
      const int o = threadIdx.x + 256 * k;
      if (o < nout) {
        const int mu = o / rem, j = o - mu * rem;
        part[((size_t)blockIdx.x * p + mu) * Ls + l0 + j] = ffc_to(acc[k]);
      }
    }
  }
}

// In place: each complex FP64 factor entry becomes its float-float pair
// (same 16 bytes), the form the contractions above stage.
__global__ void k_factors_to_ff(int64_t n, double2* __restrict__ a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double2 v = a[i];
    ((ffc*)a)[i] = ffc_from(v);
  }
}

// The same for the far factors, slot by slot (block b, term t: one CTA);
// the slots past a block's rank hold no factor and are skipped.
__global__ void __launch_bounds__(256) k_far_factors_to_ff(int cap, int pp, const int* __restrict__ rank,
                                                           double2* __restrict__ a) {
  const int b = (int)(blockIdx.x / cap), t = (int)(blockIdx.x - (unsigned)b * cap);
  if (t >= rank[b]) return;
  double2* s = a + (size_t)blockIdx.x * pp;
  for (int e = threadIdx.x; e < pp; e += blockDim.x) {
    const double2 v = s[e];
    ((ffc*)s)[e] = ffc_from(v);
  }
}

int factors_to_ff(cqm_handle* h) {
  ProfScope ps_(h, CQM_K_BASES);
  if (h->nearC.n)
    k_factors_to_ff<<<grid_for((int64_t)h->nearC.n, 256), 256, 0, h->stream>>>((int64_t)h->nearC.n, h->nearC.p);
  if (h->farC.n && h->n_far > 0)
    k_far_factors_to_ff<<<(unsigned)h->n_far * (unsigned)h->rank_cap, 256, 0, h->stream>>>(
        h->rank_cap, h->p * h->p, h->far_rank.p, h->farC.p);
  CQM_CHECK_LAUNCH();
  h->factors_ff = true;
  return CQM_OK;
}

static size_t coupling_smem_ff(int p) { return sizeof(ffc) * (PMAX * LCF + (size_t)p * (p + 1)); }

int setup_ff(cqm_handle* h) {
  CQM_CUDA_TRY(cudaFuncSetAttribute(k_far_coupling_ff, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)coupling_smem_ff(h->p)));
  return CQM_OK;
}

int near_apply_ff(cqm_handle* h, const double2* x, double2* y) {
  ProfScope ps_(h, CQM_K_NEAR_EXACT);
  if (h->near_expanded) return h->nearV_ff ? near_apply_expanded_ff(h, x, y) : near_apply_expanded(h, x, y, true);
  k_near_apply_ff<<<(unsigned)h->n_near_items, 256, 0, h->stream>>>(
      h->M, h->Ls, h->rank_cap, h->near_items.p, h->near_rc.p, h->near_rank.p, h->near_off.p,
      (const ffc*)h->nearC.p, h->nearD.p, h->node_begin.p, h->node_end.p, h->perm.p, x, h->part_d.p);
  k_near_reduce_d<<<(unsigned)h->h_leaves.size(), 256, 0, h->stream>>>(
      h->M, h->Ls, h->d_leaves.p, h->near_item_ptr.p, h->node_begin.p, h->node_end.p, h->perm.p,
      h->part_d.p, y);
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

int far_coupling_ff(cqm_handle* h) {
  ProfScope ps_(h, CQM_K_FAR_EXACT);
  if (h->far_expanded) return far_apply_expanded_ff(h);
  k_far_coupling_ff<<<(unsigned)h->n_far_items, 256, coupling_smem_ff(h->p), h->stream>>>(
      h->Ls, h->p, h->rank_cap, h->far_items.p, h->far_rc.p, h->far_rank.p, (const ffc*)h->farC.p, h->farD.p,
      h->xhat.p, h->part_d.p);
  k_far_reduce_d<<<(unsigned)h->h_far_rows.size(), 256, 0, h->stream>>>(
      h->Ls, h->p, h->d_far_rows.p, h->far_item_ptr.p, h->part_d.p, h->yhat.p);
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

}  // namespace cqm

namespace cqm {

// Expanded far couplings for the FP64-accurate apply: S_b(l) = sum_t C_t d_t(l)
// (eq. lrfinal) per far block and solved frequency, as float-float pairs,
// stored column-major per frequency: entry (l, mu, nu) of block b at
// (b Ls + l) p^2 + nu p + mu.  One block per (far block, chunk of FAR_NF
// frequencies), a thread per entry.
namespace {
constexpr int FAR_NF = 8;
}

__global__ void __launch_bounds__(256) k_far_expand_ff(int Ls, int p, int cap, const int* __restrict__ rank,
                                                       const ffc* __restrict__ Cf, const double2* __restrict__ Df,
                                                       ffc* __restrict__ S) {
  __shared__ ffc Ds[64][FAR_NF];  // rank <= rank_cap <= 64
  // one-dimensional grid, block-major: the frequency chunks of one block are
  // consecutive blocks and share its factors in L2
  const int nch = (Ls + FAR_NF - 1) / FAR_NF;
  const int b = (int)(blockIdx.x / nch), l0 = (int)(blockIdx.x - (unsigned)b * nch) * FAR_NF;
  const int rk = rank[b], nf = min(FAR_NF, Ls - l0);
  for (int t = threadIdx.x; t < rk * FAR_NF; t += blockDim.x) {
    const int tt = t / FAR_NF, f = t - tt * FAR_NF;
    Ds[tt][f] = f < nf ? ffc_from(Df[((size_t)b * cap + tt) * Ls + l0 + f]) : ffc_zero();
  }
  __syncthreads();
  const int pp = p * p;
  // 16 x 16 tiles of (mu, nu), nu fastest across the threads: a warp reads
  // two runs of 16 consecutive factor entries (row-major C_t) and writes 16
  // pairs of consecutive table entries (column-major S); blockDim.x = 256
  const int nt16 = (p + 15) / 16;
  for (int tile = 0; tile < nt16 * nt16; ++tile) {
    const int mu = (tile / nt16) * 16 + (int)(threadIdx.x >> 4);
    const int nu = (tile % nt16) * 16 + (int)(threadIdx.x & 15);
    if (mu >= p || nu >= p) continue;
    ffc acc[FAR_NF];
#pragma unroll
    for (int f = 0; f < FAR_NF; ++f) acc[f] = ffc_zero();
    for (int tt = 0; tt < rk; ++tt) {
      const ffc c = Cf[((size_t)b * cap + tt) * pp + (size_t)mu * p + nu];
#pragma unroll
      for (int f = 0; f < FAR_NF; ++f) ffc_mac(acc[f], c, Ds[tt][f]);
    }
    for (int f = 0; f < nf; ++f) {
      ffc_renorm(acc[f]);
      S[((size_t)b * Ls + l0 + f) * pp + (size_t)nu * p + mu] = acc[f];
    }
  }
}

// yhat_r(l)[mu] = sum over the far blocks (r, c) of row r of
// sum_nu S_b(l)[mu][nu] xhat_c(l)[nu], in float-float: one warp per (row
// cluster, frequency), lane k owns rows k and k + 32, blocks in their stored
// order.  Overwrites yhat on the row.
__global__ void __launch_bounds__(256) k_far_dense_ff(int Ls, int p, int nrows, const int* __restrict__ rows,
                                                      const int* __restrict__ rowptr,
                                                      const int2* __restrict__ rc,
                                                      const ffc* __restrict__ S,
                                                      const double2* __restrict__ xhat,
                                                      double2* __restrict__ yhat,
                                                      const int* __restrict__ act) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int l = blockIdx.x * 8 + w;
  if (l >= Ls || (act && !act[l])) return;  // act: frequencies to compute (may be null)
  const int r = rows[blockIdx.y];
  const int pp = p * p;
  ffc acc0 = ffc_zero(), acc1 = ffc_zero();
  const bool has0 = lane < p, has1 = lane + 32 < p;
  for (int bi = rowptr[r]; bi < rowptr[r + 1]; ++bi) {
    const int c = rc[bi].y;
    const double2* xc = xhat + (size_t)c * p * Ls + l;
    const ffc x0 = has0 ? ffc_from(xc[(size_t)lane * Ls]) : ffc_zero();
    const ffc x1 = has1 ? ffc_from(xc[(size_t)(lane + 32) * Ls]) : ffc_zero();
    const ffc* Sb = S + ((size_t)bi * Ls + l) * pp;
    // nu in groups of 4: the group's loads are issued together
    for (int n0 = 0; n0 < p; n0 += 4) {
      ffc s0[4], s1[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int nu = n0 + u;
        s0[u] = (has0 && nu < p) ? Sb[(size_t)nu * p + lane] : ffc_zero();
        s1[u] = (has1 && nu < p) ? Sb[(size_t)nu * p + lane + 32] : ffc_zero();
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int nu = n0 + u;
        if (nu < p) {
          const ffc src = nu < 32 ? x0 : x1;
          ffc xv;
          xv.rh = __shfl_sync(0xffffffffu, src.rh, nu & 31);
          xv.ih = __shfl_sync(0xffffffffu, src.ih, nu & 31);
          xv.rl = __shfl_sync(0xffffffffu, src.rl, nu & 31);
          xv.il = __shfl_sync(0xffffffffu, src.il, nu & 31);
          if (has0) ffc_mac(acc0, s0[u], xv);
          if (has1) ffc_mac(acc1, s1[u], xv);
          if ((nu & 15) == 15) {
            ffc_renorm(acc0);
            ffc_renorm(acc1);
          }
        }
      }
    }
    ffc_renorm(acc0);
    ffc_renorm(acc1);
  }
  double2* yr = yhat + (size_t)r * p * Ls + l;
  if (has0) yr[(size_t)lane * Ls] = ffc_to(acc0);
  if (has1) yr[(size_t)(lane + 32) * Ls] = ffc_to(acc1);
}

int build_far_expanded(cqm_handle* h) {
  if (h->n_far == 0 || !h->factors_ff) return CQM_OK;
  const size_t n = (size_t)h->n_far * h->Ls * h->p * h->p;
  size_t free_b = 0, total_b = 0;
  CQM_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  if (n * sizeof(ffc) > total_b / 10 * 4) return CQM_OK;  // over 40% of the device: stay factored
  if (h->farS.allocate(h->alloc, n) != CQM_OK) {
    set_last_error("");
    return CQM_OK;  // the allocation did not fit: stay factored
  }
  {
    ProfScope ps_(h, CQM_K_EXPAND);
    const unsigned g = (unsigned)((h->Ls + FAR_NF - 1) / FAR_NF) * (unsigned)h->n_far;
    k_far_expand_ff<<<g, 256, 0, h->stream>>>(h->Ls, h->p, h->rank_cap, h->far_rank.p,
                                               (const ffc*)h->farC.p, h->farD.p, (ffc*)h->farS.p);
  }
  CQM_CHECK_LAUNCH();
  h->far_expanded = true;
  return CQM_OK;
}

int far_apply_expanded_ff(cqm_handle* h) {
  const int nfr = (int)h->h_far_rows.size();
  if (nfr == 0) return CQM_OK;
  dim3 g((unsigned)((h->Ls + 7) / 8), (unsigned)nfr);
  k_far_dense_ff<<<g, 256, 0, h->stream>>>(h->Ls, h->p, nfr, h->d_far_rows.p, h->far_rowptr.p,
                                            h->far_rc.p, (const ffc*)h->farS.p, h->xhat.p, h->yhat.p,
                                            h->exact_active);
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

}  // namespace cqm

namespace cqm {

// Expanded near field in float-float, for the FP64-accurate apply: the same
// table as the FP64 expansion (block b, frequency l, entry (i, j) at
// nearV_off[b] + (l #c + j) #r + i) with float-float pairs in nearV and their
// high parts in nearV_f, formed on the FP32 pipes from the float-float C
// factors.  One block per (near block, chunk of FAR_NF frequencies).
__global__ void __launch_bounds__(256) k_near_expand_ff(int Ls, int cap, const int2* __restrict__ rc,
                                                        const int* __restrict__ begin,
                                                        const int* __restrict__ end,
                                                        const int64_t* __restrict__ coff,
                                                        const int* __restrict__ rank,
                                                        const ffc* __restrict__ C,
                                                        const double2* __restrict__ D,
                                                        const int64_t* __restrict__ voff,
                                                        ffc* __restrict__ V, float2* __restrict__ Vf) {
  __shared__ ffc Ds[64][FAR_NF];  // rank <= rank_cap <= 64
  const int nch = (Ls + FAR_NF - 1) / FAR_NF;  // block-major one-dimensional grid
  const int b = (int)(blockIdx.x / nch), l0 = (int)(blockIdx.x - (unsigned)b * nch) * FAR_NF;
  const int2 c2 = rc[b];
  const int nr = end[c2.x] - begin[c2.x], nc = end[c2.y] - begin[c2.y];
  const int rk = rank[b], nf = min(FAR_NF, Ls - l0);
  for (int t = threadIdx.x; t < rk * FAR_NF; t += blockDim.x) {
    const int tt = t / FAR_NF, f = t - tt * FAR_NF;
    Ds[tt][f] = f < nf ? ffc_from(D[((size_t)b * cap + tt) * Ls + l0 + f]) : ffc_zero();
  }
  __syncthreads();
  // thread e -> (j, i) with i fastest: consecutive threads write consecutive
  // entries of the column-major table
  for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
    const int j = e / nr, i = e - j * nr;
    ffc acc[FAR_NF];
#pragma unroll
    for (int f = 0; f < FAR_NF; ++f) acc[f] = ffc_zero();
    for (int tt = 0; tt < rk; ++tt) {
      const ffc c = C[coff[b] + (size_t)tt * nr * nc + (size_t)i * nc + j];
#pragma unroll
      for (int f = 0; f < FAR_NF; ++f) ffc_mac(acc[f], c, Ds[tt][f]);
    }
    for (int f = 0; f < nf; ++f) {
      ffc_renorm(acc[f]);
      const size_t o = voff[b] + ((size_t)(l0 + f) * nc + j) * nr + i;
      V[o] = acc[f];
      Vf[o] = make_float2(acc[f].rh, acc[f].ih);
    }
  }
}

// y_l[perm[rb + i]] = sum over the near blocks (r, c) of leaf row r of
// sum_j V_l[i][j] x_l[perm[cb + j]] in float-float: one warp per (leaf row,
// frequency), lanes over the rows, blocks in their stored order.
__global__ void __launch_bounds__(256) k_near_dense_ff(int M, int Ls, const int* __restrict__ leaves,
                                                       const int* __restrict__ rowptr,
                                                       const int2* __restrict__ rc,
                                                       const int* __restrict__ begin,
                                                       const int* __restrict__ end,
                                                       const int* __restrict__ perm,
                                                       const int64_t* __restrict__ voff,
                                                       const ffc* __restrict__ V,
                                                       const double2* __restrict__ x,
                                                       double2* __restrict__ y,
                                                       const int* __restrict__ act) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int l = blockIdx.x * 8 + w;
  if (l >= Ls || (act && !act[l])) return;  // act: frequencies to compute (may be null)
  const int r = leaves[blockIdx.y];
  const int rb = begin[r], nr = end[r] - rb;
  const double2* xl = x + (size_t)l * M;
  ffc acc = ffc_zero();
  for (int bi = rowptr[r]; bi < rowptr[r + 1]; ++bi) {
    const int c = rc[bi].y;
    const int cb = begin[c], nc = end[c] - cb;
    const ffc xj = lane < nc ? ffc_from(xl[perm[cb + lane]]) : ffc_zero();
    const ffc* Vb = V + voff[bi] + (size_t)l * nc * nr;
    // columns in groups of 8: the group's loads are issued together
    for (int j0 = 0; j0 < nc; j0 += 8) {
      ffc v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = (lane < nr && j0 + u < nc) ? Vb[(size_t)(j0 + u) * nr + lane] : ffc_zero();
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u;
        if (j < nc) {
          ffc xv;
          xv.rh = __shfl_sync(0xffffffffu, xj.rh, j);
          xv.ih = __shfl_sync(0xffffffffu, xj.ih, j);
          xv.rl = __shfl_sync(0xffffffffu, xj.rl, j);
          xv.il = __shfl_sync(0xffffffffu, xj.il, j);
          if (lane < nr) ffc_mac(acc, v[u], xv);
          if ((j & 15) == 15) ffc_renorm(acc);
        }
      }
    }
    ffc_renorm(acc);
  }
  if (lane < nr) y[(size_t)l * M + perm[rb + lane]] = ffc_to(acc);
}

int build_near_expanded_ff(cqm_handle* h) {
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
    const unsigned g = (unsigned)((h->Ls + FAR_NF - 1) / FAR_NF) * (unsigned)nb;
    k_near_expand_ff<<<g, 256, 0, h->stream>>>(h->Ls, h->rank_cap, h->near_rc.p, h->node_begin.p,
                                               h->node_end.p, h->near_off.p, h->near_rank.p,
                                               (const ffc*)h->nearC.p, h->nearD.p, h->nearV_off.p,
                                               (ffc*)h->nearV.p, h->nearV_f.p);
  }
  CQM_CHECK_LAUNCH();
  h->near_expanded = true;
  h->nearV_ff = true;
  return CQM_OK;
}

int near_apply_expanded_ff(cqm_handle* h, const double2* x, double2* y) {
  const int nleaf = (int)h->h_leaves.size();
  if (nleaf == 0) return CQM_OK;
  dim3 g((unsigned)((h->Ls + 7) / 8), (unsigned)nleaf);
  k_near_dense_ff<<<g, 256, 0, h->stream>>>(h->M, h->Ls, h->d_leaves.p, h->near_rowptr.p, h->near_rc.p,
                                            h->node_begin.p, h->node_end.p, h->perm.p, h->nearV_off.p,
                                            (const ffc*)h->nearV.p, x, y, h->exact_active);
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

}  // namespace cqm
