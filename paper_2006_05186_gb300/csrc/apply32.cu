// FP32 SIMT contractions of the inner operator (mixed-precision GMRES) from
// the factors: the far coupling with tensor_cores = 0 (or m < 4, through the
// generic kernel) and the near field with expand_near = 0.  Register tiled:
// one block covers a work item (a row cluster and a run of its blocks) and up
// to 32 * NLT frequencies, so a stored factor C_{b,t} is read once per apply;
// the items' partial tiles are summed per row in item order.  Every thread keeps a tile of
// rows x NLT frequencies of complex accumulators, and d_t[l] is folded into
// the staged x_c (yhat[mu][l] += sum_nu C_t[mu][nu] (d_t[l] xhat[nu][l])),
// which is eq. lrfinal applied to all frequencies at once.
#include <algorithm>

#include "handle.cuh"

namespace cqm {

constexpr int NLT_MAX = 5;  // frequencies per thread: 160 per block pass

__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Far coupling; p = 64 (8 warps x 8 rows each).
template <int NLT>
__global__ void __launch_bounds__(256) k_far_coupling_f32(int Ls, int cap,
                                                          const int4* __restrict__ items,
                                                          const int2* __restrict__ blocks,
                                                          const int* __restrict__ rank,
                                                          const float2* __restrict__ Cf,
                                                          const float2* __restrict__ Df,
                                                          const float2* __restrict__ xhat,
                                                          float2* __restrict__ part) {
  constexpr int P = 64, LW = 32 * NLT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* Xs = (float2*)smraw;  // P x LW
  float2* Cs = Xs + P * LW;     // P x P
  const int4 it = items[blockIdx.x];  // (row, first block, end block, -)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int mu0 = w * 8;
  for (int l0 = 0; l0 < Ls; l0 += LW) {
    float2 acc[8][NLT];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int k = 0; k < NLT; ++k) acc[i][k] = make_float2(0.f, 0.f);
    for (int bi = it.y; bi < it.z; ++bi) {
      const int c = blocks[bi].y;
      __syncthreads();
      for (int t = threadIdx.x; t < P * LW; t += blockDim.x) {
        const int nu = t / LW, l = t - nu * LW;
        Xs[t] = (l0 + l < Ls) ? xhat[((size_t)c * P + nu) * Ls + l0 + l] : make_float2(0.f, 0.f);
      }
      const int rk = rank[bi];
      for (int tt = 0; tt < rk; ++tt) {
        __syncthreads();
        const float4* Ct = (const float4*)(Cf + ((size_t)bi * cap + tt) * P * P);
        for (int t = threadIdx.x; t < P * P / 2; t += blockDim.x) ((float4*)Cs)[t] = Ct[t];
        float2 d[NLT];
#pragma unroll
        for (int k = 0; k < NLT; ++k) {
          const int l = l0 + lane + 32 * k;
          d[k] = l < Ls ? Df[((size_t)bi * cap + tt) * Ls + l] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int nu = 0; nu < P; ++nu) {
          float2 xd[NLT];
#pragma unroll
          for (int k = 0; k < NLT; ++k) xd[k] = f2mul(d[k], Xs[nu * LW + lane + 32 * k]);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float2 cv = Cs[(mu0 + i) * P + nu];
#pragma unroll
            for (int k = 0; k < NLT; ++k) cfma(acc[i][k], cv, xd[k]);
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int k = 0; k < NLT; ++k) {
        const int l = l0 + lane + 32 * k;
        if (l < Ls) part[((size_t)blockIdx.x * P + mu0 + i) * Ls + l] = acc[i][k];
      }
  }
}

// yhat_r[mu][l] += sum of the partial tiles of row r's items, in item order.
__global__ void k_far_reduce_f32(int Ls, int lmax, const int* __restrict__ rows,
                                 const int* __restrict__ item_ptr, const float2* __restrict__ part,
                                 float2* __restrict__ yhat, const int* __restrict__ act) {
  constexpr int P = 64;
  const int k = blockIdx.x;  // index into the list of far rows
  const int r = rows[k];
  for (int e = threadIdx.x; e < P * Ls; e += blockDim.x) {
    if (e % Ls >= lmax) continue;  // frequencies the partial tiles do not hold
    if (act && !act[e % Ls]) continue;  // converged frequencies (act may be null)
    float2 a = make_float2(0.f, 0.f);
    for (int it = item_ptr[k]; it < item_ptr[k + 1]; ++it) a = cadd(a, part[(size_t)it * P * Ls + e]);
    float2* o = yhat + (size_t)r * P * Ls + e;
    *o = cadd(*o, a);
  }
}

// Near field; leaf clusters of at most 32 triangles: warp w owns rows
// w, w + 8, w + 16, w + 24, so a leaf of #r rows keeps every warp at
// ceil(#r / 8) rows or one fewer.
template <int NLT>
__global__ void __launch_bounds__(256) k_near_apply_f32(
    int M, int Ls, int cap, const int4* __restrict__ items, const int2* __restrict__ blocks,
    const int* __restrict__ rank, const int64_t* __restrict__ off, const float2* __restrict__ Cn,
    const float2* __restrict__ Dn, const int* __restrict__ begin, const int* __restrict__ end,
    const int* __restrict__ perm, const double2* __restrict__ X, float2* __restrict__ part) {
  constexpr int LW = 32 * NLT;
  __shared__ float2 Xs[32 * LW];
  __shared__ float2 Cs[32 * 32];
  const int4 it = items[blockIdx.x];  // (leaf row, first block, end block, -)
  const int r = it.x;
  const int rb = begin[r], nr = end[r] - rb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nrw = (nr - w + 7) >> 3;  // rows of this warp: w + 8 i for i < nrw
  for (int l0 = 0; l0 < Ls; l0 += LW) {
    float2 acc[4][NLT];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < NLT; ++k) acc[i][k] = make_float2(0.f, 0.f);
    for (int bi = it.y; bi < it.z; ++bi) {
      const int c = blocks[bi].y;
      const int cb = begin[c], nc = end[c] - cb;
      __syncthreads();
      for (int t = threadIdx.x; t < nc * LW; t += blockDim.x) {
        const int j = t / LW, l = t - j * LW;
        const double2 v = (l0 + l < Ls) ? X[(size_t)(l0 + l) * M + perm[cb + j]] : make_double2(0.0, 0.0);
        Xs[t] = make_float2((float)v.x, (float)v.y);
      }
      const int rk = rank[bi];
      for (int tt = 0; tt < rk; ++tt) {
        __syncthreads();
        const float2* Ct = Cn + off[bi] + (size_t)tt * nr * nc;
        for (int t = threadIdx.x; t < nr * nc; t += blockDim.x) Cs[t] = Ct[t];
        float2 d[NLT];
#pragma unroll
        for (int k = 0; k < NLT; ++k) {
          const int l = l0 + lane + 32 * k;
          d[k] = l < Ls ? Dn[((size_t)bi * cap + tt) * Ls + l] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int j = 0; j < nc; ++j) {
          float2 xd[NLT];
#pragma unroll
          for (int k = 0; k < NLT; ++k) xd[k] = f2mul(d[k], Xs[j * LW + lane + 32 * k]);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (i < nrw) {
              const float2 cv = Cs[(w + 8 * i) * nc + j];
#pragma unroll
              for (int k = 0; k < NLT; ++k) cfma(acc[i][k], cv, xd[k]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < NLT; ++k) {
        const int l = l0 + lane + 32 * k;
        if (i < nrw && l < Ls) part[((size_t)blockIdx.x * 32 + w + 8 * i) * Ls + l] = acc[i][k];
      }
  }
}

// Y[l][perm[rb + i]] = sum of the partial tiles of leaf row k's items, in item order.
__global__ void k_near_reduce_f32(int M, int Ls, const int* __restrict__ leaves,
                                  const int* __restrict__ item_ptr, const int* __restrict__ begin,
                                  const int* __restrict__ end, const int* __restrict__ perm,
                                  const float2* __restrict__ part, double2* __restrict__ Y) {
  const int k = blockIdx.x;
  const int r = leaves[k];
  const int rb = begin[r], nr = end[r] - rb;
  for (int e = threadIdx.x; e < nr * Ls; e += blockDim.x) {
    const int i = e / Ls, l = e - i * Ls;
    float2 a = make_float2(0.f, 0.f);
    for (int it = item_ptr[k]; it < item_ptr[k + 1]; ++it) a = cadd(a, part[((size_t)it * 32 + i) * Ls + l]);
    Y[(size_t)l * M + perm[rb + i]] = make_double2(a.x, a.y);
  }
}

static int nlt_for(int Ls) { return std::max(1, std::min(NLT_MAX, (Ls + 31) / 32)); }

template <int NLT>
static size_t far_smem() { return sizeof(float2) * (64 * 32 * NLT + 64 * 64); }

int setup_f32_kernels(cqm_handle* h) {
#define SETUP_NLT(N)                                                                              \
  CQM_CUDA_TRY(cudaFuncSetAttribute(k_far_coupling_f32<N>,                                        \
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)far_smem<N>()));
  SETUP_NLT(1) SETUP_NLT(2) SETUP_NLT(3) SETUP_NLT(4) SETUP_NLT(5)
#undef SETUP_NLT
  CQM_TRY(setup_tc2(h));
  return setup_tc_kernels(h);
}

int far_coupling_f32(cqm_handle* h) {
  const int n = h->n_far_items;
  if (h->p != 64) return far_coupling_generic_f32(h);  // the tiled kernels are written for m = 4
  if (h->params.tensor_cores == 1 && h->p == 64) {
    int l_tail = h->Ls;
    CQM_TRY(far_coupling_tc2(h, &l_tail));
    k_far_reduce_f32<<<(unsigned)h->h_far_rows.size(), 256, 0, h->stream>>>(
        h->Ls, l_tail, h->d_far_rows.p, h->far_item_ptr.p, h->part_f.p, h->yhat_f.p,
        h->inner_active);
    CQM_CHECK_LAUNCH();
    return CQM_OK;
  }
  if (h->params.tensor_cores == 2 && h->p == 64) {
    CQM_TRY(far_coupling_tc(h));
    k_far_reduce_f32<<<(unsigned)h->h_far_rows.size(), 256, 0, h->stream>>>(
        h->Ls, h->Ls, h->d_far_rows.p, h->far_item_ptr.p, h->part_f.p, h->yhat_f.p,
        h->inner_active);
    CQM_CHECK_LAUNCH();
    return CQM_OK;
  }
  ProfScope ps_(h, CQM_K_FAR_COUPLING);
#define LAUNCH_NLT(N)                                                                              \
  k_far_coupling_f32<N><<<n, 256, far_smem<N>(), h->stream>>>(                                     \
      h->Ls, h->rank_cap, h->far_items.p, h->far_rc.p, h->far_rank.p, h->farC_f.p, h->farD_f.p,     \
      h->xhat_f.p, h->part_f.p)
  switch (nlt_for(h->Ls)) {
    case 1: LAUNCH_NLT(1); break;
    case 2: LAUNCH_NLT(2); break;
    case 3: LAUNCH_NLT(3); break;
    case 4: LAUNCH_NLT(4); break;
    default: LAUNCH_NLT(5); break;
  }
#undef LAUNCH_NLT
  k_far_reduce_f32<<<(unsigned)h->h_far_rows.size(), 256, 0, h->stream>>>(
      h->Ls, h->Ls, h->d_far_rows.p, h->far_item_ptr.p, h->part_f.p, h->yhat_f.p,
        h->inner_active);
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

int near_apply_f32(cqm_handle* h, const double2* x, double2* y) {
  const int n = h->n_near_items;
  ProfScope ps_(h, CQM_K_NEAR_APPLY);
  if (h->near_expanded) return near_apply_expanded(h, x, y, false);
#define LAUNCH_NLT(N)                                                                              \
  k_near_apply_f32<N><<<n, 256, 0, h->stream>>>(                                                   \
      h->M, h->Ls, h->rank_cap, h->near_items.p, h->near_rc.p, h->near_rank.p, h->near_off.p,      \
      h->nearC_f.p, h->nearD_f.p, h->node_begin.p, h->node_end.p, h->perm.p, x, h->part_f.p)
  switch (nlt_for(h->Ls)) {
    case 1: LAUNCH_NLT(1); break;
    case 2: LAUNCH_NLT(2); break;
    case 3: LAUNCH_NLT(3); break;
    case 4: LAUNCH_NLT(4); break;
    default: LAUNCH_NLT(5); break;
  }
#undef LAUNCH_NLT
  k_near_reduce_f32<<<(unsigned)h->h_leaves.size(), 256, 0, h->stream>>>(
      h->M, h->Ls, h->d_leaves.p, h->near_item_ptr.p, h->node_begin.p, h->node_end.p, h->perm.p,
      h->part_f.p, y);
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

}  // namespace cqm
