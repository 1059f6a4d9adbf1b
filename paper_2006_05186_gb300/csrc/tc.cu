// Far-field coupling of the inner operator on the tensor cores.
//
// yhat_r[mu][l] += sum_{b=(r,c)} sum_t sum_nu C_{b,t}[mu][nu] (d_t[l] xhat_c[nu][l])
// (eq. lrfinal at all frequencies) is a dense contraction.  Written in real
// arithmetic it is, per (b, t), a 128 x 128 by 128 x L product
//   [Re y; Im y] += [[Re C, -Im C], [Im C, Re C]] [Re x~; Im x~],
// x~ = d_t (.) xhat_c.  Each warp owns 16 of the 128 output rows and all
// frequency columns of a chunk; the product runs on mma.sync m16n8k8 TF32 with
// each operand split as hi + lo (TF32 each) and three products
// hi*hi + hi*lo + lo*hi accumulated in FP32, which keeps FP32-level accuracy
// (the inner operator is FP32; FP64-accurate residuals are computed apart).
// Work items and the per-row reduction of their partial tiles are the same as
// for the SIMT kernel.
#include <algorithm>

#include "handle.cuh"

namespace cqm {

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int TC_P = 64;      // Chebyshev points per cluster (m = 4)
constexpr int TC_CPAD = 68;   // row stride of the staged C planes (conflict-free A loads)

// Row stride of the staged real x~: = 8 or 24 mod 32 words, so that the four
// rows a B fragment reads fall into distinct banks.
__host__ __device__ constexpr int xt_stride(int nc) { return nc + ((40 - (nc % 32)) % 32); }

// NT = 8-column tiles per frequency chunk (chunk = 8 NT columns).
template <int NT>
__global__ void __launch_bounds__(256, 1) k_far_coupling_tc(int Ls, int cap,
                                                            const int4* __restrict__ items,
                                                            const int2* __restrict__ blocks,
                                                            const int* __restrict__ rank,
                                                            const float2* __restrict__ Cf,
                                                            const float2* __restrict__ Df,
                                                            const float2* __restrict__ xhat,
                                                            float2* __restrict__ part) {
  constexpr int NC = 8 * NT;          // columns per chunk
  constexpr int XT_STRIDE = xt_stride(NC);
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* Xh = (float2*)smraw;                       // TC_P x NC   (xhat chunk, complex)
  float* Xt = (float*)(Xh + TC_P * NC);              // 128 x NC    (real [Re x~; Im x~])
  float* Cr = Xt + 128 * XT_STRIDE;                  // TC_P x TC_CPAD
  float* Ci = Cr + TC_P * TC_CPAD;                   // TC_P x TC_CPAD
  float2* Ds = (float2*)(Ci + TC_P * TC_CPAD);       // NC
  const int4 it = items[blockIdx.x];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int row0 = 16 * w;  // rows row0 .. row0+15 of the real 128-row output
  for (int l0 = 0; l0 < Ls; l0 += NC) {
    float acc[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[n][q] = 0.f;
    for (int bi = it.y; bi < it.z; ++bi) {
      const int c = blocks[bi].y;
      __syncthreads();
      for (int e = threadIdx.x; e < TC_P * NC; e += blockDim.x) {
        const int nu = e / NC, l = e - nu * NC;
        Xh[e] = (l0 + l < Ls) ? xhat[((size_t)c * TC_P + nu) * Ls + l0 + l] : make_float2(0.f, 0.f);
      }
      const int rk = rank[bi];
      for (int tt = 0; tt < rk; ++tt) {
        __syncthreads();
        const float2* Ct = Cf + ((size_t)bi * cap + tt) * TC_P * TC_P;
        for (int e = threadIdx.x; e < TC_P * TC_P; e += blockDim.x) {
          const float2 v = Ct[e];
          const int mu = e >> 6, nu = e & 63;
          Cr[mu * TC_CPAD + nu] = v.x;
          Ci[mu * TC_CPAD + nu] = v.y;
        }
        for (int l = threadIdx.x; l < NC; l += blockDim.x)
          Ds[l] = (l0 + l < Ls) ? Df[((size_t)bi * cap + tt) * Ls + l0 + l] : make_float2(0.f, 0.f);
        __syncthreads();
        for (int e = threadIdx.x; e < TC_P * NC; e += blockDim.x) {
          const int nu = e / NC, l = e - nu * NC;
          const float2 x = Xh[e], d = Ds[l];
          Xt[nu * XT_STRIDE + l] = fmaf(d.x, x.x, -d.y * x.y);
          Xt[(nu + TC_P) * XT_STRIDE + l] = fmaf(d.x, x.y, d.y * x.x);
        }
        __syncthreads();
#pragma unroll 2
        for (int kk = 0; kk < 128; kk += 8) {
          // A fragment: rows row0 + g (+8), columns kk + tq (+4)
          float av[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int row = row0 + g + ((q & 1) ? 8 : 0);
            const int k = kk + tq + ((q & 2) ? 4 : 0);
            const int mu = row & 63, nu = k & 63;
            const bool im_row = row >= 64, im_col = k >= 64;
            float v;
            if (!im_row) v = im_col ? -Ci[mu * TC_CPAD + nu] : Cr[mu * TC_CPAD + nu];
            else v = im_col ? Cr[mu * TC_CPAD + nu] : Ci[mu * TC_CPAD + nu];
            av[q] = v;
          }
          uint32_t ah[4], al[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) split_tf32(av[q], ah[q], al[q]);
#pragma unroll
          for (int n = 0; n < NT; ++n) {
            const float b0 = Xt[(kk + tq) * XT_STRIDE + 8 * n + g];
            const float b1 = Xt[(kk + tq + 4) * XT_STRIDE + 8 * n + g];
            uint32_t bh[2], bl[2];
            split_tf32(b0, bh[0], bl[0]);
            split_tf32(b1, bh[1], bl[1]);
            mma_tf32(acc[n], al, bh);
            mma_tf32(acc[n], ah, bl);
            mma_tf32(acc[n], ah, bh);
          }
        }
      }
    }
    // D fragment: rows row0 + g (+8), columns 8n + 2 tq (+1)
    const bool im = row0 >= 64;
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = row0 + g + ((q & 2) ? 8 : 0);
        const int l = l0 + 8 * n + 2 * tq + (q & 1);
        if (l < Ls) {
          float* o = (float*)&part[((size_t)blockIdx.x * TC_P + (row & 63)) * Ls + l];
          o[im ? 1 : 0] = acc[n][q];
        }
      }
  }
}

template <int NT>
static size_t tc_smem() {
  constexpr int NC = 8 * NT;
  return sizeof(float2) * TC_P * NC + sizeof(float) * 128 * xt_stride(NC) +
         2 * sizeof(float) * TC_P * TC_CPAD + sizeof(float2) * NC;
}

static int nt_for(int Ls) { return std::min(17, std::max(1, (Ls + 7) / 8)); }

int setup_tc_kernels(cqm_handle* h) {
#define TC_SETUP(N)                                                                             \
  CQM_CUDA_TRY(cudaFuncSetAttribute(k_far_coupling_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                    (int)tc_smem<N>()));
  TC_SETUP(1) TC_SETUP(2) TC_SETUP(3) TC_SETUP(4) TC_SETUP(5) TC_SETUP(6) TC_SETUP(8)
  TC_SETUP(9) TC_SETUP(12) TC_SETUP(17)
#undef TC_SETUP
  return CQM_OK;
}

int far_coupling_tc(cqm_handle* h) {
  const int n = h->n_far_items;
  ProfScope ps_(h, CQM_K_FAR_COUPLING);
#define TC_LAUNCH(N)                                                                            \
  k_far_coupling_tc<N><<<n, 256, tc_smem<N>(), h->stream>>>(h->Ls, h->rank_cap, h->far_items.p, \
                                                             h->far_rc.p, h->far_rank.p, h->farC_f.p, \
                                                             h->farD_f.p, h->xhat_f.p, h->part_f.p)
  const int nt = nt_for(h->Ls);
  if (nt <= 1) TC_LAUNCH(1);
  else if (nt <= 2) TC_LAUNCH(2);
  else if (nt <= 3) TC_LAUNCH(3);
  else if (nt <= 4) TC_LAUNCH(4);
  else if (nt <= 5) TC_LAUNCH(5);
  else if (nt <= 6) TC_LAUNCH(6);
  else if (nt <= 8) TC_LAUNCH(8);
  else if (nt <= 9) TC_LAUNCH(9);
  else if (nt <= 12) TC_LAUNCH(12);
  else TC_LAUNCH(17);
#undef TC_LAUNCH
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

}  // namespace cqm
