// R-scaled discrete Fourier transforms between time steps and CQM frequencies
// (Sec. 3.1, eq. omega_n; Remark in Sec. 6.2):
//   forward  ghat_l = sum_{n=0..N} R^n b_n zeta^{n l},            l < Ls
//   inverse  q_n = R^{-n} / L sum_{l=0..L-1} qhat_l zeta^{-n l},  with
//            qhat_{L-l} = conj(qhat_l) (real data, s_{L-l} = conj s_l), so
//            q_n = R^{-n}/L [Re qhat_0 + 2 sum_{0<l<L/2} Re(qhat_l zeta^{-nl})
//                            (+ Re(qhat_{L/2} (-1)^n) for even L)].
// Twiddles zeta^k for k = (n l) mod L come from a table in shared memory.
// Layout: time data (N+1) x M real, frequency data Ls x M complex (row l).
#include "handle.cuh"

namespace cqm {

// Shared-memory twiddle table cos/sin(2 pi k / L) and powers R^(+-n).
__device__ void load_tables(int L, double R, double sign_pow, double2* tw, double* rp) {
  for (int k = threadIdx.x; k < L; k += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)k / (double)L, &sn, &cs);
    tw[k] = make_double2(cs, sn);
    rp[k] = pow(R, sign_pow * (double)k);
  }
  __syncthreads();
}

// One thread per element i, a tile of FT frequencies per block row.
template <int FT>
__global__ void k_forward(int M, int L, int Ls, double R, const double* __restrict__ b,
                          double2* __restrict__ ghat) {
  extern __shared__ double smem[];
  double2* tw = (double2*)smem;
  double* rp = (double*)(tw + L);
  load_tables(L, R, 1.0, tw, rp);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int l0 = blockIdx.y * FT;
  if (i >= M) return;
  double2 acc[FT];
#pragma unroll
  for (int f = 0; f < FT; ++f) acc[f] = make_double2(0.0, 0.0);
  for (int n = 0; n < L; ++n) {
    const double v = rp[n] * b[(size_t)n * M + i];
#pragma unroll
    for (int f = 0; f < FT; ++f) {
      int l = l0 + f;
      if (l < Ls) {
        double2 z = tw[(int)(((long long)n * l) % L)];
        acc[f].x += v * z.x;
        acc[f].y += v * z.y;
      }
    }
  }
#pragma unroll
  for (int f = 0; f < FT; ++f)
    if (l0 + f < Ls) ghat[(size_t)(l0 + f) * M + i] = acc[f];
}

template <int NT>
__global__ void k_inverse(int M, int L, int Ls, double R, const double2* __restrict__ qhat,
                          double* __restrict__ q) {
  extern __shared__ double smem[];
  double2* tw = (double2*)smem;
  double* rp = (double*)(tw + L);
  load_tables(L, R, -1.0, tw, rp);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n0 = blockIdx.y * NT;
  if (i >= M) return;
  const bool even = (L % 2) == 0;
  const int lmax = even ? L / 2 : Ls;  // exclusive bound of the doubled terms
  double acc[NT];
  const double2 q0 = qhat[i];
#pragma unroll
  for (int f = 0; f < NT; ++f) acc[f] = q0.x;
  for (int l = 1; l < Ls; ++l) {
    const double2 v = qhat[(size_t)l * M + i];
    const double fac = (even && l == L / 2) ? 1.0 : 2.0;
#pragma unroll
    for (int f = 0; f < NT; ++f) {
      int n = n0 + f;
      if (n < L) {
        double2 z = tw[(int)(((long long)n * l) % L)];  // zeta^{+nl}; zeta^{-nl} = conj
        acc[f] += fac * (v.x * z.x + v.y * z.y);
      }
    }
  }
  (void)lmax;
#pragma unroll
  for (int f = 0; f < NT; ++f) {
    int n = n0 + f;
    if (n < L) q[(size_t)n * M + i] = acc[f] * rp[n] / (double)L;
  }
}

// Shared memory of the tables: 24 L bytes (L <= CQM_MAX_STEPS + 1, checked
// at setup); above the default 48 KB the kernels opt in to more.
static size_t table_bytes(int L) { return (size_t)L * (sizeof(double2) + sizeof(double)); }

template <class K>
static int opt_in(K kernel, size_t sh) {
  if (sh > 48 * 1024)
    CQM_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
  return CQM_OK;
}

// The transforms of ncol columns (nt for the P0 data, nv for vertex data).
int forward_transform_cols(cqm_handle* h, int ncol, const double* d_b, double2* d_ghat) {
  constexpr int FT = 8;
  dim3 grid(grid_for(ncol, 128), grid_for(h->Ls, FT));
  const size_t sh = table_bytes(h->L);
  CQM_TRY(opt_in(k_forward<FT>, sh));
  {
    ProfScope ps_(h, CQM_K_FORWARD_DFT);
    k_forward<FT><<<grid, 128, sh, h->stream>>>(ncol, h->L, h->Ls, h->R, d_b, d_ghat);
  }
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

int inverse_transform_cols(cqm_handle* h, int ncol, const double2* d_qhat, double* d_q) {
  constexpr int NT = 8;
  dim3 grid(grid_for(ncol, 128), grid_for(h->L, NT));
  const size_t sh = table_bytes(h->L);
  CQM_TRY(opt_in(k_inverse<NT>, sh));
  {
    ProfScope ps_(h, CQM_K_INVERSE_DFT);
    k_inverse<NT><<<grid, 128, sh, h->stream>>>(ncol, h->L, h->Ls, h->R, d_qhat, d_q);
  }
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

int forward_transform(cqm_handle* h, const double* d_b, double2* d_ghat) {
  return forward_transform_cols(h, h->M, d_b, d_ghat);
}

int inverse_transform(cqm_handle* h, const double2* d_qhat, double* d_q) {
  return inverse_transform_cols(h, h->M, d_qhat, d_q);
}

}  // namespace cqm
