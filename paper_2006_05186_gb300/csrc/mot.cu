// Marching on in time with the compressed CQM weights (Sec. 3.2, the time
// stepping of the Galerkin CQM system; Sec. 6.2, eqs. fastdft and fastrhs).
//
// The CQM weights of the single layer are Vhat_n = R^-n / L sum_l V_l zeta^{-nl}
// (eq. dft with L = N + 1).  Every block of the partition holds
// V_l = sum_t C_t d_t(l) for the solved frequencies l < Ls (eq. lrfinal; far
// blocks between their cluster bases), and V_{L-l} = conj V_l, so
//
//   Vhat_n = Re sum_t C_t dhat_t[n],
//   dhat_t[n] = R^-n / L sum_{l < Ls} c_l d_t(l) zeta^{-nl}    (eq. fastdft)
//
// with c_l = 1 for l = 0 and for l = L/2 (L even), else 2: the transform acts
// on the MACA fibres only.  The time-discrete system is the causal convolution
// sum_{k <= n} Vhat_{n-k} q_k = b_n, solved step by step:
//
//   Vhat_0 q_n = b_n - Re sum_t C_t (sum_{k < n} dhat_t[n-k] q_k)  (eq. fastrhs)
//
// per near block with q_k restricted to the column cluster, per far block
// with its basis coefficients xhat_c(k) = U_c^T q_k, followed by the
// down-sweep and the leaf bases.  Vhat_0 is real symmetric positive definite;
// it is assembled densely once (tree order), inverted once by blocked
// Gauss-Jordan elimination, and each step applies the inverse (one GEMV).
// The weights, the inverse and the step solve are FP64 (the weights carry
// R^-n ~ 1e5 at the last steps); the history sums, the bulk of the work, run
// in float-float (~48 bits) on the FP32 pipes when the factors are held as
// float-float pairs, and in FP64 otherwise.
#include <algorithm>
#include <vector>

#include "ffexp.cuh"
#include "handle.cuh"

namespace cqm {

namespace {
constexpr int GJ = 32;        // Gauss-Jordan tile
constexpr int TP = 64;        // max Chebyshev points per cluster (p <= 64)
}  // namespace

// C factor entry e of the flat factor array, FP64 or float-float pairs.
__device__ __forceinline__ double2 c_at(const double2* __restrict__ C, bool ff, size_t e) {
  if (!ff) return C[e];
  const float4 v = reinterpret_cast<const float4*>(C)[e];  // (re hi, im hi, re lo, im lo)
  return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}

// eq. fastdft for every term of every block: one CTA per block, threads over
// the steps n; d_t of the solved frequencies is staged in shared memory.
__global__ void __launch_bounds__(256) k_mot_fastdft(int L, int Ls, int cap, double R,
                                                     const int* __restrict__ rank,
                                                     const double2* __restrict__ D,
                                                     const double2* __restrict__ tw,
                                                     double2* __restrict__ Dh) {
  extern __shared__ double2 ds[];  // Ls
  const int b = blockIdx.x;
  const int rk = rank[b];
  const double invL = 1.0 / (double)L;
  for (int t = 0; t < rk; ++t) {
    const double2* d = D + ((size_t)b * cap + t) * Ls;
    __syncthreads();
    for (int l = threadIdx.x; l < Ls; l += blockDim.x) {
      const double c = (l == 0 || 2 * l == L) ? 1.0 : 2.0;
      ds[l] = cscale(d[l], c);
    }
    __syncthreads();
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
      double2 acc = make_double2(0.0, 0.0);
      int j = 0;  // n l mod L
      for (int l = 0; l < Ls; ++l) {
        cfma(acc, ds[l], tw[j]);  // tw[j] = zeta^{-j}
        j += n;
        if (j >= L) j -= L;
      }
      Dh[((size_t)b * cap + t) * L + n] = cscale(acc, pow(R, -(double)n) * invL);
    }
  }
}

// zeta^{-j} = exp(-2 pi i j / L), j = 0..L-1
__global__ void k_mot_twiddles(int L, double2* tw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L) return;
  double sn, cs;
  sincospi(-2.0 * (double)j / (double)L, &sn, &cs);
  tw[j] = make_double2(cs, sn);
}

// Explicit cluster bases: Ue_r (#r x p, row i = tree position begin_r + i).
// Leaves copy their rows of the leaf basis; a parent r stacks its sons' rows
// times the transfer matrix, U_r[i][mu] = sum_lambda U_s[i][lambda] E_s[lambda][mu]
// (Def. 5).  One CTA per node of one level; deepest level first.
__global__ void __launch_bounds__(256) k_mot_bases(int node0, int m, int p, const int* __restrict__ begin,
                                                   const int* __restrict__ end,
                                                   const int* __restrict__ son0,
                                                   const int* __restrict__ son1,
                                                   const double* __restrict__ Uleaf,
                                                   const double* __restrict__ Etr,
                                                   const int64_t* __restrict__ off, double* Ue) {
  __shared__ double E[TP * TP];
  const int r = node0 + blockIdx.x;
  const int rb = begin[r], nr = end[r] - rb;
  double* dst = Ue + off[r];
  if (son0[r] < 0) {
    for (int e = threadIdx.x; e < nr * p; e += blockDim.x) dst[e] = Uleaf[(size_t)rb * p + e];
    return;
  }
  for (int si = 0; si < 2; ++si) {
    const int s = si ? son1[r] : son0[r];
    const double* f = Etr + (size_t)s * 3 * m * m;
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
      const int lam = e / p, mu = e - lam * p;
      const int lx = lam % m, ly = (lam / m) % m, lz = lam / (m * m);
      const int mx = mu % m, my = (mu / m) % m, mz = mu / (m * m);
      E[e] = f[lx * m + mx] * f[m * m + ly * m + my] * f[2 * m * m + lz * m + mz];
    }
    __syncthreads();
    const int sb = begin[s] - rb, ns = end[s] - begin[s];
    const double* src = Ue + off[s];
    for (int e = threadIdx.x; e < ns * p; e += blockDim.x) {
      const int i = e / p, mu = e - i * p;
      double acc = 0.0;
      for (int lam = 0; lam < p; ++lam) acc = fma(src[(size_t)i * p + lam], E[lam * p + mu], acc);
      dst[(size_t)(sb + i) * p + mu] = acc;
    }
  }
}

// Dense weight Vhat_n in tree order (A[a * M + b], a, b tree positions).
// Near blocks: Re sum_t C_t[i][j] dhat_t[n]; one CTA per block.
__global__ void __launch_bounds__(256) k_mot_weight_near(int n, int L, int cap, int M,
                                                         const int2* __restrict__ rc,
                                                         const int* __restrict__ begin,
                                                         const int* __restrict__ end,
                                                         const int64_t* __restrict__ off,
                                                         const int* __restrict__ rank,
                                                         const double2* __restrict__ C, int ff,
                                                         const double2* __restrict__ Dh,
                                                         double* __restrict__ A) {
  __shared__ double2 dn[64];
  const int b = blockIdx.x;
  const int2 c2 = rc[b];
  const int rb = begin[c2.x], nr = end[c2.x] - rb, cb = begin[c2.y], nc = end[c2.y] - cb;
  const int rk = rank[b];
  for (int t = threadIdx.x; t < rk; t += blockDim.x) dn[t] = Dh[((size_t)b * cap + t) * L + n];
  __syncthreads();
  for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
    const int i = e / nc, j = e - i * nc;
    double v = 0.0;
    for (int t = 0; t < rk; ++t) {
      const double2 c = c_at(C, ff != 0, (size_t)off[b] + (size_t)t * nr * nc + e);
      v = fma(c.x, dn[t].x, fma(-c.y, dn[t].y, v));
    }
    A[(size_t)(rb + i) * M + cb + j] = v;
  }
}

// Far blocks: Ue_r S Ue_c^T with S = Re sum_t C_t dhat_t[n] (p x p); rows in
// chunks of 16 (T = Ue_r S staged in shared memory).  One CTA per block.
__global__ void __launch_bounds__(256) k_mot_weight_far(int n, int L, int cap, int M, int p,
                                                        const int2* __restrict__ rc,
                                                        const int* __restrict__ begin,
                                                        const int* __restrict__ end,
                                                        const int* __restrict__ rank,
                                                        const double2* __restrict__ C, int ff,
                                                        const double2* __restrict__ Dh,
                                                        const double* __restrict__ Ue,
                                                        const int64_t* __restrict__ uoff,
                                                        double* __restrict__ A) {
  __shared__ double S[TP * TP];
  __shared__ double T[16 * TP];
  __shared__ double2 dn[64];
  const int b = blockIdx.x;
  const int2 c2 = rc[b];
  const int rb = begin[c2.x], nr = end[c2.x] - rb, cb = begin[c2.y], nc = end[c2.y] - cb;
  const int rk = rank[b], pp = p * p;
  for (int t = threadIdx.x; t < rk; t += blockDim.x) dn[t] = Dh[((size_t)b * cap + t) * L + n];
  __syncthreads();
  for (int e = threadIdx.x; e < pp; e += blockDim.x) {
    double v = 0.0;
    for (int t = 0; t < rk; ++t) {
      const double2 c = c_at(C, ff != 0, ((size_t)b * cap + t) * pp + e);
      v = fma(c.x, dn[t].x, fma(-c.y, dn[t].y, v));
    }
    S[e] = v;
  }
  const double* Ur = Ue + uoff[c2.x];
  const double* Uc = Ue + uoff[c2.y];
  for (int i0 = 0; i0 < nr; i0 += 16) {
    const int ni = min(16, nr - i0);
    __syncthreads();
    for (int e = threadIdx.x; e < ni * p; e += blockDim.x) {
      const int i = e / p, nu = e - i * p;
      double v = 0.0;
      for (int mu = 0; mu < p; ++mu) v = fma(Ur[(size_t)(i0 + i) * p + mu], S[mu * p + nu], v);
      T[i * p + nu] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ni * nc; e += blockDim.x) {
      const int i = e / nc, j = e - i * nc;
      const double* uc = Uc + (size_t)j * p;
      double v = 0.0;
      for (int nu = 0; nu < p; ++nu) v = fma(T[i * p + nu], uc[nu], v);
      A[(size_t)(rb + i0 + i) * M + cb + j] = v;
    }
  }
}

// W[perm[a]][perm[b]] = A[a][b] (tree order to the caller's numbering)
__global__ void k_mot_untree(int M, const int* __restrict__ perm, const double* __restrict__ A,
                             double* __restrict__ W) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * M) return;
  const int a = (int)(e / M), b = (int)(e - (int64_t)a * M);
  W[(size_t)perm[a] * M + perm[b]] = A[e];
}

// ---- blocked Gauss-Jordan inversion of the SPD matrix A (M x M, in place) ---
// For each diagonal tile K: P = A_KK^-1; A_Kj <- P A_Kj (j != K);
// A_ij <- A_ij - A_iK A_Kj (i, j != K, with the new A_Kj); A_iK <- -A_iK P;
// A_KK <- P.  Without pivoting: the pivot tiles are Schur complements of an
// SPD matrix, hence SPD.  Tiles of GJ x GJ; the last ones ragged.

// P = inverse of the diagonal tile K by scalar Gauss-Jordan (one CTA, a
// thread per element; rows and columns past the matrix act as identity).
__global__ void __launch_bounds__(GJ * GJ) k_gj_diag(int K, int M, const double* __restrict__ A,
                                                     double* __restrict__ P) {
  __shared__ double a[GJ][GJ + 1];
  const int i = threadIdx.x / GJ, j = threadIdx.x % GJ;
  const int k0 = K * GJ, kb = min(GJ, M - k0);
  a[i][j] = (i < kb && j < kb) ? A[(size_t)(k0 + i) * M + k0 + j] : (i == j ? 1.0 : 0.0);
  __syncthreads();
  for (int k = 0; k < GJ; ++k) {
    const double pinv = 1.0 / a[k][k];
    const double aik = a[i][k], akj = a[k][j], aij = a[i][j];
    __syncthreads();
    double v;
    if (i == k && j == k) v = pinv;
    else if (i == k) v = akj * pinv;
    else if (j == k) v = -aik * pinv;
    else v = aij - aik * akj * pinv;
    a[i][j] = v;
    __syncthreads();
  }
  P[i * GJ + j] = a[i][j];
}

// Tile t: the row panel A_Kt <- P A_Kt (t != K) and a copy of the column
// panel A_tK into colbuf (t != K); tile K receives P.
__global__ void __launch_bounds__(GJ * GJ) k_gj_row(int K, int M, double* __restrict__ A,
                                                    const double* __restrict__ P,
                                                    double* __restrict__ colbuf) {
  __shared__ double ps[GJ][GJ + 1], xs[GJ][GJ + 1];
  const int t = blockIdx.x;
  const int i = threadIdx.x / GJ, j = threadIdx.x % GJ;
  const int k0 = K * GJ, kb = min(GJ, M - k0);
  const int t0 = t * GJ, tb = min(GJ, M - t0);
  if (t == K) {
    if (i < kb && j < kb) A[(size_t)(k0 + i) * M + k0 + j] = P[i * GJ + j];
    return;
  }
  ps[i][j] = P[i * GJ + j];
  xs[i][j] = (i < kb && j < tb) ? A[(size_t)(k0 + i) * M + t0 + j] : 0.0;
  if (i < tb && j < kb) colbuf[(size_t)(t0 + i) * GJ + j] = A[(size_t)(t0 + i) * M + k0 + j];
  __syncthreads();
  if (i < kb && j < tb) {
    double v = 0.0;
    for (int k = 0; k < kb; ++k) v = fma(ps[i][k], xs[k][j], v);
    A[(size_t)(k0 + i) * M + t0 + j] = v;
  }
}

// Tile (I, J), I != K: A_IJ -= colbuf_I A_KJ (J != K) or A_IK = -colbuf_I P.
__global__ void __launch_bounds__(GJ * GJ) k_gj_update(int K, int M, double* __restrict__ A,
                                                       const double* __restrict__ P,
                                                       const double* __restrict__ colbuf) {
  __shared__ double cs[GJ][GJ + 1], rs[GJ][GJ + 1];
  const int I = blockIdx.y, J = blockIdx.x;
  if (I == K) return;
  const int i = threadIdx.x / GJ, j = threadIdx.x % GJ;
  const int k0 = K * GJ, kb = min(GJ, M - k0);
  const int i0 = I * GJ, ib = min(GJ, M - i0), j0 = J * GJ, jb = min(GJ, M - j0);
  cs[i][j] = (i < ib && j < kb) ? colbuf[(size_t)(i0 + i) * GJ + j] : 0.0;
  if (J == K) rs[i][j] = P[i * GJ + j];
  else rs[i][j] = (i < kb && j < jb) ? A[(size_t)(k0 + i) * M + j0 + j] : 0.0;
  __syncthreads();
  if (i >= ib || j >= jb) return;
  double v = 0.0;
  for (int k = 0; k < kb; ++k) v = fma(cs[i][k], rs[k][j], v);
  double* o = A + (size_t)(i0 + i) * M + j0 + j;
  *o = (J == K) ? -v : *o - v;
}

// ---- one step n > 0: history sums (eq. fastrhs) ----------------------------

// Near block b = (r, c): part[b][i] = sum_t sum_j Re(C_t[i][j] z_t[j]),
// z_t[j] = sum_{k < n} dhat_t[n-k] q_k[c_j] (q in tree order, (L, M)).
// Warp w forms the terms t = w + 8u (lanes over the columns j), then rows
// i = w + 8v (lanes over j, warp sum).
__global__ void __launch_bounds__(256) k_mot_hist_near(int n, int L, int cap, int M,
                                                       const int2* __restrict__ rc,
                                                       const int* __restrict__ begin,
                                                       const int* __restrict__ end,
                                                       const int64_t* __restrict__ off,
                                                       const int* __restrict__ rank,
                                                       const double2* __restrict__ C, int ff,
                                                       const double2* __restrict__ Dh,
                                                       const double* __restrict__ qt,
                                                       double* __restrict__ part) {
  __shared__ double2 zs[64][32];
  const int b = blockIdx.x;
  const int2 c2 = rc[b];
  const int rb = begin[c2.x], nr = end[c2.x] - rb, cb = begin[c2.y], nc = end[c2.y] - cb;
  const int rk = rank[b];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  {
    double2 acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = make_double2(0.0, 0.0);
    const double2* dh = Dh + (size_t)b * cap * L + n;  // dhat_t[n - k] at dh[t L - k]
    for (int k = 0; k < n; ++k) {
      const double x = lane < nc ? qt[(size_t)k * M + cb + lane] : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = w + 8 * u;
        if (t < rk) {
          const double2 d = dh[(ptrdiff_t)t * L - k];
          acc[u].x = fma(d.x, x, acc[u].x);
          acc[u].y = fma(d.y, x, acc[u].y);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (w + 8 * u < rk) zs[w + 8 * u][lane] = acc[u];
  }
  __syncthreads();
  for (int i = w; i < nr; i += 8) {
    double v = 0.0;
    if (lane < nc)
      for (int t = 0; t < rk; ++t) {
        const double2 c = c_at(C, ff != 0, (size_t)off[b] + (size_t)t * nr * nc + (size_t)i * nc + lane);
        const double2 z = zs[t][lane];
        v = fma(c.x, z.x, fma(-c.y, z.y, v));
      }
    v = warp_sum(v);
    if (lane == 0) part[(size_t)b * 32 + i] = v;
  }
}

// Far block b = (r, c): part[b][mu] = sum_t sum_nu Re(C_t[mu][nu] z_t[nu]),
// z_t[nu] = sum_{k < n} dhat_t[n-k] xhat_c(k)[nu] (xhat: (node, k, nu)).
// Terms in passes of 32: thread (nu, g) forms the terms g + 4u of the pass;
// warp w then takes the rows mu = w + 8v with lanes over nu.
__global__ void __launch_bounds__(256) k_mot_hist_far(int n, int L, int cap, int p,
                                                      const int2* __restrict__ rc,
                                                      const int* __restrict__ rank,
                                                      const double2* __restrict__ C, int ff,
                                                      const double2* __restrict__ Dh,
                                                      const double* __restrict__ Xh,
                                                      double* __restrict__ part) {
  __shared__ double2 zs[32][TP];
  const int b = blockIdx.x;
  const int c = rc[b].y;
  const int rk = rank[b], pp = p * p;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nu = threadIdx.x & 63, g = threadIdx.x >> 6;
  double out[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) out[v] = 0.0;
  const double* xc = Xh + (size_t)c * L * p;
  for (int t0 = 0; t0 < rk; t0 += 32) {
    double2 acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = make_double2(0.0, 0.0);
    const double2* dh = Dh + (size_t)b * cap * L + n;
    for (int k = 0; k < n; ++k) {
      const double x = nu < p ? xc[(size_t)k * p + nu] : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = t0 + g + 4 * u;
        if (t < rk) {
          const double2 d = dh[(ptrdiff_t)t * L - k];
          acc[u].x = fma(d.x, x, acc[u].x);
          acc[u].y = fma(d.y, x, acc[u].y);
        }
      }
    }
    __syncthreads();  // the previous pass has read zs
#pragma unroll
    for (int u = 0; u < 8; ++u) zs[g + 4 * u][nu] = acc[u];
    __syncthreads();
    const int nt = min(32, rk - t0);
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int mu = w + 8 * v;
      if (mu < p)
        for (int t = 0; t < nt; ++t) {
          const size_t base = ((size_t)b * cap + t0 + t) * pp + (size_t)mu * p;
          if (lane < p) {
            const double2 cv = c_at(C, ff != 0, base + lane), z = zs[t][lane];
            out[v] = fma(cv.x, z.x, fma(-cv.y, z.y, out[v]));
          }
          if (lane + 32 < p) {
            const double2 cv = c_at(C, ff != 0, base + lane + 32), z = zs[t][lane + 32];
            out[v] = fma(cv.x, z.x, fma(-cv.y, z.y, out[v]));
          }
        }
    }
  }
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const double s = warp_sum(out[v]);
    if (lane == 0 && w + 8 * v < p) part[(size_t)b * TP + w + 8 * v] = s;
  }
}

// ---- the same history sums in float-float on the FP32 pipes ---------------
// (used when the C factors are held as float-float pairs).  The transformed
// fibres, the densities and the basis coefficients come as float-float
// copies (dhat: (re hi, im hi, re lo, im lo); reals: (hi, lo)); the sums
// carry about 48 bits, renormalised every 16 terms.
__device__ __forceinline__ ff ffv(float2 v) { return ff{v.x, v.y}; }

__global__ void __launch_bounds__(256) k_mot_hist_near_ff(int n, int L, int cap, int M,
                                                          const int2* __restrict__ rc,
                                                          const int* __restrict__ begin,
                                                          const int* __restrict__ end,
                                                          const int64_t* __restrict__ off,
                                                          const int* __restrict__ rank,
                                                          const float4* __restrict__ C,
                                                          const float4* __restrict__ Dh,
                                                          const float2* __restrict__ qt,
                                                          double* __restrict__ part) {
  __shared__ float4 zs[64][32];
  const int b = blockIdx.x;
  const int2 c2 = rc[b];
  const int rb = begin[c2.x], nr = end[c2.x] - rb, cb = begin[c2.y], nc = end[c2.y] - cb;
  const int rk = rank[b];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  {
    ff ar[8], ai[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) ar[u] = ai[u] = ff{0.f, 0.f};
    const float4* dh = Dh + (size_t)b * cap * L + n;  // dhat_t[n - k] at dh[t L - k]
    for (int k = 0; k < n; ++k) {
      const ff x = lane < nc ? ffv(qt[(size_t)k * M + cb + lane]) : ff{0.f, 0.f};
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = w + 8 * u;
        if (t < rk) {
          const float4 d = dh[(ptrdiff_t)t * L - k];
          ff_acc(ar[u], ff_mul(ff{d.x, d.z}, x));
          ff_acc(ai[u], ff_mul(ff{d.y, d.w}, x));
        }
      }
      if ((k & 15) == 15) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          ff_norm(ar[u]);
          ff_norm(ai[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      ff_norm(ar[u]);
      ff_norm(ai[u]);
      if (w + 8 * u < rk) zs[w + 8 * u][lane] = make_float4(ar[u].h, ai[u].h, ar[u].l, ai[u].l);
    }
  }
  __syncthreads();
  for (int i = w; i < nr; i += 8) {
    ff v = {0.f, 0.f};
    if (lane < nc)
      for (int t = 0; t < rk; ++t) {
        const float4 c = C[(size_t)off[b] + (size_t)t * nr * nc + (size_t)i * nc + lane];
        const float4 z = zs[t][lane];
        ff_acc(v, ff_mul(ff{c.x, c.z}, ff{z.x, z.z}));
        const ff q2 = ff_mul(ff{c.y, c.w}, ff{z.y, z.w});
        ff_acc(v, ff{-q2.h, -q2.l});
        if ((t & 15) == 15) ff_norm(v);
      }
    ff_norm(v);
    const double vd = warp_sum(ff_to_double(v));
    if (lane == 0) part[(size_t)b * 32 + i] = vd;
  }
}

__global__ void __launch_bounds__(256) k_mot_hist_far_ff(int n, int L, int cap, int p,
                                                         const int2* __restrict__ rc,
                                                         const int* __restrict__ rank,
                                                         const float4* __restrict__ C,
                                                         const float4* __restrict__ Dh,
                                                         const float2* __restrict__ Xh,
                                                         double* __restrict__ part) {
  __shared__ float4 zs[32][TP];
  const int b = blockIdx.x;
  const int c = rc[b].y;
  const int rk = rank[b], pp = p * p;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nu = threadIdx.x & 63, g = threadIdx.x >> 6;
  ff out[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) out[v] = ff{0.f, 0.f};
  const float2* xc = Xh + (size_t)c * L * p;
  for (int t0 = 0; t0 < rk; t0 += 32) {
    ff ar[8], ai[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) ar[u] = ai[u] = ff{0.f, 0.f};
    const float4* dh = Dh + (size_t)b * cap * L + n;
    for (int k = 0; k < n; ++k) {
      const ff x = nu < p ? ffv(xc[(size_t)k * p + nu]) : ff{0.f, 0.f};
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = t0 + g + 4 * u;
        if (t < rk) {
          const float4 d = dh[(ptrdiff_t)t * L - k];
          ff_acc(ar[u], ff_mul(ff{d.x, d.z}, x));
          ff_acc(ai[u], ff_mul(ff{d.y, d.w}, x));
        }
      }
      if ((k & 15) == 15) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          ff_norm(ar[u]);
          ff_norm(ai[u]);
        }
      }
    }
    __syncthreads();  // the previous pass has read zs
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      ff_norm(ar[u]);
      ff_norm(ai[u]);
      zs[g + 4 * u][nu] = make_float4(ar[u].h, ai[u].h, ar[u].l, ai[u].l);
    }
    __syncthreads();
    const int nt = min(32, rk - t0);
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int mu = w + 8 * v;
      if (mu < p) {
        for (int t = 0; t < nt; ++t) {
          const size_t base = ((size_t)b * cap + t0 + t) * pp + (size_t)mu * p;
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int nv = lane + 32 * hh;
            if (nv < p) {
              const float4 cv = C[base + nv], z = zs[t][nv];
              ff_acc(out[v], ff_mul(ff{cv.x, cv.z}, ff{z.x, z.z}));
              const ff q2 = ff_mul(ff{cv.y, cv.w}, ff{z.y, z.w});
              ff_acc(out[v], ff{-q2.h, -q2.l});
            }
          }
          if ((t & 7) == 7) ff_norm(out[v]);
        }
        ff_norm(out[v]);
      }
    }
  }
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const double sd = warp_sum(ff_to_double(out[v]));
    if (lane == 0 && w + 8 * v < p) part[(size_t)b * TP + w + 8 * v] = sd;
  }
}

// float-float copies: dhat (complex) and reals
__global__ void k_mot_to_ffc(int64_t n, const double2* __restrict__ a, float4* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = a[i];
  const ff re = ff_of(v.x), im = ff_of(v.y);
  b[i] = make_float4(re.h, im.h, re.l, im.l);
}
__global__ void k_mot_to_ffr(int64_t n, const double* __restrict__ a, float2* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ff v = ff_of(a[i]);
  b[i] = make_float2(v.h, v.l);
}

// yh[r][mu] = sum of the far blocks of row cluster r in stored order (0 if none).
__global__ void k_mot_reduce_far(int p, const int* __restrict__ rowptr, const double* __restrict__ part,
                                 double* __restrict__ yh) {
  const int r = blockIdx.x, mu = threadIdx.x;
  if (mu >= p) return;
  double v = 0.0;
  for (int b = rowptr[r]; b < rowptr[r + 1]; ++b) v += part[(size_t)b * TP + mu];
  yh[(size_t)r * p + mu] = v;
}

// f[pos] = b_n[perm[pos]] - (near history of pos's leaf row) - (far history:
// sum over the clusters r containing pos of Ue_r[pos - begin_r] . yh_r).
// hist = 0 at step 0.  One thread per tree position.
__global__ void k_mot_rhs(int n, int M, int p, int hist, const int* __restrict__ perm,
                          const int* __restrict__ leaf_of, const int* __restrict__ parent,
                          const int* __restrict__ begin, const int* __restrict__ near_rowptr,
                          const double* __restrict__ part_near, const double* __restrict__ Ue,
                          const int64_t* __restrict__ uoff, const double* __restrict__ yh,
                          const double* __restrict__ b, double* __restrict__ f) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= M) return;
  double v = b[(size_t)n * M + perm[pos]];
  if (hist) {
    const int lf = leaf_of[pos];
    const int i = pos - begin[lf];
    double h = 0.0;
    for (int bb = near_rowptr[lf]; bb < near_rowptr[lf + 1]; ++bb) h += part_near[(size_t)bb * 32 + i];
    for (int r = lf; r >= 0; r = parent[r]) {
      const double* u = Ue + uoff[r] + (size_t)(pos - begin[r]) * p;
      const double* y = yh + (size_t)r * p;
      for (int mu = 0; mu < p; ++mu) h = fma(u[mu], y[mu], h);
    }
    v -= h;
  }
  f[pos] = v;
}

// qt[n][a] = sum_b Ainv[a][b] f[b]: a warp per row.
__global__ void __launch_bounds__(256) k_mot_gemv(int M, const double* __restrict__ Ainv,
                                                  const double* __restrict__ f, double* __restrict__ q,
                                                  float2* __restrict__ qff) {
  const int a = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (a >= M) return;
  const double* row = Ainv + (size_t)a * M;
  double v = 0.0;
  for (int j = lane; j < M; j += 32) v = fma(row[j], f[j], v);
  v = warp_sum(v);
  if (lane == 0) {
    q[a] = v;
    if (qff) {
      const ff vf = ff_of(v);
      qff[a] = make_float2(vf.h, vf.l);
    }
  }
}

// xhat_r(n)[mu] = sum_i Ue_r[i][mu] q_n[begin_r + i] for every node r; one CTA
// per node, four row groups reduced in shared memory.
__global__ void __launch_bounds__(256) k_mot_forward(int n, int L, int p, const int* __restrict__ begin,
                                                     const int* __restrict__ end, const double* __restrict__ Ue,
                                                     const int64_t* __restrict__ uoff,
                                                     const double* __restrict__ q, double* __restrict__ Xh,
                                                     float2* __restrict__ Xff) {
  __shared__ double red[4][TP];
  const int r = blockIdx.x;
  const int rb = begin[r], nr = end[r] - rb;
  const int mu = threadIdx.x & 63, g = threadIdx.x >> 6;
  const double* u = Ue + uoff[r];
  double v = 0.0;
  if (mu < p)
    for (int i = g; i < nr; i += 4) v = fma(u[(size_t)i * p + mu], q[rb + i], v);
  red[g][mu] = v;
  __syncthreads();
  if (g == 0 && mu < p) {
    const double x = (red[0][mu] + red[1][mu]) + (red[2][mu] + red[3][mu]);
    Xh[((size_t)r * L + n) * p + mu] = x;
    if (Xff) {
      const ff xf = ff_of(x);
      Xff[((size_t)r * L + n) * p + mu] = make_float2(xf.h, xf.l);
    }
  }
}

// q[n][perm[pos]] = qt[n][pos]
__global__ void k_mot_untree_q(int L, int M, const int* __restrict__ perm, const double* __restrict__ qt,
                               double* __restrict__ q) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)L * M) return;
  const int n = (int)(e / M), pos = (int)(e - (int64_t)n * M);
  q[(size_t)n * M + perm[pos]] = qt[e];
}

__global__ void k_mot_leaf_of(int n_nodes, const int* __restrict__ son0, const int* __restrict__ begin,
                              const int* __restrict__ end, int* __restrict__ leaf_of) {
  const int r = blockIdx.x;
  if (son0[r] >= 0) return;
  for (int pos = begin[r] + threadIdx.x; pos < end[r]; pos += blockDim.x) leaf_of[pos] = r;
}

// ---- host --------------------------------------------------------------

void mot_release(cqm_handle* h) {
  Allocator& A = h->alloc;
  h->mot_dn.free(A);
  h->mot_df.free(A);
  h->mot_Ue.free(A);
  h->mot_Ainv.free(A);
  h->mot_Ue_off.free(A);
  h->mot_dn_ff.free(A);
  h->mot_df_ff.free(A);
  h->mot_ready = false;
}

// Dense Vhat_n in tree order into A (M x M).
static int assemble_weight(cqm_handle* h, int n, double* A) {
  const int ff = h->factors_ff ? 1 : 0;
  if (h->n_near > 0)
    k_mot_weight_near<<<h->n_near, 256, 0, h->stream>>>(n, h->L, h->rank_cap, h->M, h->near_rc.p,
                                                         h->node_begin.p, h->node_end.p, h->near_off.p,
                                                         h->near_rank.p, h->nearC.p, ff, h->mot_dn.p, A);
  if (h->n_far > 0)
    k_mot_weight_far<<<h->n_far, 256, 0, h->stream>>>(n, h->L, h->rank_cap, h->M, h->p, h->far_rc.p,
                                                       h->node_begin.p, h->node_end.p, h->far_rank.p,
                                                       h->farC.p, ff, h->mot_df.p, h->mot_Ue.p,
                                                       h->mot_Ue_off.p, A);
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

// Transformed fibres (eq. fastdft), explicit bases, Vhat_0 and its inverse.
int mot_prepare(cqm_handle* h) {
  if (h->mot_ready) return CQM_OK;
  if (h->params.mode != CQM_MODE_H2MACA) {
    set_last_error("marching on in time needs the H2MACA mode");
    return CQM_EINVAL;
  }
  Allocator& A = h->alloc;
  const int L = h->L, Ls = h->Ls, cap = h->rank_cap, M = h->M, p = h->p;
  cudaStream_t S = h->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CQM_CUDA_TRY(cudaEventCreate(&e0));
  CQM_CUDA_TRY(cudaEventCreate(&e1));
  cudaEventRecord(e0, S);
  int st = CQM_OK;
  DArray<double2> tw;
  DArray<double> P, colbuf;
  do {
    ProfScope ps_(h, CQM_K_MOT_WEIGHTS);
    if ((st = tw.allocate(A, L)) != CQM_OK) break;
    k_mot_twiddles<<<grid_for(L, 256), 256, 0, S>>>(L, tw.p);
    const size_t sh = sizeof(double2) * Ls;
    if (sh > 48 * 1024 &&
        cudaFuncSetAttribute(k_mot_fastdft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh) != cudaSuccess) {
      set_last_error("marching on in time: shared memory of the fibre transform");
      st = CQM_ECUDA;
      break;
    }
    if ((st = h->mot_dn.allocate(A, (size_t)std::max(1, h->n_near) * cap * L)) != CQM_OK) break;
    if ((st = h->mot_df.allocate(A, (size_t)std::max(1, h->n_far) * cap * L)) != CQM_OK) break;
    if (h->n_near > 0)
      k_mot_fastdft<<<h->n_near, 256, sh, S>>>(L, Ls, cap, h->R, h->near_rank.p, h->nearD.p, tw.p, h->mot_dn.p);
    if (h->n_far > 0)
      k_mot_fastdft<<<h->n_far, 256, sh, S>>>(L, Ls, cap, h->R, h->far_rank.p, h->farD.p, tw.p, h->mot_df.p);
    if (h->factors_ff) {  // float-float copies for the history sums
      if ((st = h->mot_dn_ff.allocate(A, h->mot_dn.n)) != CQM_OK) break;
      if ((st = h->mot_df_ff.allocate(A, h->mot_df.n)) != CQM_OK) break;
      k_mot_to_ffc<<<grid_for((int64_t)h->mot_dn.n, 256), 256, 0, S>>>((int64_t)h->mot_dn.n, h->mot_dn.p,
                                                                        h->mot_dn_ff.p);
      k_mot_to_ffc<<<grid_for((int64_t)h->mot_df.n, 256), 256, 0, S>>>((int64_t)h->mot_df.n, h->mot_df.p,
                                                                        h->mot_df_ff.p);
    }
    // explicit bases, deepest level first
    std::vector<int64_t> off(h->n_nodes + 1, 0);
    for (int r = 0; r < h->n_nodes; ++r) off[r + 1] = off[r] + (int64_t)(h->h_end[r] - h->h_begin[r]) * p;
    if ((st = h->mot_Ue_off.allocate(A, h->n_nodes + 1)) != CQM_OK) break;
    if ((st = h->mot_Ue.allocate(A, (size_t)std::max<int64_t>(1, off[h->n_nodes]))) != CQM_OK) break;
    if (cudaMemcpyAsync(h->mot_Ue_off.p, off.data(), sizeof(int64_t) * (h->n_nodes + 1),
                        cudaMemcpyHostToDevice, S) != cudaSuccess) {
      st = CQM_ECUDA;
      break;
    }
    for (int lv = (int)h->level_begin.size() - 2; lv >= 0; --lv) {
      const int n0 = h->level_begin[lv], cnt = h->level_begin[lv + 1] - n0;
      if (cnt > 0)
        k_mot_bases<<<cnt, 256, 0, S>>>(n0, h->m, p, h->node_begin.p, h->node_end.p, h->node_son0.p,
                                        h->node_son1.p, h->Uleaf.p, h->Etr.p, h->mot_Ue_off.p, h->mot_Ue.p);
    }
    // Vhat_0 and its inverse (blocked Gauss-Jordan)
    if ((st = h->mot_Ainv.allocate(A, (size_t)M * M)) != CQM_OK) break;
    if ((st = assemble_weight(h, 0, h->mot_Ainv.p)) != CQM_OK) break;
    const int nb = (M + GJ - 1) / GJ;
    if ((st = P.allocate(A, GJ * GJ)) != CQM_OK) break;
    if ((st = colbuf.allocate(A, (size_t)nb * GJ * GJ)) != CQM_OK) break;
    for (int K = 0; K < nb; ++K) {
      k_gj_diag<<<1, GJ * GJ, 0, S>>>(K, M, h->mot_Ainv.p, P.p);
      k_gj_row<<<nb, GJ * GJ, 0, S>>>(K, M, h->mot_Ainv.p, P.p, colbuf.p);
      k_gj_update<<<dim3(nb, nb), GJ * GJ, 0, S>>>(K, M, h->mot_Ainv.p, P.p, colbuf.p);
    }
    if (cudaGetLastError() != cudaSuccess) {
      set_last_error("marching on in time: weight launches failed");
      st = CQM_ECUDA;
    }
  } while (false);
  cudaEventRecord(e1, S);
  if (st == CQM_OK && cudaStreamSynchronize(S) != cudaSuccess) {
    set_last_error("marching on in time: weights failed");
    st = CQM_ECUDA;
  }
  float ms = 0.f;
  if (st == CQM_OK) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tw.free(A);
  P.free(A);
  colbuf.free(A);
  if (st != CQM_OK) {
    mot_release(h);
    return st;
  }
  h->mot_setup_ms = ms;
  h->mot_ready = true;
  return CQM_OK;
}

int mot_weight(cqm_handle* h, int n, double* d_W) {
  if (n < 0 || n > h->N) {
    set_last_error("step index out of range");
    return CQM_EINVAL;
  }
  CQM_TRY(mot_prepare(h));
  DArray<double> T;
  CQM_TRY(T.allocate(h->alloc, (size_t)h->M * h->M));
  int st = assemble_weight(h, n, T.p);
  if (st == CQM_OK) {
    const int64_t MM = (int64_t)h->M * h->M;
    k_mot_untree<<<grid_for(MM, 256), 256, 0, h->stream>>>(h->M, h->perm.p, T.p, d_W);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) {
      set_last_error("marching on in time: weight assembly failed");
      st = CQM_ECUDA;
    }
  }
  T.free(h->alloc);
  return st;
}

// q_n for n = 0..N by marching on in time; d_b, d_q: (L, M) device, caller's
// numbering.
int mot_solve(cqm_handle* h, const double* d_b, double* d_q, cqm_solve_info* info) {
  CQM_TRY(mot_prepare(h));
  Allocator& A = h->alloc;
  const int L = h->L, M = h->M, p = h->p, cap = h->rank_cap, nn = h->n_nodes;
  const int ff = h->factors_ff ? 1 : 0;
  cudaStream_t S = h->stream;
  DArray<double> qt, Xh, pn, pf, yh, f;
  DArray<float2> qff, Xff;
  DArray<int> leaf_of;
  const bool ffh = h->factors_ff && h->mot_dn_ff.p != nullptr;  // float-float history sums
  auto release = [&]() {
    qt.free(A); Xh.free(A); pn.free(A); pf.free(A); yh.free(A); f.free(A); leaf_of.free(A);
    qff.free(A); Xff.free(A);
  };
  int st = CQM_OK;
#define MOT_TRY(e) do { if ((st = (e)) != CQM_OK) { release(); return st; } } while (0)
  MOT_TRY(qt.allocate(A, (size_t)L * M));
  MOT_TRY(Xh.allocate(A, (size_t)nn * L * p));
  MOT_TRY(pn.allocate(A, (size_t)std::max(1, h->n_near) * 32));
  MOT_TRY(pf.allocate(A, (size_t)std::max(1, h->n_far) * TP));
  MOT_TRY(yh.allocate(A, (size_t)nn * p));
  MOT_TRY(f.allocate(A, M));
  MOT_TRY(leaf_of.allocate(A, M));
  if (ffh) {
    MOT_TRY(qff.allocate(A, (size_t)L * M));
    MOT_TRY(Xff.allocate(A, (size_t)nn * L * p));
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    release();
    set_last_error("cudaEventCreate failed");
    return CQM_ECUDA;
  }
  cudaMemsetAsync(yh.p, 0, sizeof(double) * nn * p, S);
  k_mot_leaf_of<<<nn, 128, 0, S>>>(nn, h->node_son0.p, h->node_begin.p, h->node_end.p, leaf_of.p);
  cudaEventRecord(e0, S);
  for (int n = 0; n < L; ++n) {
    const int hist = n > 0 ? 1 : 0;
    {
      ProfScope ps_(h, CQM_K_MOT_HISTORY);
      if (hist && h->n_near > 0) {
        if (ffh)
          k_mot_hist_near_ff<<<h->n_near, 256, 0, S>>>(n, L, cap, M, h->near_rc.p, h->node_begin.p,
                                                       h->node_end.p, h->near_off.p, h->near_rank.p,
                                                       (const float4*)h->nearC.p, h->mot_dn_ff.p, qff.p, pn.p);
        else
          k_mot_hist_near<<<h->n_near, 256, 0, S>>>(n, L, cap, M, h->near_rc.p, h->node_begin.p,
                                                    h->node_end.p, h->near_off.p, h->near_rank.p,
                                                    h->nearC.p, ff, h->mot_dn.p, qt.p, pn.p);
      }
      if (hist && h->n_far > 0) {
        if (ffh)
          k_mot_hist_far_ff<<<h->n_far, 256, 0, S>>>(n, L, cap, p, h->far_rc.p, h->far_rank.p,
                                                     (const float4*)h->farC.p, h->mot_df_ff.p, Xff.p, pf.p);
        else
          k_mot_hist_far<<<h->n_far, 256, 0, S>>>(n, L, cap, p, h->far_rc.p, h->far_rank.p, h->farC.p, ff,
                                                  h->mot_df.p, Xh.p, pf.p);
        k_mot_reduce_far<<<nn, TP, 0, S>>>(p, h->far_rowptr.p, pf.p, yh.p);
      }
      k_mot_rhs<<<grid_for(M, 256), 256, 0, S>>>(n, M, p, hist, h->perm.p, leaf_of.p, h->node_parent.p,
                                                 h->node_begin.p, h->near_rowptr.p, pn.p, h->mot_Ue.p,
                                                 h->mot_Ue_off.p, yh.p, d_b, f.p);
    }
    {
      ProfScope ps_(h, CQM_K_MOT_STEP);
      k_mot_gemv<<<grid_for(M, 8), 256, 0, S>>>(M, h->mot_Ainv.p, f.p, qt.p + (size_t)n * M,
                                                 ffh ? qff.p + (size_t)n * M : nullptr);
      if (n + 1 < L)
        k_mot_forward<<<nn, 256, 0, S>>>(n, L, p, h->node_begin.p, h->node_end.p, h->mot_Ue.p,
                                         h->mot_Ue_off.p, qt.p + (size_t)n * M, Xh.p,
                                         ffh ? Xff.p : nullptr);
    }
    if (cudaGetLastError() != cudaSuccess) {
      set_last_error("marching on in time: step launch failed");
      st = CQM_ECUDA;
      break;
    }
  }
  if (st == CQM_OK)
    k_mot_untree_q<<<grid_for((int64_t)L * M, 256), 256, 0, S>>>(L, M, h->perm.p, qt.p, d_q);
  cudaEventRecord(e1, S);
  if (st == CQM_OK && (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(S) != cudaSuccess)) {
    set_last_error("marching on in time failed");
    st = CQM_ECUDA;
  }
  float ms = 0.f;
  if (st == CQM_OK) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release();
#undef MOT_TRY
  if (st != CQM_OK) return st;
  if (info) {
    info->iterations = L;  // time steps
    info->restarts = 0;
    info->converged = L;
    info->Ls = h->Ls;
    info->max_rel_residual = 0.0;
    info->max_imag = 0.0;
    info->t_forward_ms = h->mot_setup_ms;  // weights of the first call (0 after)
    info->t_gmres_ms = ms;
    info->t_inverse_ms = 0.0;
    info->arnoldi_vectors = info->arnoldi_freq_steps = info->restart_freq_applies = 0;
  }
  h->mot_setup_ms = 0.0;
  return CQM_OK;
}

}  // namespace cqm
