// Multivariate adaptive cross approximation of every block of the tensor
// partition over the solved frequencies (Sec. 5.1, Alg. 2; Alg. 3):
//   G^(l) = sum_{t<l} C_t x_3 d_t,  C_l = G[:,:,k_l] - G^(l-1)[:,:,k_l],
//   (i_l, j_l) = first argmax |C_l| (row-major), d_l = (G[i_l,j_l,:] -
//   G^(l-1)[i_l,j_l,:]) / C_l[i_l,j_l], k_{l+1} = argmax over unused k of
//   |d_l[k]| (ties: smallest k), k_1 = 0; stop when ||C_l||_F ||d_l||_2 <=
//   eps ||G^(l)||_F (norm from the Gram identity of Sec. 5.1), on a zero pivot
//   (|pivot| <= 1e-300) or when every frequency is used; every computed update
//   is kept.
// Near blocks take entries from the Galerkin quadrature (Alg. 3 NEAR), far
// blocks from the kernel at the Chebyshev points (Alg. 3 FAR).
// All blocks advance one rank step per round of four launches:
//   slice -> residual update + pivot + Gram(C) -> fibre -> finalize.
// The Galerkin matrix and the far-field kernel are symmetric and the
// partition is symmetric (one cluster tree for rows and columns), so only the
// blocks r <= c run the MACA; block (c, r) then takes the factors of (r, c)
// with every C_t transposed.
#include <algorithm>
#include <unordered_map>
#include <vector>

#include "ffexp.cuh"
#include "handle.cuh"

namespace cqm {

struct MacaBlocks {
  int n;            // blocks
  int kind;         // 0 near, 1 far
  int Ls, cap, p, m;
  const int2* rc;   // (row, col) clusters
  const int* begin;
  const int* end;
  const int* perm;
  const double* cheb;  // far: Chebyshev nodes
  const int64_t* off;  // near: C slot base per block
  double2* C;
  double2* D;          // (b * cap + t) * Ls
  int* rank;
  int* active;
  int* kcur;
  int2* piv;
  double2* pval;
  double* cn2;
  double* norm2;
  double2* gramc;      // b * cap + t
  unsigned* used;      // b * words
  int words;
  int* counters;       // [0] active blocks, [1] capacity overflow
  double eps;
  // near field: cached quadrature points (r, weight / (4 pi r)) of every pair;
  // pair k of block b is pair_base[b] + i * #c + j, its points start at pt_off[k]
  const int64_t* pt_off;
  const int* pt_cnt;
  const double* pt_r;
  const double* pt_c;
  // maca_ff: the cached near points hold float-float d = r - r0 and c (same
  // bytes as pt_r, pt_c), r0 per pair; far blocks' points in fpt_*; the
  // exponential tables as float-float pairs
  int ff;
  const double* pt_r0;
  const float2* fpt_d;
  const float2* fpt_c;
  const double* fpt_r0;
  const float2* t2ff;
  const float4* csff;
};

// The float-float exponential tables of a block, in shared memory.
struct FFTables {
  float2 t2[1024];
  float4 cs[1024];
};
__device__ __forceinline__ void load_ff_tables(FFTables& T, const MacaBlocks& B) {
  for (int k = threadIdx.x; k < 1024; k += blockDim.x) {
    T.t2[k] = B.t2ff[k];
    T.cs[k] = B.csff[k];
  }
  __syncthreads();
}

// Warp sum of a float-float value (result in every lane).
__device__ __forceinline__ ff warp_sum_ff(ff a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const ff b = {__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
    a = ff_add(a, b);
  }
  return a;
}

// sum over this lane's points k = lane, lane + 32, ... of c_k exp(-s d_k)
__device__ __forceinline__ void lane_points_ff(const float2* __restrict__ pd, const float2* __restrict__ pc,
                                               int n, int lane, const ffs& sf, const FFTables& T, ff& ar,
                                               ff& ai) {
  int cnt = 0;
  for (int k = lane; k < n; k += 32) {
    const float2 dd = pd[k], cc = pc[k];
    ff vr, vi;
    cexp_ff(ff{dd.x, dd.y}, ff{cc.x, cc.y}, sf, T.t2, T.cs, vr, vi);
    ff_acc(ar, vr);
    ff_acc(ai, vi);
    if ((++cnt & 15) == 0) {
      ff_norm(ar);
      ff_norm(ai);
    }
  }
  ff_norm(ar);
  ff_norm(ai);
}

__device__ __forceinline__ int rows_of(const MacaBlocks& B, int b) {
  return B.kind == 0 ? B.end[B.rc[b].x] - B.begin[B.rc[b].x] : B.p;
}
__device__ __forceinline__ int cols_of(const MacaBlocks& B, int b) {
  return B.kind == 0 ? B.end[B.rc[b].y] - B.begin[B.rc[b].y] : B.p;
}
__device__ __forceinline__ double2* slot(const MacaBlocks& B, int b, int t, int nr, int nc) {
  return B.kind == 0 ? B.C + B.off[b] + (size_t)t * nr * nc
                     : B.C + ((size_t)b * B.cap + t) * (size_t)B.p * B.p;
}

// Chebyshev point mu of cluster r.
__device__ __forceinline__ void cheb_point(const double* cheb, int r, int m, int mu, double* x) {
  const double* nd = cheb + (size_t)r * 3 * m;
  x[0] = nd[mu % m];
  x[1] = nd[m + (mu / m) % m];
  x[2] = nd[2 * m + mu / (m * m)];
}

__device__ __forceinline__ double2 kernel_value(double r, double2 s, const Quad& q) {
  return cexp_c(r, 1.0 / (CQM_FOUR_PI * r), s, q);
}

// Slice G[:,:,k] of every active block into slot rank[b].
__global__ void __launch_bounds__(256, 4) k_maca_slice(MacaBlocks B, Geom g, Quad q,
                                                    const double2* __restrict__ s) {
  const int b = blockIdx.x;
  if (!B.active[b]) return;
  const int nr = rows_of(B, b), nc = cols_of(B, b);
  const int t = B.rank[b];
  double2* out = slot(B, b, t, nr, nc);
  const double2 sk = s[B.kcur[b]];
  const int2 rc = B.rc[b];
  if (B.ff) {
    // entries E0 * sum_k c_k exp(-s d_k), E0 = exp(-s r0) in FP64, the sum in
    // float-float from the cached points
    __shared__ FFTables T;
    __shared__ double2 E0s;
    load_ff_tables(T, B);
    const ffs sf = ffs_of(sk);
    if (B.kind == 1) {
      if (threadIdx.x == 0) E0s = cexp_c(B.fpt_r0[b], 1.0, sk, q);
      __syncthreads();
      const double2 E0 = E0s;
      const size_t pp = (size_t)B.p * B.p;
      for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
        const float2 dd = B.fpt_d[(size_t)b * pp + e], cc = B.fpt_c[(size_t)b * pp + e];
        ff vr, vi;
        cexp_ff(ff{dd.x, dd.y}, ff{cc.x, cc.y}, sf, T.t2, T.cs, vr, vi);
        out[e] = cmul(make_double2(ff_to_double(vr), ff_to_double(vi)), E0);
      }
      return;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t base = B.off[b] / B.cap;
    const bool diag = rc.x == rc.y;
    const int npair = diag ? nr * (nr + 1) / 2 : nr * nc;
    const float2* pd = (const float2*)B.pt_r;
    const float2* pc = (const float2*)B.pt_c;
    // The warp's pairs e2 = w, w + nw, ... in groups of 32: lane kk owns pair
    // g0 + kk nw and keeps its sum, and the FP64 part (exp(-s r0), the
    // product, the conversion) runs once per group with every lane busy,
    // instead of on one lane per pair (an FP64 warp instruction costs the same
    // pipe time with one active lane as with 32).  Pairs of at most SMALL_PTS
    // points (the regular 7 x 7 rule) run four at a time on eight lanes each,
    // which spends a three-step reduction on each instead of a five-step one
    // and idles fewer lanes; the others run one at a time on the whole warp.
    constexpr int SMALL_PTS = 64;
    for (int g0 = w; g0 < npair; g0 += 32 * nw) {
      const int e2 = g0 + lane * nw;
      int i = 0, j = 0, e = -1, cnt = 0;
      int64_t o = 0;
      if (e2 < npair) {
        if (diag) {
          int rem = e2;
          while (rem >= nr - i) {
            rem -= nr - i;
            ++i;
          }
          j = i + rem;
        } else {
          i = e2 / nc;
          j = e2 - i * nc;
        }
        e = i * nc + j;
        o = B.pt_off[base + e];
        cnt = B.pt_cnt[base + e];
      }
      const unsigned small = __ballot_sync(0xffffffffu, e >= 0 && cnt <= SMALL_PTS);
      unsigned big = __ballot_sync(0xffffffffu, e >= 0 && cnt > SMALL_PTS);
      ff mr = {0.f, 0.f}, mim = {0.f, 0.f};
      const int sg = lane >> 3, sl = lane & 7;
      const int mypos = __popc(small & ((1u << lane) - 1u));  // rank among the small pairs
      const int nsmall = __popc(small);
      for (int it = 0; 4 * it < nsmall; ++it) {
        const int idx = 4 * it + sg;  // the small pair of this eight-lane group
        unsigned mm = small;
        for (int k = 0; k < idx && mm; ++k) mm &= mm - 1u;
        const int src = idx < nsmall ? __ffs(mm) - 1 : 0;
        // every lane takes part in both shuffles; idle groups get no points
        const int64_t po = __shfl_sync(0xffffffffu, o, src);
        const int pn_src = __shfl_sync(0xffffffffu, cnt, src);
        const int pn = idx < nsmall ? pn_src : 0;
        ff ar = {0.f, 0.f}, ai = {0.f, 0.f};
        for (int k = sl; k < pn; k += 8) {
          const float2 dd = pd[po + k], cc = pc[po + k];
          ff vr, vi;
          cexp_ff(ff{dd.x, dd.y}, ff{cc.x, cc.y}, sf, T.t2, T.cs, vr, vi);
          ff_acc(ar, vr);
          ff_acc(ai, vi);
        }
        ff_norm(ar);
        ff_norm(ai);
#pragma unroll
        for (int of = 4; of > 0; of >>= 1) {
          ar = ff_add(ar, ff{__shfl_xor_sync(0xffffffffu, ar.h, of), __shfl_xor_sync(0xffffffffu, ar.l, of)});
          ai = ff_add(ai, ff{__shfl_xor_sync(0xffffffffu, ai.h, of), __shfl_xor_sync(0xffffffffu, ai.l, of)});
        }
        // the owner of each of the four pairs takes its sum from the group's first lane
        const int from = 8 * (mypos & 3);
        const ff vr = {__shfl_sync(0xffffffffu, ar.h, from), __shfl_sync(0xffffffffu, ar.l, from)};
        const ff vi = {__shfl_sync(0xffffffffu, ai.h, from), __shfl_sync(0xffffffffu, ai.l, from)};
        if (((small >> lane) & 1u) && (mypos >> 2) == it) {
          mr = vr;
          mim = vi;
        }
      }
      while (big) {
        const int kk = __ffs(big) - 1;
        big &= big - 1u;
        const int64_t po = __shfl_sync(0xffffffffu, o, kk);
        const int pn = __shfl_sync(0xffffffffu, cnt, kk);
        ff ar = {0.f, 0.f}, ai = {0.f, 0.f};
        lane_points_ff(pd + po, pc + po, pn, lane, sf, T, ar, ai);
        ar = warp_sum_ff(ar);
        ai = warp_sum_ff(ai);
        if (lane == kk) {
          mr = ar;
          mim = ai;
        }
      }
      if (e >= 0) {
        const double2 E0 = cexp_c(B.pt_r0[base + e], 1.0, sk, q);
        const double2 v = cmul(make_double2(ff_to_double(mr), ff_to_double(mim)), E0);
        out[e] = v;
        if (diag) out[j * nc + i] = v;
      }
    }
    return;
  }
  if (B.kind == 1) {
    for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
      const int mu = e / nc, nu = e - mu * nc;
      double xr[3], xc[3];
      cheb_point(B.cheb, rc.x, B.m, mu, xr);
      cheb_point(B.cheb, rc.y, B.m, nu, xc);
      const double d0 = xc[0] - xr[0], d1 = xc[1] - xr[1], d2 = xc[2] - xr[2];
      out[e] = kernel_value(sqrt(d0 * d0 + d1 * d1 + d2 * d2), sk, q);
    }
    return;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rb = B.begin[rc.x], cb = B.begin[rc.y];
  double2 sv[1] = {sk};
  if (B.pt_r) {
    // a diagonal block evaluates its pairs i <= j (the pair order is
    // canonical, so V[i][j] and V[j][i] are the same sum) and writes both
    const int64_t base = B.off[b] / B.cap;
    const bool diag = rc.x == rc.y;
    const int npair = diag ? nr * (nr + 1) / 2 : nr * nc;
    for (int e2 = w; e2 < npair; e2 += nw) {
      int i, j;
      if (diag) {  // e2 -> (i, j), i <= j, row-major over the upper triangle
        i = 0;
        int rem = e2;
        while (rem >= nr - i) {
          rem -= nr - i;
          ++i;
        }
        j = i + rem;
      } else {
        i = e2 / nc;
        j = e2 - i * nc;
      }
      const int e = i * nc + j;
      const int64_t o = B.pt_off[base + e];
      const int n = B.pt_cnt[base + e];
      double2 acc[1] = {make_double2(0.0, 0.0)};
      for (int k = lane; k < n; k += 32) kernel_accumulate_c<1>(B.pt_r[o + k], B.pt_c[o + k], sv, 1, acc, q);
      acc[0] = warp_sum2(acc[0]);
      if (lane == 0) {
        out[e] = acc[0];
        if (diag) out[j * nc + i] = acc[0];
      }
    }
    return;
  }
  for (int e = w; e < nr * nc; e += nw) {
    const int i = e / nc, j = e - i * nc;
    const int I = B.perm[rb + i], J = B.perm[cb + j];
    double2 acc[1] = {make_double2(0.0, 0.0)};
    const int cse = pair_case(g, q, I, J);
    pair_accumulate<1>(g, q, I, J, cse, lane, 32, sv, 1, acc);
    acc[0] = warp_sum2(acc[0]);
    if (lane == 0) out[e] = acc[0];
  }
}

// Residual update of the new slice, pivot search, ||C_l||^2 and <C_t, C_l>.
__global__ void __launch_bounds__(256) k_maca_pivot(MacaBlocks B) {
  __shared__ double sh[32];
  __shared__ double s_best[32];
  __shared__ int s_bidx[32];
  __shared__ double2 dk[64];
  const int b = blockIdx.x;
  if (!B.active[b]) return;
  const int nr = rows_of(B, b), nc = cols_of(B, b), n = nr * nc;
  const int l = B.rank[b];
  const int k = B.kcur[b];
  for (int t = threadIdx.x; t < l; t += blockDim.x) dk[t] = B.D[((size_t)b * B.cap + t) * B.Ls + k];
  __syncthreads();
  double2* Cl = slot(B, b, l, nr, nc);
  double best = -1.0, nrm = 0.0;
  int bidx = 0x7fffffff;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    double2 v = Cl[e];
    for (int t = 0; t < l; ++t) {
      const double2 c = slot(B, b, t, nr, nc)[e];
      v = csub(v, cmul(c, dk[t]));
    }
    Cl[e] = v;
    const double a = cabs2(v);
    nrm += a;
    if (a > best) { best = a; bidx = e; }
  }
  // block argmax: largest |v|^2, smallest index on ties
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
  }
  if (lane == 0) { s_best[warp] = best; s_bidx[warp] = bidx; }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    best = lane < nw ? s_best[lane] : -1.0;
    bidx = lane < nw ? s_bidx[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if (lane == 0) { s_best[0] = best; s_bidx[0] = bidx; }
  }
  __syncthreads();
  nrm = block_sum(nrm, sh);
  const int pi = s_bidx[0];
  if (threadIdx.x == 0) {
    const double2 pv = Cl[pi];
    B.piv[b] = make_int2(pi / nc, pi - (pi / nc) * nc);
    B.pval[b] = pv;
    B.cn2[b] = nrm;
    if (!(sqrt(cabs2(pv)) > 1e-300)) {
      B.active[b] = 0;
      atomicSub(&B.counters[0], 1);
    }
  }
  // Gram products <C_t, C_l> = sum conj(C_t) C_l
  for (int t = 0; t < l; ++t) {
    const double2* Ct = slot(B, b, t, nr, nc);
    double re = 0.0, im = 0.0;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const double2 a = Ct[e], c = Cl[e];
      re += a.x * c.x + a.y * c.y;
      im += a.x * c.y - a.y * c.x;
    }
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    if (threadIdx.x == 0) B.gramc[(size_t)b * B.cap + t] = make_double2(re, im);
  }
}

// Fibre G[i_l, j_l, :] of every active block into D slot rank[b] (raw).
__global__ void __launch_bounds__(256, 2) k_maca_fibre(MacaBlocks B, Geom g, Quad q,
                                                    const double2* __restrict__ s) {
  const int b = blockIdx.x;
  if (!B.active[b]) return;
  const int l = B.rank[b];
  double2* out = B.D + ((size_t)b * B.cap + l) * B.Ls;
  const int2 rc = B.rc[b];
  const int2 pv = B.piv[b];
  if (B.kind == 1) {
    double xr[3], xc[3];
    cheb_point(B.cheb, rc.x, B.m, pv.x, xr);
    cheb_point(B.cheb, rc.y, B.m, pv.y, xc);
    const double d0 = xc[0] - xr[0], d1 = xc[1] - xr[1], d2 = xc[2] - xr[2];
    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    for (int k = threadIdx.x; k < B.Ls; k += blockDim.x) out[k] = kernel_value(r, s[k], q);
    return;
  }
  const int I = B.perm[B.begin[rc.x] + pv.x], J = B.perm[B.begin[rc.y] + pv.y];
  const int cse = pair_case(g, q, I, J);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int NF = 8;
  if (B.ff) {
    __shared__ FFTables T;
    load_ff_tables(T, B);
    const int nc = B.end[rc.y] - B.begin[rc.y];
    const bool swap = rc.x == rc.y && pv.x > pv.y;
    const int64_t k = B.off[b] / B.cap + (swap ? (int64_t)pv.y * nc + pv.x : (int64_t)pv.x * nc + pv.y);
    const int64_t o = B.pt_off[k];
    const int n = B.pt_cnt[k];
    const double r0 = B.pt_r0[k];
    const float2* pd = (const float2*)B.pt_r + o;
    const float2* pc = (const float2*)B.pt_c + o;
    // lane gi NF + f keeps frequency f of the warp's group gi; the FP64 part
    // (exp(-s r0), the product, the conversion) runs for 32 / NF groups at once
    ff mr = {0.f, 0.f}, mim = {0.f, 0.f};
    int mf = -1, gi = 0;
    for (int f0 = w * NF; f0 < B.Ls; f0 += nw * NF) {
      const int nf = min(NF, B.Ls - f0);
      ffs sv[NF];
      ff ar[NF], ai[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        sv[f] = ffs_of(f < nf ? s[f0 + f] : make_double2(0.0, 0.0));
        ar[f] = ai[f] = ff{0.f, 0.f};
      }
      int cnt = 0;
      for (int p = lane; p < n; p += 32) {
        const float2 dd = pd[p], cc = pc[p];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          ff vr, vi;
          cexp_ff(ff{dd.x, dd.y}, ff{cc.x, cc.y}, sv[f], T.t2, T.cs, vr, vi);
          ff_acc(ar[f], vr);
          ff_acc(ai[f], vi);
        }
        if ((++cnt & 15) == 0) {
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            ff_norm(ar[f]);
            ff_norm(ai[f]);
          }
        }
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        ff_norm(ar[f]);
        ff_norm(ai[f]);
        ar[f] = warp_sum_ff(ar[f]);
        ai[f] = warp_sum_ff(ai[f]);
      }
#pragma unroll
      for (int f = 0; f < NF; ++f)
        if (lane == gi * NF + f && f < nf) {
          mr = ar[f];
          mim = ai[f];
          mf = f0 + f;
        }
      if (++gi == 32 / NF) {
        if (mf >= 0)  // frequency mf scaled by exp(-s r0)
          out[mf] = cmul(make_double2(ff_to_double(mr), ff_to_double(mim)), cexp_c(r0, 1.0, s[mf], q));
        mf = -1;
        gi = 0;
      }
    }
    if (mf >= 0) out[mf] = cmul(make_double2(ff_to_double(mr), ff_to_double(mim)), cexp_c(r0, 1.0, s[mf], q));
    return;
  }
  if (B.pt_r) {
    const int nc = B.end[rc.y] - B.begin[rc.y];
    // a diagonal block caches its pairs i <= j only; (i, j) and (j, i) are one pair
    const bool swap = rc.x == rc.y && pv.x > pv.y;
    const int64_t k = B.off[b] / B.cap + (swap ? (int64_t)pv.y * nc + pv.x : (int64_t)pv.x * nc + pv.y);
    const int64_t o = B.pt_off[k];
    const int n = B.pt_cnt[k];
    for (int f0 = w * NF; f0 < B.Ls; f0 += nw * NF) {
      const int nf = min(NF, B.Ls - f0);
      double2 sv[NF], acc[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        sv[f] = f < nf ? s[f0 + f] : make_double2(0.0, 0.0);
        acc[f] = make_double2(0.0, 0.0);
      }
      for (int p = lane; p < n; p += 32) kernel_accumulate_c<NF>(B.pt_r[o + p], B.pt_c[o + p], sv, nf, acc, q);
#pragma unroll
      for (int f = 0; f < NF; ++f) acc[f] = warp_sum2(acc[f]);
      if (lane == 0)
        for (int f = 0; f < nf; ++f) out[f0 + f] = acc[f];
    }
    return;
  }
  for (int f0 = w * NF; f0 < B.Ls; f0 += nw * NF) {
    const int nf = min(NF, B.Ls - f0);
    double2 sv[NF], acc[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      sv[f] = f < nf ? s[f0 + f] : make_double2(0.0, 0.0);
      acc[f] = make_double2(0.0, 0.0);
    }
    pair_accumulate<NF>(g, q, I, J, cse, lane, 32, sv, nf, acc);
#pragma unroll
    for (int f = 0; f < NF; ++f) acc[f] = warp_sum2(acc[f]);
    if (lane == 0)
      for (int f = 0; f < nf; ++f) out[f0 + f] = acc[f];
  }
}

// d_l = (fibre - sum_t C_t[i,j] d_t) / pivot, Gram <d_t, d_l>, norm update,
// stopping test and the next slice.
__global__ void __launch_bounds__(256) k_maca_finalize(MacaBlocks B) {
  __shared__ double sh[32];
  __shared__ double2 cij[64];
  __shared__ double s_best[32];
  __shared__ int s_bidx[32];
  const int b = blockIdx.x;
  if (!B.active[b]) return;
  const int nr = rows_of(B, b), nc = cols_of(B, b);
  const int l = B.rank[b];
  const int2 pv = B.piv[b];
  const double2 piv = B.pval[b];
  const int pe = pv.x * nc + pv.y;
  for (int t = threadIdx.x; t < l; t += blockDim.x) cij[t] = slot(B, b, t, nr, nc)[pe];
  __syncthreads();
  double2* dl = B.D + ((size_t)b * B.cap + l) * B.Ls;
  double dn = 0.0;
  for (int k = threadIdx.x; k < B.Ls; k += blockDim.x) {
    double2 v = dl[k];
    for (int t = 0; t < l; ++t) v = csub(v, cmul(cij[t], B.D[((size_t)b * B.cap + t) * B.Ls + k]));
    v = cdiv(v, piv);
    dl[k] = v;
    dn += cabs2(v);
  }
  dn = block_sum(dn, sh);
  double cross = 0.0;  // 2 Re sum_t <C_t,C_l> <d_t,d_l>
  for (int t = 0; t < l; ++t) {
    const double2* dt = B.D + ((size_t)b * B.cap + t) * B.Ls;
    double re = 0.0, im = 0.0;
    for (int k = threadIdx.x; k < B.Ls; k += blockDim.x) {
      const double2 a = dt[k], c = dl[k];
      re += a.x * c.x + a.y * c.y;
      im += a.x * c.y - a.y * c.x;
    }
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    const double2 gc = B.gramc[(size_t)b * B.cap + t];
    cross += 2.0 * (gc.x * re - gc.y * im);
  }
  // next slice: argmax |d_l[k]| over unused k, smallest k on ties
  unsigned* used = B.used + (size_t)b * B.words;
  const int kc = B.kcur[b];
  double best = -1.0;
  int bidx = 0x7fffffff;
  for (int k = threadIdx.x; k < B.Ls; k += blockDim.x) {
    const bool u = (k == kc) || ((used[k >> 5] >> (k & 31)) & 1u);
    if (u) continue;
    const double a = cabs2(dl[k]);
    if (a > best || (a == best && k < bidx)) { best = a; bidx = k; }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
  }
  if (lane == 0) { s_best[warp] = best; s_bidx[warp] = bidx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int w2 = 1; w2 < nw; ++w2)
      if (s_best[w2] > best || (s_best[w2] == best && s_bidx[w2] < bidx)) { best = s_best[w2]; bidx = s_bidx[w2]; }
    used[kc >> 5] |= 1u << (kc & 31);
    const double n2 = B.norm2[b] + cross + B.cn2[b] * dn;
    B.norm2[b] = n2;
    const int r = l + 1;
    B.rank[b] = r;
    const bool small = sqrt(B.cn2[b]) * sqrt(dn) <= B.eps * sqrt(fmax(n2, 0.0));
    const bool all = (r >= B.Ls) || bidx == 0x7fffffff;
    bool done = small || all;
    if (!done && r >= B.cap) {
      atomicAdd(&B.counters[1], 1);
      done = true;
    }
    if (done) {
      B.active[b] = 0;
      atomicSub(&B.counters[0], 1);
    } else {
      B.kcur[b] = bidx;
    }
  }
}

__global__ void k_maca_init(int n, int words, const int2* __restrict__ rc, int* rank, int* active,
                            int* kcur, double* norm2, unsigned* used) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  rank[b] = 0;
  active[b] = rc[b].x <= rc[b].y ? 1 : 0;  // the lower blocks mirror the upper ones
  kcur[b] = 0;
  norm2[b] = 0.0;
  for (int w = 0; w < words; ++w) used[(size_t)b * words + w] = 0u;
}

// Block (c, r) of a lower-triangle block b takes the factors of its mirror
// (r, c): the same rank and d_t, every C_t transposed.
__global__ void __launch_bounds__(256) k_maca_mirror(MacaBlocks B, const int* __restrict__ mirror) {
  const int b = blockIdx.x;
  const int2 rc = B.rc[b];
  if (rc.x <= rc.y) return;
  const int m = mirror[b];
  const int rk = B.rank[m];
  const int nr = rows_of(B, b), nc = cols_of(B, b);  // the mirror is nc x nr
  if (threadIdx.x == 0) B.rank[b] = rk;
  for (int t = 0; t < rk; ++t) {
    const double2* src = slot(B, m, t, nc, nr);
    double2* dst = slot(B, b, t, nr, nc);
    for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
      const int i = e / nc, j = e - i * nc;
      dst[e] = src[(size_t)j * nr + i];
    }
    const double2* ds = B.D + ((size_t)m * B.cap + t) * B.Ls;
    double2* dd = B.D + ((size_t)b * B.cap + t) * B.Ls;
    for (int l = threadIdx.x; l < B.Ls; l += blockDim.x) dd[l] = ds[l];
  }
}

// Point counts of every pair of near block b (CTA per block) and their
// exclusive scan within the block; block totals for the global scan.
__global__ void __launch_bounds__(1024) k_pair_counts(const int2* __restrict__ rc, const int* __restrict__ begin,
                                                     const int* __restrict__ end, const int* __restrict__ perm,
                                                     const int64_t* __restrict__ off, int cap, Geom g, Quad q,
                                                     int* cnt, int64_t* pt_off, int64_t* block_total) {
  __shared__ int64_t sh[33];
  const int b = blockIdx.x;
  const int2 c2 = rc[b];
  const int rb = begin[c2.x], nr = end[c2.x] - rb, cb = begin[c2.y], nc = end[c2.y] - cb;
  const int64_t base = off[b] / cap;
  const int n = nr * nc;  // <= 1024 (leaves of at most 32)
  const bool upper = c2.x <= c2.y;  // lower blocks are mirrored, not evaluated
  int v = 0;
  if ((int)threadIdx.x < n) {
    const int i = threadIdx.x / nc, j = threadIdx.x - i * nc;
    const bool keep = upper && (c2.x != c2.y || i <= j);  // diagonal blocks: pairs i <= j
    v = keep ? pair_npoints(q, pair_case(g, q, perm[rb + i], perm[cb + j])) : 0;
    cnt[base + threadIdx.x] = v;
  }
  // block exclusive scan (int64)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int64_t wv = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
    int64_t z = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    sh[lane] = z - wv;
    if (lane == 31) sh[32] = z;
  }
  __syncthreads();
  if ((int)threadIdx.x < n) pt_off[base + threadIdx.x] = sh[warp] + x - v;
  if (threadIdx.x == 0) block_total[b] = sh[32];
}

// Exclusive scan of n int64 values in one CTA; out[n] = total.
__global__ void __launch_bounds__(1024) k_scan_i64(int n, const int64_t* __restrict__ in, int64_t* out) {
  __shared__ int64_t sh[33];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int b0 = 0; b0 < n; b0 += blockDim.x) {
    const int k = b0 + threadIdx.x;
    const int64_t v = k < n ? in[k] : 0;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const int64_t wv = sh[lane];
      int64_t z = wv;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= o) z += y;
      }
      sh[lane] = z - wv;
      if (lane == 31) sh[32] = z;
    }
    __syncthreads();
    if (k < n) out[k] = carry + sh[warp] + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += sh[32];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

// Radius of the ball about the centroid that holds triangle t.
__device__ __forceinline__ double tri_radius(const Geom& g, int t) {
  const double* P = g.P + 9 * t;
  const double* c = g.cen + 3 * t;
  double r2 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double dx = P[3 * k] - c[0], dy = P[3 * k + 1] - c[1], dz = P[3 * k + 2] - c[2];
    r2 = fmax(r2, dx * dx + dy * dy + dz * dz);
  }
  return sqrt(r2) * (1.0 + 1e-12);
}

// Geometry of every point of every pair of near block b: one warp per pair.
// With ff, the points hold float-float d = r - r0 and c (in the bytes of
// pt_r and pt_c) and pt_r0 the pair's bound r0 <= r: 0 for pairs that share a
// vertex, else the centroid distance minus the two triangles' radii.
__global__ void __launch_bounds__(256) k_pair_geometry(const int2* __restrict__ rc, const int* __restrict__ begin,
                                                      const int* __restrict__ end, const int* __restrict__ perm,
                                                      const int64_t* __restrict__ off, int cap, Geom g, Quad q,
                                                      const int64_t* __restrict__ block_base,
                                                      int64_t* pt_off, double* pt_r, double* pt_c,
                                                      int ff_mode, double* pt_r0) {
  const int b = blockIdx.x;
  const int2 c2 = rc[b];
  if (c2.x > c2.y) return;  // mirrored block: no points
  const int rb = begin[c2.x], nr = end[c2.x] - rb, cb = begin[c2.y], nc = end[c2.y] - cb;
  const int64_t base = off[b] / cap;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // The warp's pairs e = w, w + nw, ... in groups of 32, lane kk owning pair
  // g0 + kk nw: it converts the pair's offset, classifies it and forms r0
  // (FP64, once per pair with the warp's lanes on 32 pairs).  Regular pairs
  // (49 points) run four at a time on eight lanes each, which idles fewer
  // lanes than 49 points on 32; the others one at a time on the whole warp.
  // Every point is computed as before, so the cache is the same bit for bit.
  auto emit = [&](int I, int J, int cse, int sub, int nsub, int64_t o, double r0) {
    if (!ff_mode) {
      pair_points(g, q, I, J, cse, sub, nsub, [&](int k, double r, double c) {
        pt_r[o + k] = r;
        pt_c[o + k] = c;
      });
      return;
    }
    float2* pd = (float2*)pt_r;
    float2* pc = (float2*)pt_c;
    pair_points(g, q, I, J, cse, sub, nsub, [&](int k, double r, double c) {
      const ff d = ff_of(fmax(r - r0, 0.0)), cf = ff_of(c);
      pd[o + k] = make_float2(d.h, d.l);
      pc[o + k] = make_float2(cf.h, cf.l);
    });
  };
  for (int g0 = w; g0 < nr * nc; g0 += 32 * nw) {
    const int e = g0 + lane * nw;
    bool have = e < nr * nc;
    int i = 0, j = 0;
    if (have) {
      i = e / nc;
      j = e - i * nc;
      if (c2.x == c2.y && i > j) have = false;  // diagonal blocks cache their pairs i <= j
    }
    int I = 0, J = 0, cse = CASE_REGULAR;
    int64_t o = 0;
    double r0 = 0.0;
    if (have) {
      I = perm[rb + i];
      J = perm[cb + j];
      o = pt_off[base + e] + block_base[b];
      pt_off[base + e] = o;
      cse = pair_case(g, q, I, J);
      if (ff_mode) {
        if (cse == CASE_REGULAR || cse == CASE_NEAR) {
          const double* ci = g.cen + 3 * I;
          const double* cj = g.cen + 3 * J;
          const double dx = ci[0] - cj[0], dy = ci[1] - cj[1], dz = ci[2] - cj[2];
          r0 = fmax(0.0, sqrt(dx * dx + dy * dy + dz * dz) * (1.0 - 1e-12) - tri_radius(g, I) - tri_radius(g, J));
        }
        pt_r0[base + e] = r0;
      }
    }
    const unsigned small = __ballot_sync(0xffffffffu, have && cse == CASE_REGULAR);
    unsigned big = __ballot_sync(0xffffffffu, have && cse != CASE_REGULAR);
    const int sg = lane >> 3, sl = lane & 7, nsmall = __popc(small);
    for (int it = 0; 4 * it < nsmall; ++it) {
      const int idx = 4 * it + sg;  // the regular pair of this eight-lane group
      unsigned mm = small;
      for (int k = 0; k < idx && mm; ++k) mm &= mm - 1u;
      const int src = idx < nsmall ? __ffs(mm) - 1 : 0;
      // every lane takes part in the shuffles; idle groups emit nothing
      const int sI = __shfl_sync(0xffffffffu, I, src), sJ = __shfl_sync(0xffffffffu, J, src);
      const int64_t so = __shfl_sync(0xffffffffu, o, src);
      const double sr0 = __shfl_sync(0xffffffffu, r0, src);
      if (idx < nsmall) emit(sI, sJ, CASE_REGULAR, sl, 8, so, sr0);
    }
    while (big) {
      const int kk = __ffs(big) - 1;
      big &= big - 1u;
      const int sI = __shfl_sync(0xffffffffu, I, kk), sJ = __shfl_sync(0xffffffffu, J, kk);
      const int scse = __shfl_sync(0xffffffffu, cse, kk);
      const int64_t so = __shfl_sync(0xffffffffu, o, kk);
      const double sr0 = __shfl_sync(0xffffffffu, r0, kk);
      emit(sI, sJ, scse, lane, 32, so, sr0);
    }
  }
}

// Kernel points of the far blocks (the Chebyshev pairs, Alg. 3 FAR) for the
// float-float slices: entry (mu, nu) of upper block b holds d = |xi_nu -
// xi_mu| - r0 and c = 1 / (4 pi |xi_nu - xi_mu|), r0 the distance of the
// boxes of the two clusters' Chebyshev points (a bound of every entry's).
__global__ void __launch_bounds__(256) k_far_points(const int2* __restrict__ rc, const double* __restrict__ cheb,
                                                   int m, int p, float2* fd, float2* fc, double* fr0) {
  const int b = blockIdx.x;
  const int2 c2 = rc[b];
  if (c2.x > c2.y) return;  // mirrored block: no MACA
  __shared__ double s_r0;
  if (threadIdx.x == 0) {
    const double* a = cheb + (size_t)c2.x * 3 * m;
    const double* z = cheb + (size_t)c2.y * 3 * m;
    double d2 = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
      double alo = a[ax * m], ahi = alo, zlo = z[ax * m], zhi = zlo;
      for (int k = 1; k < m; ++k) {
        alo = fmin(alo, a[ax * m + k]); ahi = fmax(ahi, a[ax * m + k]);
        zlo = fmin(zlo, z[ax * m + k]); zhi = fmax(zhi, z[ax * m + k]);
      }
      const double gap = fmax(0.0, fmax(zlo - ahi, alo - zhi));
      d2 += gap * gap;
    }
    s_r0 = sqrt(d2) * (1.0 - 1e-12);
    fr0[b] = s_r0;
  }
  __syncthreads();
  const double r0 = s_r0;
  const size_t pp = (size_t)p * p;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int mu = e / p, nu = e - mu * p;
    double xr[3], xc[3];
    cheb_point(cheb, c2.x, m, mu, xr);
    cheb_point(cheb, c2.y, m, nu, xc);
    const double d0 = xc[0] - xr[0], d1 = xc[1] - xr[1], d2 = xc[2] - xr[2];
    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const ff d = ff_of(fmax(r - r0, 0.0)), c = ff_of(1.0 / (CQM_FOUR_PI * r));
    fd[(size_t)b * pp + e] = make_float2(d.h, d.l);
    fc[(size_t)b * pp + e] = make_float2(c.h, c.l);
  }
}

static Geom geom_from(const cqm_handle* h);

// Quadrature points of every near-field pair, computed once for all MACA
// slices and fibres (r and weight / (4 pi r) per point).
static int build_point_cache(cqm_handle* h, int64_t n_pairs) {
  const int nb = h->n_near;
  if (nb == 0 || !h->params.cache_quadrature) return CQM_OK;
  CQM_TRY(h->pt_cnt.allocate(h->alloc, n_pairs));
  CQM_TRY(h->pt_off.allocate(h->alloc, n_pairs));
  DArray<int64_t> tot, bbase;
  int st = tot.allocate(h->alloc, nb);
  if (st == CQM_OK) st = bbase.allocate(h->alloc, nb + 1);
  int64_t npts = 0;
  if (st == CQM_OK) {
    const Geom g = geom_from(h);
    {
      ProfScope ps_(h, CQM_K_POINTS);
      k_pair_counts<<<nb, 1024, 0, h->stream>>>(h->near_rc.p, h->node_begin.p, h->node_end.p, h->perm.p,
                                               h->near_off.p, h->rank_cap, g, h->quad, h->pt_cnt.p,
                                               h->pt_off.p, tot.p);
      k_scan_i64<<<1, 1024, 0, h->stream>>>(nb, tot.p, bbase.p);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&npts, bbase.p + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream);
    h->h_block_points.assign(nb, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->h_block_points.data(), tot.p, sizeof(int64_t) * nb, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      set_last_error(std::string("point cache: ") + cudaGetErrorString(e));
      st = CQM_ECUDA;
    }
    if (st == CQM_OK) st = h->pt_r.allocate(h->alloc, std::max<int64_t>(npts, 1));
    if (st == CQM_OK) st = h->pt_c.allocate(h->alloc, std::max<int64_t>(npts, 1));
    if (st == CQM_OK) {
      ProfScope ps_(h, CQM_K_POINTS);
      const bool ffm = h->params.maca_ff != 0;
      if (ffm) st = h->pt_r0.allocate(h->alloc, std::max<int64_t>(n_pairs, 1));
      if (st == CQM_OK)
        k_pair_geometry<<<nb, 256, 0, h->stream>>>(h->near_rc.p, h->node_begin.p, h->node_end.p, h->perm.p,
                                                  h->near_off.p, h->rank_cap, g, h->quad, bbase.p,
                                                  h->pt_off.p, h->pt_r.p, h->pt_c.p, ffm ? 1 : 0,
                                                  h->pt_r0.p);
      if (cudaGetLastError() != cudaSuccess) st = CQM_ECUDA;
    }
  }
  tot.free(h->alloc);
  bbase.free(h->alloc);
  h->n_points = npts;
  return st;
}

static Geom geom_from(const cqm_handle* h) {
  Geom g;
  g.M = h->M; g.tri = h->tri.p; g.P = h->P.p; g.area = h->area.p; g.cen = h->cen.p; g.diam = h->diam.p;
  return g;
}

// Runs MACA on one list of blocks; fills rank (device and host).
static int run_maca(cqm_handle* h, int kind, int n, const int2* rc, DArray<double2>& C,
                    DArray<double2>& D, DArray<int>& rank, const int64_t* d_off, size_t c_entries,
                    const std::vector<int2>& h_rc, std::vector<int>& h_rank) {
  h_rank.assign(n, 0);
  if (n == 0) return CQM_OK;
  const int Ls = h->Ls, cap = h->rank_cap;
  CQM_TRY(C.allocate(h->alloc, c_entries));
  CQM_TRY(D.allocate(h->alloc, (size_t)n * cap * Ls));
  CQM_TRY(rank.allocate(h->alloc, n));
  DArray<int> active, kcur, counters, mirror;
  DArray<int2> piv;
  DArray<double2> pval, gramc;
  DArray<double> cn2, norm2;
  DArray<unsigned> used;
  const int words = (Ls + 31) / 32;
  auto release = [&]() {
    active.free(h->alloc); kcur.free(h->alloc); counters.free(h->alloc); piv.free(h->alloc);
    pval.free(h->alloc); gramc.free(h->alloc); cn2.free(h->alloc); norm2.free(h->alloc);
    used.free(h->alloc); mirror.free(h->alloc);
  };
  int st = CQM_OK;
#define MT(e) do { if ((st = (e)) != CQM_OK) { release(); return st; } } while (0)
  MT(active.allocate(h->alloc, n));
  MT(kcur.allocate(h->alloc, n));
  MT(counters.allocate(h->alloc, 4));
  MT(piv.allocate(h->alloc, n));
  MT(pval.allocate(h->alloc, n));
  MT(gramc.allocate(h->alloc, (size_t)n * cap));
  MT(cn2.allocate(h->alloc, n));
  MT(norm2.allocate(h->alloc, n));
  MT(used.allocate(h->alloc, (size_t)n * words));
  // mirror[b]: index of block (c, r) for b = (r, c)
  std::vector<int> h_mirror(n, -1);
  int n_upper = 0;
  {
    std::unordered_map<uint64_t, int> at;
    at.reserve(2 * (size_t)n);
    for (int b = 0; b < n; ++b) at[((uint64_t)(uint32_t)h_rc[b].x << 32) | (uint32_t)h_rc[b].y] = b;
    for (int b = 0; b < n; ++b) {
      const auto f = at.find(((uint64_t)(uint32_t)h_rc[b].y << 32) | (uint32_t)h_rc[b].x);
      if (f == at.end()) {
        release();
        set_last_error("block partition is not symmetric");
        return CQM_EINVAL;
      }
      h_mirror[b] = f->second;
      if (h_rc[b].x <= h_rc[b].y) ++n_upper;
    }
  }
  MT(mirror.allocate(h->alloc, n));
  if (cudaMemcpyAsync(mirror.p, h_mirror.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream) !=
      cudaSuccess) {
    release();
    return CQM_ECUDA;
  }
  MacaBlocks B;
  B.n = n; B.kind = kind; B.Ls = Ls; B.cap = cap; B.p = h->p; B.m = h->m;
  B.rc = rc; B.begin = h->node_begin.p; B.end = h->node_end.p; B.perm = h->perm.p;
  B.cheb = h->cheb.p; B.off = d_off; B.C = C.p; B.D = D.p; B.rank = rank.p;
  B.active = active.p; B.kcur = kcur.p; B.piv = piv.p; B.pval = pval.p; B.cn2 = cn2.p;
  B.norm2 = norm2.p; B.gramc = gramc.p; B.used = used.p; B.words = words;
  B.counters = counters.p; B.eps = h->params.aca_eps;
  const bool cached = kind == 0 && h->pt_r.p != nullptr;
  B.pt_off = cached ? h->pt_off.p : nullptr;
  B.pt_cnt = cached ? h->pt_cnt.p : nullptr;
  B.pt_r = cached ? h->pt_r.p : nullptr;
  B.pt_c = cached ? h->pt_c.p : nullptr;
  B.ff = 0;
  B.pt_r0 = nullptr;
  B.fpt_d = B.fpt_c = nullptr;
  B.fpt_r0 = nullptr;
  B.t2ff = h->exp_t2_ff.p;
  B.csff = h->exp_cs_ff.p;
  if (h->params.maca_ff && kind == 0 && cached) {
    B.ff = 1;
    B.pt_r0 = h->pt_r0.p;
  }
  if (h->params.maca_ff && kind == 1 && h->cache_far_points) {
    B.ff = 1;
    B.fpt_d = h->fpt_d.p;
    B.fpt_c = h->fpt_c.p;
    B.fpt_r0 = h->fpt_r0.p;
  }
  cudaStream_t S = h->stream;
  const Geom g = geom_from(h);
  {
    ProfScope ps_(h, CQM_K_MACA_FINALIZE);
    k_maca_init<<<grid_for(n, 256), 256, 0, S>>>(n, words, rc, rank.p, active.p, kcur.p, norm2.p, used.p);
  }
  int hc[2] = {n_upper, 0};
  cudaMemcpyAsync(counters.p, hc, 2 * sizeof(int), cudaMemcpyHostToDevice, S);
  for (int step = 0; step < cap; ++step) {
    {
      ProfScope ps_(h, CQM_K_MACA_SLICE);
      k_maca_slice<<<n, 256, 0, S>>>(B, g, h->quad, h->s.p);
    }
    {
      ProfScope ps_(h, CQM_K_MACA_PIVOT);
      k_maca_pivot<<<n, 256, 0, S>>>(B);
    }
    {
      ProfScope ps_(h, CQM_K_MACA_FIBRE);
      k_maca_fibre<<<n, 256, 0, S>>>(B, g, h->quad, h->s.p);
    }
    {
      ProfScope ps_(h, CQM_K_MACA_FINALIZE);
      k_maca_finalize<<<n, 256, 0, S>>>(B);
    }
    if (cudaGetLastError() != cudaSuccess) {
      set_last_error("maca launch failed");
      release();
      return CQM_ECUDA;
    }
    if ((step & 3) == 3 || step == cap - 1) {
      cudaMemcpyAsync(hc, counters.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, S);
      if (cudaStreamSynchronize(S) != cudaSuccess) {
        set_last_error("maca failed");
        release();
        return CQM_ECUDA;
      }
      if (hc[0] == 0) break;
    }
  }
  {
    ProfScope ps_(h, CQM_K_MACA_FINALIZE);
    k_maca_mirror<<<n, 256, 0, S>>>(B, mirror.p);
  }
  cudaMemcpyAsync(hc, counters.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, S);
  cudaMemcpyAsync(h_rank.data(), rank.p, sizeof(int) * n, cudaMemcpyDeviceToHost, S);
  cudaError_t e = cudaStreamSynchronize(S);
  release();
  if (e != cudaSuccess) {
    set_last_error(std::string("maca: ") + cudaGetErrorString(e));
    return CQM_ECUDA;
  }
  if (hc[1] > 0) {
    set_last_error(std::to_string(hc[1]) + " blocks need more than rank_cap = " +
                   std::to_string(cap) + " MACA terms");
    return CQM_ECAPACITY;
  }
  return CQM_OK;
#undef MT
}

int build_maca(cqm_handle* h) {
  // near C slots: cap entries of #r x #c per block
  h->h_near_off.resize(h->n_near);
  int64_t total = 0;
  for (int b = 0; b < h->n_near; ++b) {
    h->h_near_off[b] = total;
    const int2 rc = h->h_near[b];
    total += (int64_t)h->rank_cap * (h->h_end[rc.x] - h->h_begin[rc.x]) * (h->h_end[rc.y] - h->h_begin[rc.y]);
  }
  CQM_TRY(h->near_off.allocate(h->alloc, std::max(1, h->n_near)));
  CQM_CUDA_TRY(cudaMemcpyAsync(h->near_off.p, h->h_near_off.data(), sizeof(int64_t) * h->n_near,
                               cudaMemcpyHostToDevice, h->stream));
  CQM_TRY(build_point_cache(h, total / std::max(1, h->rank_cap)));
  CQM_TRY(run_maca(h, 0, h->n_near, h->near_rc.p, h->nearC, h->nearD, h->near_rank, h->near_off.p,
                   (size_t)std::max<int64_t>(total, 1), h->h_near, h->h_near_rank));
  // the point cache serves the near-field slices and fibres only
  h->pt_r.free(h->alloc);
  h->pt_c.free(h->alloc);
  h->pt_off.free(h->alloc);
  h->pt_cnt.free(h->alloc);
  h->pt_r0.free(h->alloc);
  h->cache_far_points = false;
  if (h->params.maca_ff && h->params.cache_quadrature && h->n_far > 0) {
    const size_t n = (size_t)h->n_far * h->p * h->p;
    CQM_TRY(h->fpt_d.allocate(h->alloc, n));
    CQM_TRY(h->fpt_c.allocate(h->alloc, n));
    CQM_TRY(h->fpt_r0.allocate(h->alloc, h->n_far));
    {
      ProfScope ps_(h, CQM_K_POINTS);
      k_far_points<<<h->n_far, 256, 0, h->stream>>>(h->far_rc.p, h->cheb.p, h->m, h->p, h->fpt_d.p,
                                                    h->fpt_c.p, h->fpt_r0.p);
    }
    CQM_CHECK_LAUNCH();
    h->cache_far_points = true;
  }
  CQM_TRY(run_maca(h, 1, h->n_far, h->far_rc.p, h->farC, h->farD, h->far_rank, nullptr,
                   (size_t)h->n_far * h->rank_cap * h->p * h->p, h->h_far, h->h_far_rank));
  h->fpt_d.free(h->alloc);
  h->fpt_c.free(h->alloc);
  h->fpt_r0.free(h->alloc);
  h->cache_far_points = false;
  cqm_setup_info& I = h->info;
  I.near_entries = 0;
  I.near_rank_entries = 0;
  I.rank_sum_near = I.rank_sum_far = 0;
  I.rank_max = 0;
  for (int b = 0; b < h->n_near; ++b) {
    const int2 rc = h->h_near[b];
    I.near_entries += (int64_t)(h->h_end[rc.x] - h->h_begin[rc.x]) * (h->h_end[rc.y] - h->h_begin[rc.y]);
    I.rank_sum_near += h->h_near_rank[b];
    I.near_rank_entries += (int64_t)h->h_near_rank[b] * (h->h_end[rc.x] - h->h_begin[rc.x]) *
                           (h->h_end[rc.y] - h->h_begin[rc.y]);
    I.rank_max = std::max(I.rank_max, h->h_near_rank[b]);
  }
  for (int b = 0; b < h->n_far; ++b) {
    I.rank_sum_far += h->h_far_rank[b];
    I.rank_max = std::max(I.rank_max, h->h_far_rank[b]);
  }
  I.far_coupling = (int64_t)h->n_far * h->p * h->p;
  // kernel evaluations of the MACA of the upper blocks (the lower ones are mirrored)
  I.maca_slice_evals = I.maca_fibre_evals = 0;
  const bool have_pts = (int)h->h_block_points.size() == h->n_near;
  for (int b = 0; have_pts && b < h->n_near; ++b) {
    const int2 rc = h->h_near[b];
    if (rc.x > rc.y) continue;
    const int64_t nr = h->h_end[rc.x] - h->h_begin[rc.x], nc = h->h_end[rc.y] - h->h_begin[rc.y];
    const int64_t pairs = rc.x == rc.y ? nr * (nr + 1) / 2 : nr * nc;
    const int64_t pts = h->h_block_points[b], rk = h->h_near_rank[b];
    I.maca_slice_evals += rk * pts;
    if (pairs > 0) I.maca_fibre_evals += rk * h->Ls * pts / pairs;
  }
  for (int b = 0; b < h->n_far; ++b) {
    if (h->h_far[b].x > h->h_far[b].y) continue;
    I.maca_slice_evals += (int64_t)h->h_far_rank[b] * h->p * h->p;
    I.maca_fibre_evals += (int64_t)h->h_far_rank[b] * h->Ls;
  }
  return CQM_OK;
}

// Work items of the apply: every row's blocks split into consecutive runs of
// about equal work (rank, times #r #c for the near field), so that long rows
// do not serialise on one SM; about 4 items per SM in total.
int build_work_items(cqm_handle* h) {
  const int target = 4 * 152;
  auto split = [&](const std::vector<int>& rows, const std::vector<int2>& blk,
                   const std::vector<int>& rank, bool near, std::vector<int4>& items,
                   std::vector<int>& ptr) {
    std::vector<int> start(h->n_nodes + 1, 0);
    for (auto& b : blk) start[b.x + 1]++;
    for (int r = 0; r < h->n_nodes; ++r) start[r + 1] += start[r];
    auto weight = [&](int bi) -> double {
      const int2 rc = blk[bi];
      const double sz = near ? (double)(h->h_end[rc.x] - h->h_begin[rc.x]) * (h->h_end[rc.y] - h->h_begin[rc.y])
                             : 1.0;
      return std::max(1, rank[bi]) * sz;
    };
    double total = 0.0;
    for (size_t bi = 0; bi < blk.size(); ++bi) total += weight((int)bi);
    const double cap = std::max(1.0, total / target);
    ptr.assign(1, 0);
    for (int r : rows) {
      int b0 = start[r];
      double acc = 0.0;
      for (int bi = start[r]; bi < start[r + 1]; ++bi) {
        acc += weight(bi);
        if (acc >= cap || bi + 1 == start[r + 1]) {
          items.push_back(make_int4(r, b0, bi + 1, 0));
          b0 = bi + 1;
          acc = 0.0;
        }
      }
      if (start[r + 1] == start[r]) items.push_back(make_int4(r, start[r], start[r], 0));
      ptr.push_back((int)items.size());
    }
  };
  std::vector<int4> fi, ni;
  std::vector<int> fp, np;
  split(h->h_far_rows, h->h_far, h->h_far_rank, false, fi, fp);
  split(h->h_leaves, h->h_near, h->h_near_rank, true, ni, np);
  // launch order of the far items: decreasing rank sum (longest first), ties by index
  std::vector<int> forder(fi.size());
  std::vector<int64_t> fw(fi.size(), 0);
  for (size_t k = 0; k < fi.size(); ++k) {
    forder[k] = (int)k;
    for (int bi = fi[k].y; bi < fi[k].z; ++bi) fw[k] += std::max(1, h->h_far_rank[bi]);
  }
  std::stable_sort(forder.begin(), forder.end(), [&](int a, int b) { return fw[a] > fw[b]; });
  h->n_far_items = (int)fi.size();
  h->n_near_items = (int)ni.size();
  CQM_TRY(h->far_items.allocate(h->alloc, std::max<size_t>(1, fi.size())));
  CQM_TRY(h->near_items.allocate(h->alloc, std::max<size_t>(1, ni.size())));
  CQM_TRY(h->far_order.allocate(h->alloc, std::max<size_t>(1, forder.size())));
  CQM_TRY(h->far_item_ptr.allocate(h->alloc, fp.size()));
  CQM_TRY(h->near_item_ptr.allocate(h->alloc, np.size()));
  cudaStream_t S = h->stream;
  if (!fi.empty()) CQM_CUDA_TRY(cudaMemcpyAsync(h->far_items.p, fi.data(), sizeof(int4) * fi.size(), cudaMemcpyHostToDevice, S));
  if (!ni.empty()) CQM_CUDA_TRY(cudaMemcpyAsync(h->near_items.p, ni.data(), sizeof(int4) * ni.size(), cudaMemcpyHostToDevice, S));
  if (!forder.empty())
    CQM_CUDA_TRY(cudaMemcpyAsync(h->far_order.p, forder.data(), sizeof(int) * forder.size(), cudaMemcpyHostToDevice, S));
  CQM_CUDA_TRY(cudaMemcpyAsync(h->far_item_ptr.p, fp.data(), sizeof(int) * fp.size(), cudaMemcpyHostToDevice, S));
  CQM_CUDA_TRY(cudaMemcpyAsync(h->near_item_ptr.p, np.data(), sizeof(int) * np.size(), cudaMemcpyHostToDevice, S));
  const size_t part = std::max((size_t)h->n_far_items * 64, (size_t)h->n_near_items * 32) * h->Ls;
  CQM_TRY(h->part_d.allocate(h->alloc, std::max<size_t>(1, part)));
  CQM_TRY(h->part_f.allocate(h->alloc, std::max<size_t>(1, part)));
  CQM_CUDA_TRY(cudaStreamSynchronize(S));  // host vectors go out of scope
  return CQM_OK;
}

}  // namespace cqm
