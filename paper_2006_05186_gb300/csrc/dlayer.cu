// The double layer of the Laplace-domain kernel and the direct formulation of
// the sound-soft (Dirichlet) problem (Sec. 2.2, eq. wavebio; Sec. 7.2,
// eq. cqmdir), decoupled in frequency as in the Remark of Sec. 6.2:
//
//   V_l qhat_l = (-1/2 M + K_l) ghat_l,   M = diag |tau_i|,
//   K_l[i][j] = int_{tau_i} int_{tau_j} (x - y).n_j (1 + s_l r) e^{-s_l r} / (4 pi r^3),
//
// P0 test and trial functions, n_j the outward unit normal of tau_j.
// The near field of K is evaluated once per frequency into a table with the
// layout of the expanded single-layer near field (block b, frequency l, entry
// (i, j) at off[b] + (l #c + j) #r + i), by the single layer's quadrature
// rules without the canonical swap (the kernel is not symmetric); on a flat
// triangle (x - y).n_j vanishes, so identical pairs are 0.  The far field
// interpolates the kernel in x and y and differentiates the y-interpolant
// (Sec. 4 and the remark after Thm. 1): K_l|_b = U_r S_b(s_l) W_c^T with the
// single layer's compressed couplings S_b (eq. lrfinal) and the column basis
// W_c[j][nu] = int_{tau_j} n_j . grad L_{c,nu}, nested with the same transfer
// matrices (grad L_{c,nu} = sum_lambda E[lambda][nu] grad L_{c',lambda}), so
// only the leaf basis differs.  All FP64 (the far couplings as the handle's
// FP64-accurate apply holds them).
#include <algorithm>
#include <vector>

#include "handle.cuh"

namespace cqm {

// Outward unit normal of triangle t from its vertices (counter-clockwise).
__device__ __forceinline__ void tri_normal(const double* P, double* n) {
  const double a0 = P[3] - P[0], a1 = P[4] - P[1], a2 = P[5] - P[2];
  const double b0 = P[6] - P[0], b1 = P[7] - P[1], b2 = P[8] - P[2];
  const double c0 = a1 * b2 - a2 * b1, c1 = a2 * b0 - a0 * b2, c2 = a0 * b1 - a1 * b0;
  const double inv = 1.0 / sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  n[0] = c0 * inv;
  n[1] = c1 * inv;
  n[2] = c2 * inv;
}

// Visit this lane's share of the quadrature points of pair (i, j) (test i,
// trial j; no swap): f(r, c) with c = weight (x - y).n_j / (4 pi r^3).  Rules
// and singular vertex orders as for the single layer; identical pairs have no
// points (the integrand vanishes on a flat triangle).
template <class F>
__device__ __forceinline__ void dl_pair_points(const Geom& g, const Quad& q, int i, int j, int cse,
                                               int lane, int nlanes, F&& f) {
  if (cse == CASE_IDENT) return;
  const double* Pi = g.P + 9 * i;
  const double* Pj = g.P + 9 * j;
  double nj[3];
  tri_normal(Pj, nj);
  if (cse == CASE_REGULAR || cse == CASE_NEAR) {
    const int nq = (cse == CASE_REGULAR) ? 7 : q.n_near;
    const double aa = g.area[i] * g.area[j];
    for (int p = lane; p < nq * nq; p += nlanes) {
      const int qa = p / nq, qb = p - qa * nq;
      double a0, a1, a2, wa, b0, b1, b2, wb;
      if (cse == CASE_REGULAR) {
        radon7(qa, a0, a1, a2, wa);
        radon7(qb, b0, b1, b2, wb);
      } else {
        const double4 A = q.near_pt[qa], B = q.near_pt[qb];
        a0 = A.x; a1 = A.y; a2 = A.z; wa = A.w;
        b0 = B.x; b1 = B.y; b2 = B.z; wb = B.w;
      }
      const double d0 = (a0 * Pi[0] + a1 * Pi[3] + a2 * Pi[6]) - (b0 * Pj[0] + b1 * Pj[3] + b2 * Pj[6]);
      const double d1 = (a0 * Pi[1] + a1 * Pi[4] + a2 * Pi[7]) - (b0 * Pj[1] + b1 * Pj[4] + b2 * Pj[7]);
      const double d2 = (a0 * Pi[2] + a1 * Pi[5] + a2 * Pi[8]) - (b0 * Pj[2] + b1 * Pj[5] + b2 * Pj[8]);
      const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      f(r, (wa * wb * aa) * (d0 * nj[0] + d1 * nj[1] + d2 * nj[2]) / (CQM_FOUR_PI * r * r * r));
    }
    return;
  }
  int vx[3], vy[3];
  singular_vertices(g.tri, i, j, cse, vx, vy);
  double X[9], Y[9];
  for (int k = 0; k < 3; ++k) {
    const int tx = (vx[k] == g.tri[3 * i]) ? 0 : (vx[k] == g.tri[3 * i + 1] ? 1 : 2);
    const int ty = (vy[k] == g.tri[3 * j]) ? 0 : (vy[k] == g.tri[3 * j + 1] ? 1 : 2);
    for (int d = 0; d < 3; ++d) {
      X[3 * k + d] = Pi[3 * tx + d];
      Y[3 * k + d] = Pj[3 * ty + d];
    }
  }
  const int t = cse - CASE_VERT;
  const double4* pt = q.ss_pt[t];
  const double* wt = q.ss_w[t];
  const int n = q.ss_n[t];
  const double aa = 4.0 * g.area[i] * g.area[j];
  for (int p = lane; p < n; p += nlanes) {
    const double4 z = pt[p];
    const double a0 = 1.0 - z.x, a1 = z.x - z.y, a2 = z.y;
    const double b0 = 1.0 - z.z, b1 = z.z - z.w, b2 = z.w;
    const double d0 = (a0 * X[0] + a1 * X[3] + a2 * X[6]) - (b0 * Y[0] + b1 * Y[3] + b2 * Y[6]);
    const double d1 = (a0 * X[1] + a1 * X[4] + a2 * X[7]) - (b0 * Y[1] + b1 * Y[4] + b2 * Y[7]);
    const double d2 = (a0 * X[2] + a1 * X[5] + a2 * X[8]) - (b0 * Y[2] + b1 * Y[5] + b2 * Y[8]);
    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    f(r, (wt[p] * aa) * (d0 * nj[0] + d1 * nj[1] + d2 * nj[2]) / (CQM_FOUR_PI * r * r * r));
  }
}

// Near-field table of K: one CTA per near block, a warp per pair, the lanes
// over the pair's points, NF frequencies per pass (lane f of the warp writes
// frequency f of the pass).
__global__ void __launch_bounds__(256) k_dl_near_table(int Ls, Geom g, Quad q, const double2* __restrict__ s,
                                                       const int2* __restrict__ rc,
                                                       const int* __restrict__ begin,
                                                       const int* __restrict__ end,
                                                       const int* __restrict__ perm,
                                                       const int64_t* __restrict__ off,
                                                       double2* __restrict__ T) {
  constexpr int NF = 8;
  const int b = blockIdx.x;
  const int2 c2 = rc[b];
  const int rb = begin[c2.x], nr = end[c2.x] - rb, cb = begin[c2.y], nc = end[c2.y] - cb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double2* Tb = T + off[b];
  for (int e = w; e < nr * nc; e += nw) {
    const int i = e / nc, j = e - i * nc;
    const int I = perm[rb + i], J = perm[cb + j];
    const int cse = pair_case(g, q, I, J);
    for (int f0 = 0; f0 < Ls; f0 += NF) {
      const int nf = min(NF, Ls - f0);
      double2 sv[NF], acc[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        sv[f] = f < nf ? s[f0 + f] : make_double2(0.0, 0.0);
        acc[f] = make_double2(0.0, 0.0);
      }
      dl_pair_points(g, q, I, J, cse, lane, 32, [&](double r, double c) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          if (f < nf) {
            // c (1 + s r) e^{-s r}
            const double2 v = cexp_c(r, c, sv[f], q);
            const double2 o = make_double2(1.0 + sv[f].x * r, sv[f].y * r);
            const double2 t = cmul(v, o);
            acc[f].x += t.x;
            acc[f].y += t.y;
          }
        }
      });
#pragma unroll
      for (int f = 0; f < NF; ++f) acc[f] = warp_sum2(acc[f]);
#pragma unroll
      for (int f = 0; f < NF; ++f)
        if (lane == f && f < nf) Tb[((size_t)(f0 + f) * nc + j) * nr + i] = acc[f];
    }
  }
}

// l_k'(x) on the m nodes of one axis
__device__ __forceinline__ double lagrange1_deriv(const double* nodes, int m, int k, double x) {
  double sum = 0.0;
  for (int i = 0; i < m; ++i) {
    if (i == k) continue;
    double v = 1.0 / (nodes[k] - nodes[i]);
    for (int j = 0; j < m; ++j)
      if (j != k && j != i) v *= (x - nodes[j]) / (nodes[k] - nodes[j]);
    sum += v;
  }
  return sum;
}
__device__ __forceinline__ double lagrange1_v(const double* nodes, int m, int k, double x) {
  double v = 1.0;
  for (int j = 0; j < m; ++j)
    if (j != k) v *= (x - nodes[j]) / (nodes[k] - nodes[j]);
  return v;
}

// Double-layer leaf basis: W[pos][nu] = |tau| sum_q w_q n . grad L_{r,nu}(x_q)
// for the triangle at position pos of leaf r (Radon rule).
__global__ void k_dl_leaf_basis(int M, int m, int p, const int* __restrict__ leaf_of,
                                const int* __restrict__ perm, const double* __restrict__ P,
                                const double* __restrict__ area, const double* __restrict__ cheb,
                                double* W) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M * p) return;
  const int pos = t / p, nu = t - pos * p;
  const int r = leaf_of[pos];
  const int tri = perm[pos];
  const double* v = P + 9 * tri;
  double n[3];
  tri_normal(v, n);
  const double* nd = cheb + (size_t)r * 3 * m;
  const int ix = nu % m, iy = (nu / m) % m, iz = nu / (m * m);
  double acc = 0.0;
  for (int q = 0; q < 7; ++q) {
    double l0, l1, l2, wq;
    radon7(q, l0, l1, l2, wq);
    const double x = l0 * v[0] + l1 * v[3] + l2 * v[6];
    const double y = l0 * v[1] + l1 * v[4] + l2 * v[7];
    const double z = l0 * v[2] + l1 * v[5] + l2 * v[8];
    const double lx = lagrange1_v(nd, m, ix, x), ly = lagrange1_v(nd + m, m, iy, y),
                 lz = lagrange1_v(nd + 2 * m, m, iz, z);
    const double dx = lagrange1_deriv(nd, m, ix, x), dy = lagrange1_deriv(nd + m, m, iy, y),
                 dz = lagrange1_deriv(nd + 2 * m, m, iz, z);
    acc += wq * (n[0] * dx * ly * lz + n[1] * lx * dy * lz + n[2] * lx * ly * dz);
  }
  W[t] = area[tri] * acc;
}

__global__ void k_dl_leaf_of(const int* __restrict__ son0, const int* __restrict__ begin,
                             const int* __restrict__ end, int* __restrict__ leaf_of) {
  const int r = blockIdx.x;
  if (son0[r] >= 0) return;
  for (int pos = begin[r] + threadIdx.x; pos < end[r]; pos += blockDim.x) leaf_of[pos] = r;
}

// rhs_l[i] += -1/2 |tau_i| ghat_l[i]
__global__ void k_dl_mass(int64_t n, int M, const double* __restrict__ area, const double2* __restrict__ g,
                          double2* __restrict__ rhs) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double a = -0.5 * area[e % M];
  rhs[e] = make_double2(fma(a, g[e].x, rhs[e].x), fma(a, g[e].y, rhs[e].y));
}

// ---- host --------------------------------------------------------------

static Geom geom_of(const cqm_handle* h) {
  Geom g;
  g.M = h->M; g.tri = h->tri.p; g.P = h->P.p; g.area = h->area.p; g.cen = h->cen.p; g.diam = h->diam.p;
  return g;
}

void dl_release(cqm_handle* h) {
  h->dl_table.free(h->alloc);
  h->dl_off.free(h->alloc);
  h->dl_W.free(h->alloc);
  h->dl_ready = false;
}

// Near-field table of K at the solved frequencies and the leaf column basis W.
static int dl_prepare(cqm_handle* h) {
  if (h->dl_ready) return CQM_OK;
  if (h->params.mode != CQM_MODE_H2MACA) {
    set_last_error("the double layer needs the H2MACA mode");
    return CQM_EINVAL;
  }
  Allocator& A = h->alloc;
  const int nb = h->n_near, M = h->M, p = h->p;
  std::vector<int64_t> off(nb + 1, 0);
  for (int b = 0; b < nb; ++b) {
    const int2 rc = h->h_near[b];
    off[b + 1] = off[b] + (int64_t)h->Ls * (h->h_end[rc.x] - h->h_begin[rc.x]) * (h->h_end[rc.y] - h->h_begin[rc.y]);
  }
  int st = CQM_OK;
  DArray<int> leaf_of;
  do {
    if ((st = h->dl_off.allocate(A, nb + 1)) != CQM_OK) break;
    if ((st = h->dl_table.allocate(A, (size_t)std::max<int64_t>(1, off[nb]))) != CQM_OK) break;
    if ((st = h->dl_W.allocate(A, (size_t)M * p)) != CQM_OK) break;
    if ((st = leaf_of.allocate(A, M)) != CQM_OK) break;
    if (cudaMemcpyAsync(h->dl_off.p, off.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess) {
      st = CQM_ECUDA;
      break;
    }
    {
      ProfScope ps_(h, CQM_K_DL_SETUP);
      if (nb > 0)
        k_dl_near_table<<<nb, 256, 0, h->stream>>>(h->Ls, geom_of(h), h->quad, h->s.p, h->near_rc.p,
                                                   h->node_begin.p, h->node_end.p, h->perm.p,
                                                   h->dl_off.p, h->dl_table.p);
      k_dl_leaf_of<<<h->n_nodes, 128, 0, h->stream>>>(h->node_son0.p, h->node_begin.p, h->node_end.p,
                                                       leaf_of.p);
      k_dl_leaf_basis<<<grid_for((int64_t)M * p, 256), 256, 0, h->stream>>>(
          M, h->m, p, leaf_of.p, h->perm.p, h->P.p, h->area.p, h->cheb.p, h->dl_W.p);
    }
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) {
      set_last_error("double layer: setup kernels failed");
      st = CQM_ECUDA;
    }
  } while (false);
  leaf_of.free(A);
  if (st != CQM_OK) {
    dl_release(h);
    return st;
  }
  h->dl_ready = true;
  return CQM_OK;
}

int dl_apply(cqm_handle* h, const double2* x, double2* y) {
  CQM_TRY(dl_prepare(h));
  {
    ProfScope ps_(h, CQM_K_DL_APPLY);
    CQM_TRY(near_apply_table(h, h->dl_table.p, h->dl_off.p, x, y));
  }
  if (h->n_far > 0) CQM_TRY(apply_far_columns(h, h->dl_W.p, x, y));
  return CQM_OK;
}

// Neumann data q (L x M) of the Dirichlet problem with P0 data coefficients
// g (L x M), both device: forward transform, right-hand sides
// (-1/2 M + K_l) ghat_l, the batched GMRES of the single layer, inverse
// transform.
int dl_solve(cqm_handle* h, const double* d_g, double* d_q, cqm_solve_info* info) {
  CQM_TRY(dl_prepare(h));
  Allocator& A = h->alloc;
  const size_t nf = (size_t)h->Ls * h->M;
  DArray<double2> gh, rhs, qh;
  int st = CQM_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  do {
    if ((st = gh.allocate(A, nf)) != CQM_OK) break;
    if ((st = rhs.allocate(A, nf)) != CQM_OK) break;
    if ((st = qh.allocate(A, nf)) != CQM_OK) break;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaEventCreate(&e2) != cudaSuccess) {
      set_last_error("cudaEventCreate failed");
      st = CQM_ECUDA;
      break;
    }
    cudaEventRecord(e0, h->stream);
    if ((st = forward_transform(h, d_g, gh.p)) != CQM_OK) break;
    if ((st = dl_apply(h, gh.p, rhs.p)) != CQM_OK) break;
    k_dl_mass<<<grid_for((int64_t)nf, 256), 256, 0, h->stream>>>((int64_t)nf, h->M, h->area.p, gh.p, rhs.p);
    if (cudaGetLastError() != cudaSuccess) {
      st = CQM_ECUDA;
      break;
    }
    cudaEventRecord(e1, h->stream);
    st = gmres_solve(h, rhs.p, qh.p, info);
    if (st != CQM_OK && st != CQM_ENOCONV) break;
    const int gst = st;
    cudaEventRecord(e2, h->stream);
    if ((st = inverse_transform(h, qh.p, d_q)) != CQM_OK) break;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
      set_last_error("double layer: solve failed");
      st = CQM_ECUDA;
      break;
    }
    if (info) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      info->t_forward_ms = ms;  // transform and right-hand sides
    }
    st = gst;
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e2) cudaEventDestroy(e2);
  gh.free(A);
  rhs.free(A);
  qh.free(A);
  return st;
}

}  // namespace cqm
