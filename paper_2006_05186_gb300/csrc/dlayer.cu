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

#include "ffexp.cuh"
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

// Radius of the ball about the centroid that holds triangle t.
__device__ __forceinline__ double dl_tri_radius(const Geom& g, int t) {
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

// One quadrature point of pair (i, j) (test i, trial j): r = |x - y| and
// c = weight (x - y).n_j / (4 pi r^3); the pair's rule data prepared once.
struct DlPair {
  int cse, npts, nq;
  double aa;
  double X[9], Y[9];  // rule-ordered vertices (singular) or the triangles' own
  double n[3];
};
__device__ __forceinline__ void dl_pair_prepare(const Geom& g, const Quad& q, int i, int j, int cse, DlPair& P) {
  P.cse = cse;
  const double* Pi = g.P + 9 * i;
  const double* Pj = g.P + 9 * j;
  tri_normal(Pj, P.n);
  if (cse == CASE_REGULAR || cse == CASE_NEAR) {
    P.nq = (cse == CASE_REGULAR) ? 7 : q.n_near;
    P.npts = P.nq * P.nq;
    P.aa = g.area[i] * g.area[j];
    for (int k = 0; k < 9; ++k) {
      P.X[k] = Pi[k];
      P.Y[k] = Pj[k];
    }
    return;
  }
  P.nq = 0;
  P.npts = cse == CASE_IDENT ? 0 : q.ss_n[cse - CASE_VERT];
  P.aa = 4.0 * g.area[i] * g.area[j];
  int vx[3], vy[3];
  singular_vertices(g.tri, i, j, cse, vx, vy);
  for (int k = 0; k < 3; ++k) {
    const int tx = (vx[k] == g.tri[3 * i]) ? 0 : (vx[k] == g.tri[3 * i + 1] ? 1 : 2);
    const int ty = (vy[k] == g.tri[3 * j]) ? 0 : (vy[k] == g.tri[3 * j + 1] ? 1 : 2);
    for (int d = 0; d < 3; ++d) {
      P.X[3 * k + d] = Pi[3 * tx + d];
      P.Y[3 * k + d] = Pj[3 * ty + d];
    }
  }
}
__device__ __forceinline__ void dl_point(const Quad& q, const DlPair& P, int p, double& r, double& c) {
  double a0, a1, a2, b0, b1, b2, w;
  if (P.cse == CASE_REGULAR || P.cse == CASE_NEAR) {
    const int qa = p / P.nq, qb = p - qa * P.nq;
    double wa, wb;
    if (P.cse == CASE_REGULAR) {
      radon7(qa, a0, a1, a2, wa);
      radon7(qb, b0, b1, b2, wb);
    } else {
      const double4 A = q.near_pt[qa], B = q.near_pt[qb];
      a0 = A.x; a1 = A.y; a2 = A.z; wa = A.w;
      b0 = B.x; b1 = B.y; b2 = B.z; wb = B.w;
    }
    w = wa * wb * P.aa;
  } else {
    const int t = P.cse - CASE_VERT;
    const double4 z = q.ss_pt[t][p];
    a0 = 1.0 - z.x; a1 = z.x - z.y; a2 = z.y;
    b0 = 1.0 - z.z; b1 = z.z - z.w; b2 = z.w;
    w = q.ss_w[t][p] * P.aa;
  }
  const double* X = P.X;
  const double* Y = P.Y;
  const double d0 = (a0 * X[0] + a1 * X[3] + a2 * X[6]) - (b0 * Y[0] + b1 * Y[3] + b2 * Y[6]);
  const double d1 = (a0 * X[1] + a1 * X[4] + a2 * X[7]) - (b0 * Y[1] + b1 * Y[4] + b2 * Y[7]);
  const double d2 = (a0 * X[2] + a1 * X[5] + a2 * X[8]) - (b0 * Y[2] + b1 * Y[5] + b2 * Y[8]);
  r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  c = w * (d0 * P.n[0] + d1 * P.n[1] + d2 * P.n[2]) / (CQM_FOUR_PI * r * r * r);
}

// Near-field table of K: one CTA per near block, a warp per pair.  With r0 a
// lower bound of the pair's distances (0 for pairs sharing a vertex) and
// d = r - r0 >= 0,
//   K_l[i][j] = e^{-s_l r0} (A_l + s_l B_l),  A_l = sum c e^{-s_l d},  B_l = sum c r e^{-s_l d}.
// The lanes take the frequencies (lane + 32 u of a group of 32 UG); the pair's
// points come in batches of 32, whose geometry one lane each forms in FP64
// (d, c, c r as float-float pairs in shared memory), and every lane then sums
// e^{-s d} for its frequencies in float-float on the FP32 pipes (Tang's table
// method, ffexp.cuh).  The FP64 part (e^{-s r0}, the combination) runs once
// per pair and frequency with every lane busy.
__global__ void __launch_bounds__(256) k_dl_near_table(int Ls, Geom g, Quad q, const double2* __restrict__ s,
                                                       const int2* __restrict__ rc,
                                                       const int* __restrict__ begin,
                                                       const int* __restrict__ end,
                                                       const int* __restrict__ perm,
                                                       const int64_t* __restrict__ off,
                                                       const float2* __restrict__ t2ff,
                                                       const float4* __restrict__ csff,
                                                       double2* __restrict__ T) {
  constexpr int UG = 4;  // frequencies per lane and group
  __shared__ float2 t2s[1024];
  __shared__ float4 css[1024];
  __shared__ float2 pd[8][32], pc[8][32], pcr[8][32];
  for (int k = threadIdx.x; k < 1024; k += blockDim.x) {
    t2s[k] = t2ff[k];
    css[k] = csff[k];
  }
  __syncthreads();
  const int b = blockIdx.x;
  const int2 c2 = rc[b];
  const int rb = begin[c2.x], nr = end[c2.x] - rb, cb = begin[c2.y], nc = end[c2.y] - cb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double2* Tb = T + off[b];
  for (int e = w; e < nr * nc; e += nw) {
    const int i = e / nc, j = e - i * nc;
    const int I = perm[rb + i], J = perm[cb + j];
    const int cse = pair_case(g, q, I, J);
    DlPair P;
    dl_pair_prepare(g, q, I, J, cse, P);
    double r0 = 0.0;
    if (cse == CASE_REGULAR || cse == CASE_NEAR) {
      const double* ci = g.cen + 3 * I;
      const double* cj = g.cen + 3 * J;
      const double dx = ci[0] - cj[0], dy = ci[1] - cj[1], dz = ci[2] - cj[2];
      r0 = fmax(0.0, sqrt(dx * dx + dy * dy + dz * dz) * (1.0 - 1e-12) - dl_tri_radius(g, I) -
                         dl_tri_radius(g, J));
    }
    for (int fg = 0; fg < Ls; fg += 32 * UG) {
      ffs sf[UG];
      ff A[UG][2], B[UG][2];
#pragma unroll
      for (int u = 0; u < UG; ++u) {
        const int l = fg + lane + 32 * u;
        sf[u] = ffs_of(l < Ls ? s[l] : make_double2(0.0, 0.0));
        A[u][0] = A[u][1] = B[u][0] = B[u][1] = ff{0.f, 0.f};
      }
      int cnt = 0;
      for (int p0 = 0; p0 < P.npts; p0 += 32) {
        const int np = min(32, P.npts - p0);
        __syncwarp();
        if (lane < np) {
          double r, c;
          dl_point(q, P, p0 + lane, r, c);
          const ff dd = ff_of(fmax(r - r0, 0.0)), cc = ff_of(c), cr = ff_of(c * r);
          pd[w][lane] = make_float2(dd.h, dd.l);
          pc[w][lane] = make_float2(cc.h, cc.l);
          pcr[w][lane] = make_float2(cr.h, cr.l);
        }
        __syncwarp();
        for (int k = 0; k < np; ++k) {
          const float2 dk = pd[w][k], ck = pc[w][k], crk = pcr[w][k];
          const ff cf = {ck.x, ck.y}, crf = {crk.x, crk.y};
#pragma unroll
          for (int u = 0; u < UG; ++u) {
            ff er, ei;  // e^{-s d}
            cexp_ff(ff{dk.x, dk.y}, ff{1.f, 0.f}, sf[u], t2s, css, er, ei);
            ff_acc(A[u][0], ff_mul(cf, er));
            ff_acc(A[u][1], ff_mul(cf, ei));
            ff_acc(B[u][0], ff_mul(crf, er));
            ff_acc(B[u][1], ff_mul(crf, ei));
          }
          if ((++cnt & 15) == 0) {
#pragma unroll
            for (int u = 0; u < UG; ++u) {
              ff_norm(A[u][0]);
              ff_norm(A[u][1]);
              ff_norm(B[u][0]);
              ff_norm(B[u][1]);
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < UG; ++u) {
        const int l = fg + lane + 32 * u;
        if (l < Ls) {
          const double2 sl = s[l];
          const double2 a = make_double2(ff_to_double(A[u][0]), ff_to_double(A[u][1]));
          const double2 bb = make_double2(ff_to_double(B[u][0]), ff_to_double(B[u][1]));
          const double2 v = cadd(a, cmul(sl, bb));
          Tb[((size_t)l * nc + j) * nr + i] = cmul(v, cexp_c(r0, 1.0, sl, q));
        }
      }
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
                                                   h->dl_off.p, h->exp_t2_ff.p, h->exp_cs_ff.p,
                                                   h->dl_table.p);
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
