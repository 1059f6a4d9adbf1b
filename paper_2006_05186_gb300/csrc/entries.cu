// Galerkin entries of the single layer at CQM frequencies (Sec. 3.2), the
// dense operator V_l (l < Ls) and its batched application.
#include <algorithm>
#include <cmath>
#include <vector>

#include "handle.cuh"

namespace cqm {

// Gauss-Legendre rule on [0, 1] with g points (Newton's method on the
// three-term recurrence of the Legendre polynomials), ascending nodes,
// weights summing to one.
static void gauss_legendre01(int g, std::vector<double>& x, std::vector<double>& w) {
  x.assign(g, 0.0);
  w.assign(g, 0.0);
  for (int k = 0; k < g; ++k) {
    double z = std::cos(M_PI * (k + 0.75) / (g + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int n = 2; n <= g; ++n) {
        double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      if (g == 1) { p0 = 1.0; p1 = z; }
      dp = g * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int n = 2; n <= g; ++n) {
        double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      dp = g * (z * p1 - p0) / (z * z - 1.0);
    }
    x[k] = 0.5 * (z + 1.0);
    w[k] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2/((1-z^2) P'^2) scaled by 1/2
  }
  std::vector<int> idx(g);
  for (int k = 0; k < g; ++k) idx[k] = k;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return x[a] < x[b]; });
  std::vector<double> xs(g), ws(g);
  for (int k = 0; k < g; ++k) { xs[k] = x[idx[k]]; ws[k] = w[idx[k]]; }
  x = xs;
  w = ws;
}

// Sauter-Schwab rules on T^ x T^ (weights sum to 1/4): for each Gauss tensor
// point (xi, e1, e2, e3) of [0,1]^4 and each region, the pair of reference
// points and the Jacobian-weighted weight.
static void sauter_schwab_rule(int cse, int g, std::vector<double4>& pts, std::vector<double>& wts) {
  std::vector<double> x, w;
  gauss_legendre01(g, x, w);
  pts.clear();
  wts.clear();
  const int nreg = (cse == CASE_IDENT) ? 6 : (cse == CASE_EDGE ? 5 : 2);
  for (int reg = 0; reg < nreg; ++reg) {
    for (int a = 0; a < g; ++a)
      for (int b = 0; b < g; ++b)
        for (int c = 0; c < g; ++c)
          for (int d = 0; d < g; ++d) {
            const double xi = x[a], e1 = x[b], e2 = x[c], e3 = x[d];
            const double W = w[a] * w[b] * w[c] * w[d];
            double x1, x2, y1, y2, J;
            if (cse == CASE_IDENT) {
              J = xi * xi * xi * e1 * e1 * e2;
              switch (reg) {
                case 0: x1 = xi; x2 = xi * (1 - e1 + e1 * e2); y1 = xi * (1 - e1 * e2 * e3); y2 = xi * (1 - e1); break;
                case 1: x1 = xi * (1 - e1 * e2 * e3); x2 = xi * (1 - e1); y1 = xi; y2 = xi * (1 - e1 + e1 * e2); break;
                case 2: x1 = xi; x2 = xi * e1 * (1 - e2 + e2 * e3); y1 = xi * (1 - e1 * e2); y2 = xi * e1 * (1 - e2); break;
                case 3: x1 = xi * (1 - e1 * e2); x2 = xi * e1 * (1 - e2); y1 = xi; y2 = xi * e1 * (1 - e2 + e2 * e3); break;
                case 4: x1 = xi * (1 - e1 * e2 * e3); x2 = xi * e1 * (1 - e2 * e3); y1 = xi; y2 = xi * e1 * (1 - e2); break;
                default: x1 = xi; x2 = xi * e1 * (1 - e2); y1 = xi * (1 - e1 * e2 * e3); y2 = xi * e1 * (1 - e2 * e3); break;
              }
            } else if (cse == CASE_EDGE) {
              J = xi * xi * xi * e1 * e1 * (reg == 0 ? 1.0 : e2);
              switch (reg) {
                case 0: x1 = xi; x2 = xi * e1 * e3; y1 = xi * (1 - e1 * e2); y2 = xi * e1 * (1 - e2); break;
                case 1: x1 = xi; x2 = xi * e1; y1 = xi * (1 - e1 * e2 * e3); y2 = xi * e1 * e2 * (1 - e3); break;
                case 2: x1 = xi * (1 - e1 * e2); x2 = xi * e1 * (1 - e2); y1 = xi; y2 = xi * e1 * e2 * e3; break;
                case 3: x1 = xi * (1 - e1 * e2 * e3); x2 = xi * e1 * e2 * (1 - e3); y1 = xi; y2 = xi * e1; break;
                default: x1 = xi * (1 - e1 * e2 * e3); x2 = xi * e1 * (1 - e2 * e3); y1 = xi; y2 = xi * e1 * e2; break;
              }
            } else {
              J = xi * xi * xi * e2;
              if (reg == 0) { x1 = xi; x2 = xi * e1; y1 = xi * e2; y2 = xi * e2 * e3; }
              else { x1 = xi * e2; x2 = xi * e2 * e3; y1 = xi; y2 = xi * e1; }
            }
            pts.push_back(make_double4(x1, x2, y1, y2));
            wts.push_back(W * J);
          }
  }
}

// Tables of the table-driven exponential: 2^(j/1024) and cis(j pi/512).
__global__ void k_exp_tables(double* t2, double2* cs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 1024) return;
  t2[j] = exp2((double)j / 1024.0);
  double sn, co;
  sincospi((double)j / 512.0, &sn, &co);
  cs[j] = make_double2(co, sn);
}

// Float-float copies of those tables: hi = the nearest float, lo = the rest.
__global__ void k_exp_tables_ff(const double* __restrict__ t2, const double2* __restrict__ cs,
                                float2* t2f, float4* csf) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 1024) return;
  const float a = (float)t2[j];
  t2f[j] = make_float2(a, (float)(t2[j] - (double)a));
  const float c = (float)cs[j].x, sn = (float)cs[j].y;
  csf[j] = make_float4(c, (float)(cs[j].x - (double)c), sn, (float)(cs[j].y - (double)sn));
}

int build_quad_tables(cqm_handle* h) {
  const int gn = h->params.g_near, gs = h->params.g_sing;
  std::vector<double> x, w;
  gauss_legendre01(gn, x, w);
  std::vector<double4> near;
  for (int a = 0; a < gn; ++a)
    for (int b = 0; b < gn; ++b) {
      double x1 = x[a], x2 = x[a] * x[b];
      near.push_back(make_double4(1.0 - x1, x1 - x2, x2, 2.0 * w[a] * w[b] * x[a]));
    }
  CQM_TRY(h->near_pt.allocate(h->alloc, near.size()));
  CQM_CUDA_TRY(cudaMemcpyAsync(h->near_pt.p, near.data(), near.size() * sizeof(double4),
                               cudaMemcpyHostToDevice, h->stream));
  h->quad.near_pt = h->near_pt.p;
  h->quad.n_near = gn * gn;
  for (int t = 0; t < 3; ++t) {
    std::vector<double4> pts;
    std::vector<double> wts;
    sauter_schwab_rule(CASE_VERT + t, gs, pts, wts);
    CQM_TRY(h->ss_pt[t].allocate(h->alloc, pts.size()));
    CQM_TRY(h->ss_w[t].allocate(h->alloc, wts.size()));
    CQM_CUDA_TRY(cudaMemcpyAsync(h->ss_pt[t].p, pts.data(), pts.size() * sizeof(double4),
                                 cudaMemcpyHostToDevice, h->stream));
    CQM_CUDA_TRY(cudaMemcpyAsync(h->ss_w[t].p, wts.data(), wts.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, h->stream));
    h->quad.ss_pt[t] = h->ss_pt[t].p;
    h->quad.ss_w[t] = h->ss_w[t].p;
    h->quad.ss_n[t] = (int)pts.size();
  }
  h->quad.near_ratio = h->params.near_ratio;
  CQM_TRY(h->exp_t2.allocate(h->alloc, 1024));
  CQM_TRY(h->exp_cs.allocate(h->alloc, 1024));
  k_exp_tables<<<4, 256, 0, h->stream>>>(h->exp_t2.p, h->exp_cs.p);
  CQM_CHECK_LAUNCH();
  CQM_TRY(h->exp_t2_ff.allocate(h->alloc, 1024));
  CQM_TRY(h->exp_cs_ff.allocate(h->alloc, 1024));
  k_exp_tables_ff<<<4, 256, 0, h->stream>>>(h->exp_t2.p, h->exp_cs.p, h->exp_t2_ff.p, h->exp_cs_ff.p);
  CQM_CHECK_LAUNCH();
  h->quad.t2 = h->exp_t2.p;
  h->quad.cs = h->exp_cs.p;
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));  // host vectors go out of scope
  return CQM_OK;
}

static Geom geom_of(const cqm_handle* h) {
  Geom g;
  g.M = h->M;
  g.tri = h->tri.p;
  g.P = h->P.p;
  g.area = h->area.p;
  g.cen = h->cen.p;
  g.diam = h->diam.p;
  return g;
}

constexpr int ENTRY_NF = 8;  // frequencies per warp pass

// One warp per (pair k, chunk of ENTRY_NF frequencies from the list `freq`).
__global__ void k_entries_list(Geom g, Quad q, int64_t npairs, const int* __restrict__ I,
                               const int* __restrict__ J, int nfreq, const int* __restrict__ freq,
                               const double2* __restrict__ s, double2* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int nchunk = (nfreq + ENTRY_NF - 1) / ENTRY_NF;
  const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= npairs * nchunk) return;
  const int64_t k = item / nchunk;
  const int f0 = (int)(item - k * nchunk) * ENTRY_NF;
  const int nf = min(ENTRY_NF, nfreq - f0);
  double2 sv[ENTRY_NF], acc[ENTRY_NF];
#pragma unroll
  for (int f = 0; f < ENTRY_NF; ++f) {
    sv[f] = (f < nf) ? s[freq[f0 + f]] : make_double2(0.0, 0.0);
    acc[f] = make_double2(0.0, 0.0);
  }
  const int i = I[k], j = J[k];
  const int cse = pair_case(g, q, i, j);
  pair_accumulate<ENTRY_NF>(g, q, i, j, cse, lane, 32, sv, nf, acc);
#pragma unroll
  for (int f = 0; f < ENTRY_NF; ++f) acc[f] = warp_sum2(acc[f]);
  if (lane == 0)
    for (int f = 0; f < nf; ++f) out[k * nfreq + f0 + f] = acc[f];
}

int entries_list(cqm_handle* h, int64_t npairs, const int* d_I, const int* d_J, int nfreq,
                 const int* d_freq, double2* d_out) {
  if (npairs == 0 || nfreq == 0) return CQM_OK;
  const int64_t items = npairs * ((nfreq + ENTRY_NF - 1) / ENTRY_NF);
  const int wpb = 8;
  {
    ProfScope ps_(h, CQM_K_ENTRIES);
    k_entries_list<<<(unsigned)((items + wpb - 1) / wpb), 32 * wpb, 0, h->stream>>>(
        geom_of(h), h->quad, npairs, d_I, d_J, nfreq, d_freq, h->s.p, d_out);
  }
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

// Dense V[l][i][j] for l < Ls: one warp per (i, j, frequency chunk).
__global__ void k_dense_assemble(Geom g, Quad q, int Ls, const double2* __restrict__ s,
                                 double2* __restrict__ V) {
  const int lane = threadIdx.x & 31;
  const int M = g.M;
  const int nchunk = (Ls + ENTRY_NF - 1) / ENTRY_NF;
  const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= (int64_t)M * M * nchunk) return;
  const int64_t k = item / nchunk;
  const int f0 = (int)(item - k * nchunk) * ENTRY_NF;
  const int nf = min(ENTRY_NF, Ls - f0);
  const int i = (int)(k / M), j = (int)(k - (int64_t)i * M);
  double2 sv[ENTRY_NF], acc[ENTRY_NF];
#pragma unroll
  for (int f = 0; f < ENTRY_NF; ++f) {
    sv[f] = (f < nf) ? s[f0 + f] : make_double2(0.0, 0.0);
    acc[f] = make_double2(0.0, 0.0);
  }
  const int cse = pair_case(g, q, i, j);
  pair_accumulate<ENTRY_NF>(g, q, i, j, cse, lane, 32, sv, nf, acc);
#pragma unroll
  for (int f = 0; f < ENTRY_NF; ++f) acc[f] = warp_sum2(acc[f]);
  if (lane == 0)
    for (int f = 0; f < nf; ++f) V[((size_t)(f0 + f) * M + i) * M + j] = acc[f];
}

int assemble_dense(cqm_handle* h) {
  const size_t n = (size_t)h->Ls * h->M * h->M;
  CQM_TRY(h->Vd.allocate(h->alloc, n));
  const int64_t items = (int64_t)h->M * h->M * ((h->Ls + ENTRY_NF - 1) / ENTRY_NF);
  const int wpb = 8;
  {
    ProfScope ps_(h, CQM_K_DENSE_ASSEMBLE);
    k_dense_assemble<<<(unsigned)((items + wpb - 1) / wpb), 32 * wpb, 0, h->stream>>>(
        geom_of(h), h->quad, h->Ls, h->s.p, h->Vd.p);
  }
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

// y_l = V_l x_l: one warp per row i of frequency l.
__global__ void k_dense_apply(int M, int Ls, const double2* __restrict__ V,
                              const double2* __restrict__ x, double2* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.y;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= M) return;
  const double2* row = V + ((size_t)l * M + i) * M;
  const double2* xl = x + (size_t)l * M;
  double2 acc = make_double2(0.0, 0.0);
  for (int j = lane; j < M; j += 32) cfma(acc, row[j], xl[j]);
  acc = warp_sum2(acc);
  if (lane == 0) y[(size_t)l * M + i] = acc;
}

int apply_dense(cqm_handle* h, const double2* x, double2* y) {
  const int wpb = 8;
  dim3 grid(grid_for(h->M, wpb), h->Ls);
  {
    ProfScope ps_(h, CQM_K_DENSE_APPLY);
    k_dense_apply<<<grid, 32 * wpb, 0, h->stream>>>(h->M, h->Ls, h->Vd.p, x, y);
  }
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

}  // namespace cqm
