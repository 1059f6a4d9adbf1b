// Galerkin matrices with piecewise linear functions for mixed boundary
// conditions (Sec. 2.3 eq. wavegalform; Sec. 3.2, the matrices K_l, K'_l, D_l
// of P0 and P1 spaces), at the solved frequencies, dense:
//
//   K1[l][m][v] = <phi0_m, K phi1_v>,  kernel dG/dn_y = (x - y).n_y (1 + s r) e^{-sr} / (4 pi r^3),
//   Kp[l][v][i] = <phi1_v, K' phi0_i>, kernel dG/dn_x = (y - x).n_x (1 + s r) e^{-sr} / (4 pi r^3),
//   D[l][u][v]  = int int G(r) [curl phi1_u . curl phi1_v + s^2 (n_x.n_y) phi1_u phi1_v]
//                 (Maue's form of the hypersingular operator, G = e^{-sr} / (4 pi r)),
//
// phi0 the triangle indicators, phi1 the vertex hats (on triangle t the hat of
// its vertex a is the barycentric coordinate lambda_a, whose surface curl
// n x grad lambda_a is the opposite edge (P_{a+1} - P_{a+2}) / (2 |t|)).  The
// quadrature is the single layer's rule set (quad.cuh) with the test triangle
// first and no symmetrisation; for the Sauter-Schwab pairs the rule's
// barycentric coordinates, which refer to the reordered vertices, are mapped
// back to each triangle's stored vertices.  Identical flat triangles
// contribute nothing to K1 and Kp ((x - y).n = 0).
//
// One CTA per test triangle i, its warps over the trial triangles j, lanes
// over the pair's points; per pair and frequency the warp sums the 16 local
// values (3 of K1, 3 of Kp, the kernel integral and its 9 hat moments for D)
// and adds them into the dense matrices with FP64 atomics (several pairs
// share a row of K1, a column of Kp and the entries of D).  FP64 throughout.
#include "handle.cuh"
#include "quad.cuh"

namespace cqm {

namespace {

// This lane's quadrature points of the pair (test i, trial j): f(X, Y, lx,
// ly, w) with X on i, Y on j, their barycentric coordinates in each
// triangle's stored vertex order and the weight (area factors included).
template <class F>
__device__ void p1_pair_points(const Geom& g, const Quad& q, int i, int j, int cse, int lane, int nl, F&& f) {
  const double* Pi = g.P + 9 * i;
  const double* Pj = g.P + 9 * j;
  if (cse == CASE_REGULAR || cse == CASE_NEAR) {
    const int nq = cse == CASE_REGULAR ? 7 : q.n_near;
    const double aa = g.area[i] * g.area[j];
    for (int p = lane; p < nq * nq; p += nl) {
      const int qa = p / nq, qb = p - qa * nq;
      double la[3], lb[3], wa, wb;
      if (cse == CASE_REGULAR) {
        radon7(qa, la[0], la[1], la[2], wa);
        radon7(qb, lb[0], lb[1], lb[2], wb);
      } else {
        const double4 A = q.near_pt[qa], B = q.near_pt[qb];
        la[0] = A.x; la[1] = A.y; la[2] = A.z; wa = A.w;
        lb[0] = B.x; lb[1] = B.y; lb[2] = B.z; wb = B.w;
      }
      double X[3], Y[3];
      for (int d = 0; d < 3; ++d) {
        X[d] = la[0] * Pi[d] + la[1] * Pi[3 + d] + la[2] * Pi[6 + d];
        Y[d] = lb[0] * Pj[d] + lb[1] * Pj[3 + d] + lb[2] * Pj[6 + d];
      }
      f(X, Y, la, lb, wa * wb * aa);
    }
    return;
  }
  int vx[3], vy[3];
  singular_vertices(g.tri, i, j, cse, vx, vy);
  // rule position of each stored vertex, and the rule's vertices in space
  int px[3] = {0, 0, 0}, py[3] = {0, 0, 0};
  double XV[9], YV[9];
  for (int k = 0; k < 3; ++k) {
    for (int a = 0; a < 3; ++a) {
      if (vx[k] == g.tri[3 * i + a]) {
        px[a] = k;
        for (int d = 0; d < 3; ++d) XV[3 * k + d] = Pi[3 * a + d];
      }
      if (vy[k] == g.tri[3 * j + a]) {
        py[a] = k;
        for (int d = 0; d < 3; ++d) YV[3 * k + d] = Pj[3 * a + d];
      }
    }
  }
  const int t = cse - CASE_VERT;
  const double4* pt = q.ss_pt[t];
  const double* wt = q.ss_w[t];
  const int n = q.ss_n[t];
  const double aa = 4.0 * g.area[i] * g.area[j];
  for (int p = lane; p < n; p += nl) {
    const double4 z = pt[p];
    const double a[3] = {1.0 - z.x, z.x - z.y, z.y};
    const double b[3] = {1.0 - z.z, z.z - z.w, z.w};
    double X[3], Y[3];
    for (int d = 0; d < 3; ++d) {
      X[d] = a[0] * XV[d] + a[1] * XV[3 + d] + a[2] * XV[6 + d];
      Y[d] = b[0] * YV[d] + b[1] * YV[3 + d] + b[2] * YV[6 + d];
    }
    const double la[3] = {a[px[0]], a[px[1]], a[px[2]]};
    const double lb[3] = {b[py[0]], b[py[1]], b[py[2]]};
    f(X, Y, la, lb, wt[p] * aa);
  }
}

__device__ __forceinline__ void tri_normal(const double* P, double n[3]) {
  const double e1[3] = {P[3] - P[0], P[4] - P[1], P[5] - P[2]};
  const double e2[3] = {P[6] - P[0], P[7] - P[1], P[8] - P[2]};
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  const double s = 1.0 / sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  n[0] *= s; n[1] *= s; n[2] *= s;
}

// curl of the hat of stored vertex a of a triangle: (P_{a+1} - P_{a+2}) / (2 |t|)
__device__ __forceinline__ void hat_curl(const double* P, double area, int a, double c[3]) {
  const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
  for (int d = 0; d < 3; ++d) c[d] = (P[3 * a1 + d] - P[3 * a2 + d]) / (2.0 * area);
}

__device__ __forceinline__ void atomic_cadd(double2* p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

constexpr int NV16 = 16;  // local values per pair and frequency

__global__ void __launch_bounds__(256) k_p1_matrices(Geom g, Quad q, int nv, int Ls, const double2* __restrict__ s,
                                                     double2* __restrict__ K1, double2* __restrict__ Kp,
                                                     double2* __restrict__ D) {
  const int i = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int M = g.M;
  double ni[3];
  tri_normal(g.P + 9 * i, ni);
  for (int j = w; j < M; j += nw) {
    const int cse = pair_case(g, q, i, j);
    double nj[3];
    tri_normal(g.P + 9 * j, nj);
    const double nn = ni[0] * nj[0] + ni[1] * nj[1] + ni[2] * nj[2];
    const bool ident = cse == CASE_IDENT;
    for (int l = 0; l < Ls; ++l) {
      const double2 sl = s[l];
      // [0..2] K1 (trial hats of j), [3..5] Kp (test hats of i), [6] int int G,
      // [7..15] int int G lx_a ly_b
      double2 acc[NV16];
#pragma unroll
      for (int k = 0; k < NV16; ++k) acc[k] = make_double2(0.0, 0.0);
      p1_pair_points(g, q, i, j, cse, lane, 32, [&](const double* X, const double* Y, const double* lx,
                                                    const double* ly, double wgt) {
        const double d0 = X[0] - Y[0], d1 = X[1] - Y[1], d2 = X[2] - Y[2];
        const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        const double2 gv = cexp_c(r, wgt / (CQM_FOUR_PI * r), sl, q);  // w G(r)
        // w (1 + s r) e^{-sr} / (4 pi r^3) = w G(r) (1 + s r) / r^2
        const double2 hv = cmul(gv, make_double2((1.0 + sl.x * r) / (r * r), sl.y * r / (r * r)));
        if (!ident) {
          const double dny = d0 * nj[0] + d1 * nj[1] + d2 * nj[2];     // (x - y).n_y
          const double dnx = -(d0 * ni[0] + d1 * ni[1] + d2 * ni[2]);  // (y - x).n_x
          for (int b = 0; b < 3; ++b) {
            acc[b].x += hv.x * dny * ly[b];
            acc[b].y += hv.y * dny * ly[b];
            acc[3 + b].x += hv.x * dnx * lx[b];
            acc[3 + b].y += hv.y * dnx * lx[b];
          }
        }
        acc[6].x += gv.x;
        acc[6].y += gv.y;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            const double m = lx[a] * ly[b];
            acc[7 + 3 * a + b].x += gv.x * m;
            acc[7 + 3 * a + b].y += gv.y * m;
          }
      });
#pragma unroll
      for (int k = 0; k < NV16; ++k) {
        acc[k].x = warp_sum(acc[k].x);
        acc[k].y = warp_sum(acc[k].y);
      }
      if (lane < 3) {  // K1[l][i][v_b], Kp[l][u_a][j] with a = b = lane
        const int b = lane;
        atomic_cadd(K1 + ((size_t)l * M + i) * nv + g.tri[3 * j + b], acc[b]);
        atomic_cadd(Kp + ((size_t)l * nv + g.tri[3 * i + b]) * M + j, acc[3 + b]);
      } else if (lane < 12) {  // D[l][u_a][v_b]
        const int a = (lane - 3) / 3, b = (lane - 3) - 3 * a;
        double ca[3], cb[3];
        hat_curl(g.P + 9 * i, g.area[i], a, ca);
        hat_curl(g.P + 9 * j, g.area[j], b, cb);
        const double cc = ca[0] * cb[0] + ca[1] * cb[1] + ca[2] * cb[2];
        const double2 s2 = cmul(sl, sl);
        // the registers of acc are the same in every lane after the sums
        double2 gl = acc[7];
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (k == 3 * a + b) gl = acc[7 + k];
        const double2 v = cadd(make_double2(acc[6].x * cc, acc[6].y * cc), cmul(make_double2(s2.x * nn, s2.y * nn), gl));
        atomic_cadd(D + ((size_t)l * nv + g.tri[3 * i + a]) * nv + g.tri[3 * j + b], v);
      }
    }
  }
}

}  // namespace

// Dense K1 (Ls x M x nv), Kp (Ls x nv x M) and D (Ls x nv x nv), complex, on
// the device; zeroed here, then summed by the kernel.
int p1_matrices(cqm_handle* h, double2* K1, double2* Kp, double2* D) {
  const size_t M = (size_t)h->M, nv = (size_t)h->nv, Ls = (size_t)h->Ls;
  CQM_CUDA_TRY(cudaMemsetAsync(K1, 0, sizeof(double2) * Ls * M * nv, h->stream));
  CQM_CUDA_TRY(cudaMemsetAsync(Kp, 0, sizeof(double2) * Ls * nv * M, h->stream));
  CQM_CUDA_TRY(cudaMemsetAsync(D, 0, sizeof(double2) * Ls * nv * nv, h->stream));
  Geom g;
  g.M = h->M; g.tri = h->tri.p; g.P = h->P.p; g.area = h->area.p; g.cen = h->cen.p; g.diam = h->diam.p;
  k_p1_matrices<<<h->M, 256, 0, h->stream>>>(g, h->quad, h->nv, h->Ls, h->s.p, K1, Kp, D);
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

}  // namespace cqm
