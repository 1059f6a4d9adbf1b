// Element geometry and quadrature of the P0 Galerkin single layer
// V_l[i,j] = int_{tau_i} int_{tau_j} exp(-s_l |x-y|) / (4 pi |x-y|)  (Sec. 3.2,
// eq. fundsol).  The paper leaves the quadrature open; the rule set is:
//   * pairs sharing 3 / 2 / 1 vertex index: Sauter-Schwab relative-coordinate
//     rules (identical: 6 regions, common edge: 5, common vertex: 2), each a
//     g^4 Gauss-Legendre tensor rule on [0,1]^4 (Sauter & Schwab, Boundary
//     Element Methods, Sec. 5.2);
//   * disjoint pairs whose centroid distance is below near_ratio times the
//     larger longest edge: a collapsed (Duffy) g x g Gauss rule per triangle;
//   * all other pairs: Radon's degree-5 seven-point rule per triangle.
// Reference triangle {0 <= x2 <= x1 <= 1}, chi(x^) = P0 + x1 (P1-P0) + x2 (P2-P1),
// barycentric coordinates (1 - x1, x1 - x2, x2).
#pragma once

#include "common.cuh"

namespace cqm {

// 4 pi as the double nearest to it times four (exact scaling of pi).
#define CQM_FOUR_PI 0x1.921fb54442d18p+3

// Radon's seven-point rule, barycentric points and weights summing to one
// (closed form with sqrt(15); constants are the correctly rounded doubles).
__host__ __device__ __forceinline__ void radon7(int q, double& l0, double& l1, double& l2,
                                                double& w) {
  const double A = 0x1.9ede99c7af58fp-4, B = 0x1.e16cebd738bc0p-2;
  const double A2 = 0x1.9848598e1429cp-1, B2 = 0x1.e931428c74400p-5;  // 1-2A, 1-2B
  const double W0 = 0x1.ccccccccccccdp-3, WA = 0x1.01ec66adccf2ap-3, WB = 0x1.0f24aa63441e7p-3;
  const double T = 0x1.5555555555555p-2;  // 1/3
  switch (q) {
    case 0: l0 = T; l1 = T; l2 = T; w = W0; break;
    case 1: l0 = A; l1 = A; l2 = A2; w = WA; break;
    case 2: l0 = A; l1 = A2; l2 = A; w = WA; break;
    case 3: l0 = A2; l1 = A; l2 = A; w = WA; break;
    case 4: l0 = B; l1 = B; l2 = B2; w = WB; break;
    case 5: l0 = B; l1 = B2; l2 = B; w = WB; break;
    default: l0 = B2; l1 = B; l2 = B; w = WB; break;
  }
}

// Per-triangle geometry on the device.
struct Geom {
  int M;
  const int* tri;      // M x 3
  const double* P;     // M x 9: v0 (xyz), v1, v2
  const double* area;  // M
  const double* cen;   // M x 3, ((P0 + P1) + P2) / 3
  const double* diam;  // M, longest edge
};

// Quadrature tables on the device.
struct Quad {
  const double4* near_pt;  // collapsed rule per triangle: (l0, l1, l2, w), n_near points
  int n_near;
  const double4* ss_pt[3];  // Sauter-Schwab (x1, x2, y1, y2): [0] vertex, [1] edge, [2] identical
  const double* ss_w[3];
  int ss_n[3];
  double near_ratio;
  const double* t2;   // 2^(j/1024), j = 0..1023
  const double2* cs;  // (cos, sin)(j pi / 512), j = 0..1023
};

// c * exp(-s r) in FP64 with table-driven argument reduction (the method of
// Tang, ACM TOMS 15(2), 1989, for the exponential; the same for the circular
// functions): x = -Re(s) r = (1024 k + j) ln2/1024 + f with |f| <= ln2/2048,
// exp(x) = 2^k 2^(j/1024) exp(f); theta = Im(s) r = m pi/512 + g with
// |g| <= pi/1024, cis(theta) = cis(m pi/512) cis(g).  The reduction constants
// are split in two (Cody-Waite) so that n * hi is exact; exp(f), sin(g) and
// cos(g) use their Taylor polynomials, whose omitted terms are below 1.2e-18
// relative on these intervals (the largest, g^6 / 720 of cos(g) at
// |g| = pi / 1024), under half an FP64 ulp.  About 20 FP64 instructions per value.
__device__ __forceinline__ double2 cexp_c(double r, double c, double2 s, const Quad& q) {
  const double x = -s.x * r;
  if (!(x > -708.0)) return make_double2(0.0, 0.0);
  if (x > 700.0) {  // growing kernel (R > 1); outside the table's exponent range
    double sn, co;
    sincos(s.y * r, &sn, &co);
    const double e = exp(x) * c;
    return make_double2(e * co, -e * sn);
  }
  const double nx = rint(x * 0x1.71547652b82fep+10);  // 1024 / ln 2
  double f = fma(-nx, 0x1.62e42ff000000p-11, x);       // ln2/1024, high part
  f = fma(-nx, -0x1.718432a1b0e26p-45, f);             // ln2/1024, low part
  const long long n = (long long)nx;
  const int j = (int)(n & 1023);
  const long long k = (n - j) >> 10;
  double e = fma(fma(fma(fma(f, 1.0 / 24.0, 1.0 / 6.0), f, 0.5), f, 1.0), f, 1.0);
  e *= __ldg(q.t2 + j) * c;
  e *= __longlong_as_double((k + 1023) << 52);          // 2^k, -1022 <= k <= 1010 here
  const double th = s.y * r;
  const double nt = rint(th * 0x1.45f306dc9c883p+7);   // 512 / pi
  double g = fma(-nt, 0x1.921fb54400000p-8, th);       // pi/512, high part
  g = fma(-nt, 0x1.0b4611a626331p-42, g);              // pi/512, low part
  const int m = (int)((long long)nt & 1023);
  const double g2 = g * g;
  const double sg = g * fma(fma(g2, 1.0 / 120.0, -1.0 / 6.0), g2, 1.0);
  const double cg = fma(fma(g2, 1.0 / 24.0, -0.5), g2, 1.0);
  const double2 T = __ldg(q.cs + m);
  const double co = T.x * cg - T.y * sg;
  const double si = T.y * cg + T.x * sg;
  return make_double2(e * co, -e * si);
}

enum { CASE_REGULAR = 0, CASE_NEAR = 1, CASE_VERT = 2, CASE_EDGE = 3, CASE_IDENT = 4 };

// sqrt((x^2 + y^2) + z^2) without contraction, matching a plain evaluation.
__device__ __forceinline__ double exact_len(double dx, double dy, double dz) {
  return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

__device__ __forceinline__ int pair_case(const Geom& g, const Quad& q, int i, int j) {
  const int* a = g.tri + 3 * i;
  const int* b = g.tri + 3 * j;
  int shared = 0;
#pragma unroll
  for (int u = 0; u < 3; ++u)
#pragma unroll
    for (int v = 0; v < 3; ++v) shared += (a[u] == b[v]);
  if (shared >= 3) return CASE_IDENT;
  if (shared == 2) return CASE_EDGE;
  if (shared == 1) return CASE_VERT;
  const double* ci = g.cen + 3 * i;
  const double* cj = g.cen + 3 * j;
  double d = exact_len(__dsub_rn(ci[0], cj[0]), __dsub_rn(ci[1], cj[1]), __dsub_rn(ci[2], cj[2]));
  double lim = __dmul_rn(q.near_ratio, fmax(g.diam[i], g.diam[j]));
  return d < lim ? CASE_NEAR : CASE_REGULAR;
}

// Vertex order for a singular pair: identical -> stored order on both;
// common edge -> (u, w, third) with (u, w) the shared vertices in the order of
// triangle i; common vertex -> both rotated to start at the shared vertex.
__device__ __forceinline__ void singular_vertices(const int* tri, int i, int j, int cse, int vx[3],
                                                  int vy[3]) {
  const int* a = tri + 3 * i;
  const int* b = tri + 3 * j;
  if (cse == CASE_IDENT) {
    for (int k = 0; k < 3; ++k) vx[k] = vy[k] = a[k];
    return;
  }
  auto in_b = [&](int v) { return v == b[0] || v == b[1] || v == b[2]; };
  if (cse == CASE_EDGE) {
    int sh[2] = {a[0], a[1]}, n = 0, oi = a[2];
    for (int k = 0; k < 3; ++k) {
      if (in_b(a[k])) {
        if (n < 2) sh[n++] = a[k];
      } else {
        oi = a[k];
      }
    }
    int oj = -1;
    for (int k = 0; k < 3; ++k)
      if (b[k] != sh[0] && b[k] != sh[1]) oj = b[k];
    vx[0] = sh[0]; vx[1] = sh[1]; vx[2] = oi;
    vy[0] = sh[0]; vy[1] = sh[1]; vy[2] = oj;
    return;
  }
  int ka = 0, kb = 0;
  for (int k = 0; k < 3; ++k)
    if (in_b(a[k])) { ka = k; break; }
  for (int k = 0; k < 3; ++k)
    if (b[k] == a[ka]) { kb = k; break; }
  for (int k = 0; k < 3; ++k) {
    vx[k] = a[(ka + k) % 3];
    vy[k] = b[(kb + k) % 3];
  }
}

// Visit this lane's share (points lane, lane+nlanes, ...) of the quadrature
// points of pair (i, j): f(k, r, c) with k the point's index within the pair,
// r = |x - y| and c = weight / (4 pi r) (weights include the area factors).
// The pair is evaluated in canonical order, lower triangle index first: the
// single-layer Galerkin matrix is symmetric (symmetric kernel, same test and
// trial space), and the common-edge rule alone is not symmetric under
// exchanging the triangles, so this keeps V_l[i][j] == V_l[j][i] bit for bit.
template <class F>
__device__ __forceinline__ void pair_points(const Geom& g, const Quad& q, int i, int j, int cse,
                                            int lane, int nlanes, F&& f) {
  if (i > j) {
    const int t = i;
    i = j;
    j = t;
  }
  const double* Pi = g.P + 9 * i;
  const double* Pj = g.P + 9 * j;
  if (cse == CASE_REGULAR || cse == CASE_NEAR) {
    const int nq = (cse == CASE_REGULAR) ? 7 : q.n_near;
    const double aa = g.area[i] * g.area[j];
    for (int p = lane; p < nq * nq; p += nlanes) {
      int qa = p / nq, qb = p - qa * nq;
      double a0, a1, a2, wa, b0, b1, b2, wb;
      if (cse == CASE_REGULAR) {
        radon7(qa, a0, a1, a2, wa);
        radon7(qb, b0, b1, b2, wb);
      } else {
        double4 A = q.near_pt[qa], B = q.near_pt[qb];
        a0 = A.x; a1 = A.y; a2 = A.z; wa = A.w;
        b0 = B.x; b1 = B.y; b2 = B.z; wb = B.w;
      }
      double d0 = (a0 * Pi[0] + a1 * Pi[3] + a2 * Pi[6]) - (b0 * Pj[0] + b1 * Pj[3] + b2 * Pj[6]);
      double d1 = (a0 * Pi[1] + a1 * Pi[4] + a2 * Pi[7]) - (b0 * Pj[1] + b1 * Pj[4] + b2 * Pj[7]);
      double d2 = (a0 * Pi[2] + a1 * Pi[5] + a2 * Pi[8]) - (b0 * Pj[2] + b1 * Pj[5] + b2 * Pj[8]);
      double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      f(p, r, (wa * wb * aa) / (CQM_FOUR_PI * r));
    }
    return;
  }
  int vx[3], vy[3];
  singular_vertices(g.tri, i, j, cse, vx, vy);
  // physical vertices in the rule's order
  double X[9], Y[9];
  for (int k = 0; k < 3; ++k) {
    int tx = (vx[k] == g.tri[3 * i]) ? 0 : (vx[k] == g.tri[3 * i + 1] ? 1 : 2);
    int ty = (vy[k] == g.tri[3 * j]) ? 0 : (vy[k] == g.tri[3 * j + 1] ? 1 : 2);
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
    double4 z = pt[p];
    double a0 = 1.0 - z.x, a1 = z.x - z.y, a2 = z.y;
    double b0 = 1.0 - z.z, b1 = z.z - z.w, b2 = z.w;
    double d0 = (a0 * X[0] + a1 * X[3] + a2 * X[6]) - (b0 * Y[0] + b1 * Y[3] + b2 * Y[6]);
    double d1 = (a0 * X[1] + a1 * X[4] + a2 * X[7]) - (b0 * Y[1] + b1 * Y[4] + b2 * Y[7]);
    double d2 = (a0 * X[2] + a1 * X[5] + a2 * X[8]) - (b0 * Y[2] + b1 * Y[5] + b2 * Y[8]);
    double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    f(p, r, (wt[p] * aa) / (CQM_FOUR_PI * r));
  }
}

// Number of quadrature points of a pair of the given case.
__device__ __forceinline__ int pair_npoints(const Quad& q, int cse) {
  if (cse == CASE_REGULAR) return 49;
  if (cse == CASE_NEAR) return q.n_near * q.n_near;
  return q.ss_n[cse - CASE_VERT];
}

// c * exp(-s r) for NF frequencies, accumulated.
template <int NF>
__device__ __forceinline__ void kernel_accumulate_c(double r, double c, const double2* s, int nf,
                                                    double2* acc, const Quad& q) {
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    if (f < nf) {
      const double2 v = cexp_c(r, c, s[f], q);
      acc[f].x += v.x;
      acc[f].y += v.y;
    }
  }
}

// Accumulate this lane's share of the pair integral (i, j) for nf <= NF
// frequencies into acc.
template <int NF>
__device__ void pair_accumulate(const Geom& g, const Quad& q, int i, int j, int cse, int lane,
                                int nlanes, const double2* s, int nf, double2* acc) {
  pair_points(g, q, i, j, cse, lane, nlanes,
              [&](int, double r, double c) { kernel_accumulate_c<NF>(r, c, s, nf, acc, q); });
}

}  // namespace cqm
