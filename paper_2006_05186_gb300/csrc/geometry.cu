// Element geometry, CQM frequencies and the Galerkin data of the incident pulse.
#include "handle.cuh"

namespace cqm {

// Per triangle: vertices, area, centroid ((P0 + P1) + P2) / 3, longest edge
// (sqrt((x^2 + y^2) + z^2), uncontracted); flags zero-area triangles.
__global__ void k_geometry(int M, const double* __restrict__ xyz, const int* __restrict__ tri,
                           double* P, double* area, double* cen, double* diam, int* flag) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M) return;
  double v[9];
  for (int k = 0; k < 3; ++k) {
    int vi = tri[3 * t + k];
    for (int d = 0; d < 3; ++d) v[3 * k + d] = xyz[3 * vi + d];
  }
  for (int k = 0; k < 9; ++k) P[9 * t + k] = v[k];
  double e1x = v[3] - v[0], e1y = v[4] - v[1], e1z = v[5] - v[2];
  double e2x = v[6] - v[0], e2y = v[7] - v[1], e2z = v[8] - v[2];
  double cx = e1y * e2z - e1z * e2y, cy = e1z * e2x - e1x * e2z, cz = e1x * e2y - e1y * e2x;
  double a = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
  area[t] = a;
  if (!(a > 0.0)) atomicOr(flag, 1);
  for (int d = 0; d < 3; ++d)
    cen[3 * t + d] = __ddiv_rn(__dadd_rn(__dadd_rn(v[d], v[3 + d]), v[6 + d]), 3.0);
  double l0 = exact_len(__dsub_rn(v[3], v[0]), __dsub_rn(v[4], v[1]), __dsub_rn(v[5], v[2]));
  double l1 = exact_len(__dsub_rn(v[6], v[3]), __dsub_rn(v[7], v[4]), __dsub_rn(v[8], v[5]));
  double l2 = exact_len(__dsub_rn(v[0], v[6]), __dsub_rn(v[1], v[7]), __dsub_rn(v[2], v[8]));
  diam[t] = fmax(fmax(l0, l1), l2);
}

int build_geometry(cqm_handle* h, const cqm_mesh* mesh) {
  const int M = mesh->nt, nv = mesh->nv;
  CQM_TRY(h->xyz.allocate(h->alloc, 3 * (size_t)nv));
  CQM_TRY(h->tri.allocate(h->alloc, 3 * (size_t)M));
  CQM_TRY(h->P.allocate(h->alloc, 9 * (size_t)M));
  CQM_TRY(h->area.allocate(h->alloc, M));
  CQM_TRY(h->cen.allocate(h->alloc, 3 * (size_t)M));
  CQM_TRY(h->diam.allocate(h->alloc, M));
  CQM_TRY(h->flag.allocate(h->alloc, 4));
  CQM_CUDA_TRY(cudaMemcpyAsync(h->xyz.p, mesh->xyz, 3 * sizeof(double) * nv,
                               cudaMemcpyHostToDevice, h->stream));
  CQM_CUDA_TRY(cudaMemcpyAsync(h->tri.p, mesh->tri, 3 * sizeof(int) * M, cudaMemcpyHostToDevice,
                               h->stream));
  CQM_CUDA_TRY(cudaMemsetAsync(h->flag.p, 0, 4 * sizeof(int), h->stream));
  {
    ProfScope ps_(h, CQM_K_GEOMETRY);
    k_geometry<<<grid_for(M, 256), 256, 0, h->stream>>>(M, h->xyz.p, h->tri.p, h->P.p, h->area.p,
                                                        h->cen.p, h->diam.p, h->flag.p);
  }
  CQM_CHECK_LAUNCH();
  int flag = 0;
  CQM_CUDA_TRY(cudaMemcpyAsync(&flag, h->flag.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (flag & 1) {
    set_last_error("mesh has a triangle of zero area");
    return CQM_EINVAL;
  }
  return CQM_OK;
}

// s_l = chi(R zeta^l) / dt, chi of BDF-k = sum_{j=1..k} (1 - z)^j / j  (eq. cqm_freq).
__global__ void k_frequencies(int L, int bdf, double R, double dt, double2* s) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  double sn, cs;
  sincospi(2.0 * (double)l / (double)L, &sn, &cs);
  double2 w = make_double2(1.0 - R * cs, -R * sn);  // 1 - z
  double2 acc = w, pw = w;
  for (int j = 2; j <= bdf; ++j) {
    pw = cmul(pw, w);
    acc = cadd(acc, cscale(pw, 1.0 / j));
  }
  s[l] = cscale(acc, 1.0 / dt);
}

int build_frequencies(cqm_handle* h) {
  CQM_TRY(h->s.allocate(h->alloc, h->L));
  {
    ProfScope ps_(h, CQM_K_GEOMETRY);
    k_frequencies<<<grid_for(h->L, 128), 128, 0, h->stream>>>(h->L, h->bdf, h->R, h->dt, h->s.p);
  }
  CQM_CHECK_LAUNCH();
  h->s_host.resize(h->L);
  CQM_CUDA_TRY(cudaMemcpyAsync(h->s_host.data(), h->s.p, sizeof(double2) * h->L,
                               cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CQM_OK;
}

// b[n][i] = |tau_i| sum_q w_q exp(-((t_n - delay - d.x_q) / width)^2), Radon rule.
__global__ void k_rhs_plane_wave(int M, int N, double dt, double dx, double dy, double dz,
                                 double width, double delay, const double* __restrict__ P,
                                 const double* __restrict__ area, double* rhs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double* v = P + 9 * i;
  double proj[7], wq[7];
  for (int q = 0; q < 7; ++q) {
    double l0, l1, l2, w;
    radon7(q, l0, l1, l2, w);
    double x = l0 * v[0] + l1 * v[3] + l2 * v[6];
    double y = l0 * v[1] + l1 * v[4] + l2 * v[7];
    double z = l0 * v[2] + l1 * v[5] + l2 * v[8];
    proj[q] = x * dx + y * dy + z * dz;
    wq[q] = w;
  }
  const double a = area[i];
  for (int n = 0; n <= N; ++n) {
    double t = dt * n, acc = 0.0;
    for (int q = 0; q < 7; ++q) {
      double u = (t - delay - proj[q]) / width;
      acc += wq[q] * exp(-u * u);
    }
    rhs[(size_t)n * M + i] = acc * a;
  }
}

int rhs_plane_wave(cqm_handle* h, const double dir[3], double width, double delay, double* d_rhs) {
  double nrm = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  if (!(nrm > 0.0) || !(width > 0.0)) {
    set_last_error("plane wave: direction must be nonzero and width > 0");
    return CQM_EINVAL;
  }
  {
    ProfScope ps_(h, CQM_K_RHS);
    k_rhs_plane_wave<<<grid_for(h->M, 128), 128, 0, h->stream>>>(
        h->M, h->N, h->dt, dir[0] / nrm, dir[1] / nrm, dir[2] / nrm, width, delay, h->P.p,
        h->area.p, d_rhs);
  }
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

}  // namespace cqm
