// C ABI of libcqmbem: argument checks, orchestration of the setup (Alg. 3)
// and of the decoupled frequency-domain solve (Remark in Sec. 6.2).
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "handle.cuh"

namespace cqm {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

int check_wait_flag(cqm_handle* h) {
  int w = 0;
  CQM_CUDA_TRY(cudaMemcpyAsync(&w, h->flag.p + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (w != 0) {
    CQM_TRY(clear_wait_flag(h));
    set_last_error("a bounded device wait expired in the tensor-core far coupling (limit " +
                   std::to_string(h->wait_limit_ns) + " ns)");
    return CQM_ETIMEOUT;
  }
  return CQM_OK;
}

int clear_wait_flag(cqm_handle* h) {
  CQM_CUDA_TRY(cudaMemsetAsync(h->flag.p + 1, 0, sizeof(int), h->stream));
  return CQM_OK;
}

// Device scratch of a call: released when the call returns.
struct Scratch {
  Allocator* a;
  std::vector<std::pair<void*, size_t>> blocks;
  explicit Scratch(Allocator* al) : a(al) {}
  template <class T>
  int get(T** p, size_t count) {
    void* q = nullptr;
    int s = a->alloc(&q, count * sizeof(T));
    if (s == CQM_OK) blocks.push_back({q, count * sizeof(T)});
    *p = (T*)q;
    return s;
  }
  ~Scratch() {
    for (auto& b : blocks) a->release(b.first, b.second);
  }
};

static float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

}  // namespace cqm

using namespace cqm;

extern "C" {

int cqm_params_default(cqm_params* p) {
  if (!p) return CQM_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->mode = CQM_MODE_H2MACA;
  p->R = 0.0;
  p->g_sing = 5;
  p->g_near = 5;
  p->near_ratio = 2.0;
  p->n_min = 32;
  p->eta = 1.0;
  p->cheb_m = 4;
  p->aca_eps = 1e-6;
  p->rank_cap = 32;
  p->gmres_restart = 50;
  p->gmres_max_iter = 3000;
  p->gmres_tol = 1e-13;
  p->profile = 0;
  p->precond = 1;
  p->inner_fp32 = 1;
  p->inner_rtol = 1e-5;
  p->exact_ff = 1;
  p->expand_near = 1;
  p->expand_far = 1;
  p->cache_quadrature = 1;
  p->maca_ff = 1;
  p->tensor_cores = 1;
  p->allocator = nullptr;
  p->tc_single_ratio = 1e-3;
  return CQM_OK;
}

const char* cqm_bem_strerror(int status) {
  switch (status) {
    case CQM_OK: return "ok";
    case CQM_EINVAL: return "invalid argument";
    case CQM_ENOMEM: return "out of device memory";
    case CQM_ENOCONV: return "GMRES did not converge within the iteration cap";
    case CQM_ETIMEOUT: return "a bounded device wait timed out";
    case CQM_ECUDA: return "CUDA runtime error";
    case CQM_ECAPACITY: return "a fixed device capacity was exceeded";
    default: return "unknown status";
  }
}

const char* cqm_bem_last_error(void) { return g_last_error.c_str(); }

int cqm_bem_destroy(cqm_handle* h) {
  if (!h) return CQM_OK;
  Allocator& A = h->alloc;
  h->xyz.free(A); h->tri.free(A); h->P.free(A); h->area.free(A); h->cen.free(A);
  h->diam.free(A); h->flag.free(A); h->near_pt.free(A);
  h->exp_t2_ff.free(A); h->exp_cs_ff.free(A); h->pt_r0.free(A);
  h->fpt_d.free(A); h->fpt_c.free(A); h->fpt_r0.free(A);
  h->tc2_first.free(A); h->tc2_img.free(A); h->tc2_tail.free(A); h->tc2_t1.free(A);
  for (int t = 0; t < 3; ++t) { h->ss_pt[t].free(A); h->ss_w[t].free(A); }
  h->s.free(A); h->Vd.free(A); h->exp_t2.free(A); h->exp_cs.free(A);
  h->perm.free(A); h->node_begin.free(A); h->node_end.free(A); h->node_son0.free(A);
  h->node_son1.free(A); h->node_parent.free(A); h->node_level.free(A); h->node_lo.free(A);
  h->node_hi.free(A);
  h->near_rc.free(A); h->far_rc.free(A); h->near_rowptr.free(A); h->far_rowptr.free(A);
  h->cheb.free(A); h->Uleaf.free(A); h->Etr.free(A);
  h->near_rank.free(A); h->far_rank.free(A); h->near_off.free(A);
  h->nearC.free(A); h->nearD.free(A); h->farC.free(A); h->farD.free(A);
  h->xhat.free(A); h->yhat.free(A); h->d_leaves.free(A); h->d_far_rows.free(A);
  h->Pinv.free(A);
  h->far_items.free(A); h->near_items.free(A); h->far_order.free(A); h->far_item_ptr.free(A); h->near_item_ptr.free(A);
  h->part_f.free(A); h->part_d.free(A);
  h->pt_off.free(A); h->pt_cnt.free(A); h->pt_r.free(A); h->pt_c.free(A);
  h->nearC_f.free(A); h->nearD_f.free(A); h->farC_f.free(A); h->farD_f.free(A);
  h->nearV.free(A); h->nearV_f.free(A); h->nearV_off.free(A); h->farS.free(A);
  h->xhat_f.free(A); h->yhat_f.free(A); h->Uleaf_f.free(A); h->Etr_f.free(A); h->x32.free(A);
  mot_release(h);
  dl_release(h);
  cudaStreamSynchronize(h->stream);
  prof_release(h);
  delete h;
  return CQM_OK;
}

int cqm_bem_setup(const cqm_mesh* mesh, double dt, int32_t N, int32_t bdf_order,
                  const cqm_params* params, void* cuda_stream, cqm_handle** out) {
  set_last_error("");
  if (!out) { set_last_error("out is NULL"); return CQM_EINVAL; }
  *out = nullptr;
  if (!mesh || !mesh->xyz || !mesh->tri || mesh->nt < 1 || mesh->nv < 3) {
    set_last_error("mesh is NULL or empty");
    return CQM_EINVAL;
  }
  if (!(dt > 0.0) || N < 1 || (bdf_order != 1 && bdf_order != 2)) {
    set_last_error("need dt > 0, N >= 1, bdf_order in {1, 2}");
    return CQM_EINVAL;
  }
  if (N > CQM_MAX_STEPS) {
    set_last_error("N = " + std::to_string(N) + " exceeds CQM_MAX_STEPS = " +
                   std::to_string(CQM_MAX_STEPS) + " (transform tables in shared memory)");
    return CQM_EINVAL;
  }
  for (int64_t k = 0; k < 3 * (int64_t)mesh->nt; ++k) {
    if (mesh->tri[k] < 0 || mesh->tri[k] >= mesh->nv) {
      set_last_error("triangle vertex index out of range at entry " + std::to_string(k));
      return CQM_EINVAL;
    }
  }
  for (int t = 0; t < mesh->nt; ++t) {
    const int32_t* v = mesh->tri + 3 * t;
    if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) {
      set_last_error("triangle " + std::to_string(t) + " repeats a vertex");
      return CQM_EINVAL;
    }
  }
  cqm_params p;
  if (params) p = *params;
  else cqm_params_default(&p);
  if ((p.mode != CQM_MODE_DENSE && p.mode != CQM_MODE_H2MACA) || p.g_sing < 1 || p.g_sing > 12 ||
      p.g_near < 1 || p.g_near > 12 || !(p.near_ratio >= 0.0) || p.n_min < 1 || !(p.eta > 0.0) ||
      p.cheb_m < 1 || p.cheb_m > 4 || !(p.aca_eps > 0.0) || p.rank_cap < 1 || p.rank_cap > 64 ||
      (p.mode == CQM_MODE_H2MACA && p.n_min > 32) ||
      p.gmres_restart < 1 || p.gmres_max_iter < 1 || !(p.gmres_tol > 0.0) ||
      !(p.inner_rtol >= 0.0 && p.inner_rtol < 1.0) || !(p.tc_single_ratio >= 0.0)) {
    set_last_error("parameter out of range");
    return CQM_EINVAL;
  }
  cqm_handle* h = new cqm_handle();
  h->stream = (cudaStream_t)cuda_stream;
  h->alloc.stream = h->stream;
  h->alloc.user = p.allocator;
  h->params = p;
  h->M = mesh->nt;
  h->nv = mesh->nv;
  h->N = N;
  h->L = N + 1;
  h->Ls = h->L / 2 + 1;
  h->bdf = bdf_order;
  h->dt = dt;
  h->R = p.R > 0.0 ? p.R : std::pow(1e-10, 1.0 / (2.0 * h->L));
  h->m = p.cheb_m;
  h->p = p.cheb_m * p.cheb_m * p.cheb_m;
  h->rank_cap = std::min(std::min(p.rank_cap, 64), h->Ls);
  h->prof_on = p.profile != 0;
  int st = CQM_OK;
  cudaEvent_t ev[5];
  for (auto& e : ev) cudaEventCreate(&e);
  cudaEventRecord(ev[0], h->stream);
  do {
    if ((st = build_geometry(h, mesh)) != CQM_OK) break;
    if ((st = build_quad_tables(h)) != CQM_OK) break;
    if ((st = build_frequencies(h)) != CQM_OK) break;
    cudaEventRecord(ev[1], h->stream);
    if (p.mode == CQM_MODE_DENSE) {
      cudaEventRecord(ev[2], h->stream);
      cudaEventRecord(ev[3], h->stream);
      if ((st = assemble_dense(h)) != CQM_OK) break;
    } else {
      if ((st = build_tree(h)) != CQM_OK) break;
      if ((st = build_partition(h)) != CQM_OK) break;
      cudaEventRecord(ev[2], h->stream);
      if ((st = build_bases(h)) != CQM_OK) break;
      cudaEventRecord(ev[3], h->stream);
      if ((st = build_maca(h)) != CQM_OK) break;
      if ((st = build_work_items(h)) != CQM_OK) break;
      if (p.precond && (st = build_precond(h)) != CQM_OK) break;
      // the expanded near field (Ls x near entries x 24 bytes) is admitted when it
      // takes at most a quarter of the device memory; otherwise it stays factored
      {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
          st = CQM_ECUDA;
          break;
        }
        const double bytes = 24.0 * (double)h->Ls * (double)h->info.near_entries;
        h->expand_near_ok = p.expand_near && bytes <= 0.25 * (double)total_b;
      }
      if (h->expand_near_ok && !p.exact_ff && (st = build_near_expanded(h)) != CQM_OK) break;
      if (p.inner_fp32) {
        if ((st = build_f32_copy(h)) != CQM_OK) break;
        h->use_f32 = true;
      }
      if (p.exact_ff && (st = factors_to_ff(h)) != CQM_OK) break;
      if (p.exact_ff && h->expand_near_ok && (st = build_near_expanded_ff(h)) != CQM_OK) break;
      if (p.exact_ff && p.expand_far && (st = build_far_expanded(h)) != CQM_OK) break;
    }
    cudaEventRecord(ev[4], h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      set_last_error(std::string("setup: ") + cudaGetErrorString(e));
      st = CQM_ECUDA;
    }
  } while (0);
  if (st == CQM_OK) {
    cqm_setup_info& I = h->info;
    I.nt = h->M; I.nv = h->nv; I.N = h->N; I.L = h->L; I.Ls = h->Ls; I.mode = p.mode;
    I.n_nodes = h->n_nodes; I.n_leaves = h->n_leaves; I.n_near = h->n_near; I.n_far = h->n_far;
    I.R = h->R;
    I.device_bytes = h->alloc.bytes_held;
    I.near_expanded = h->near_expanded ? 1 : 0;
    I.far_expanded = h->far_expanded ? 1 : 0;
    I.t_geometry_ms = elapsed(ev[0], ev[1]);
    I.t_tree_ms = elapsed(ev[1], ev[2]);
    I.t_bases_ms = elapsed(ev[2], ev[3]);
    I.t_assembly_ms = elapsed(ev[3], ev[4]);
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (st != CQM_OK) {
    std::string msg = g_last_error;
    cqm_bem_destroy(h);
    set_last_error(msg);
    return st;
  }
  *out = h;
  return CQM_OK;
}

int cqm_bem_get_info(const cqm_handle* h, cqm_setup_info* out) {
  if (!h || !out) return CQM_EINVAL;
  *out = h->info;
  return CQM_OK;
}

int cqm_bem_get_frequencies(const cqm_handle* h, double* out) {
  if (!h || !out) return CQM_EINVAL;
  std::memcpy(out, h->s_host.data(), sizeof(double2) * h->L);
  return CQM_OK;
}

int cqm_bem_rhs_plane_wave(cqm_handle* h, const double dir[3], double width, double delay,
                           double* rhs, int32_t mem) {
  if (!h || !dir || !rhs || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE)) return CQM_EINVAL;
  set_last_error("");
  const size_t n = (size_t)(h->N + 1) * h->M;
  Scratch S(&h->alloc);
  double* d = rhs;
  if (mem == CQM_MEM_HOST) CQM_TRY(S.get(&d, n));
  CQM_TRY(rhs_plane_wave(h, dir, width, delay, d));
  if (mem == CQM_MEM_HOST)
    CQM_CUDA_TRY(cudaMemcpyAsync(rhs, d, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CQM_OK;
}

int cqm_bem_forward_transform(cqm_handle* h, const double* b, double* ghat, int32_t mem) {
  if (!h || !b || !ghat || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE)) return CQM_EINVAL;
  const size_t nb = (size_t)h->L * h->M, ng = (size_t)h->Ls * h->M;
  Scratch S(&h->alloc);
  const double* db = b;
  double2* dg = (double2*)ghat;
  if (mem == CQM_MEM_HOST) {
    double* t;
    CQM_TRY(S.get(&t, nb));
    CQM_CUDA_TRY(cudaMemcpyAsync(t, b, nb * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    db = t;
    CQM_TRY(S.get(&dg, ng));
  }
  CQM_TRY(forward_transform(h, db, dg));
  if (mem == CQM_MEM_HOST)
    CQM_CUDA_TRY(cudaMemcpyAsync(ghat, dg, ng * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CQM_OK;
}

int cqm_bem_inverse_transform(cqm_handle* h, const double* qhat, double* q, int32_t mem) {
  if (!h || !qhat || !q || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE)) return CQM_EINVAL;
  const size_t nq = (size_t)h->L * h->M, ng = (size_t)h->Ls * h->M;
  Scratch S(&h->alloc);
  const double2* dg = (const double2*)qhat;
  double* dq = q;
  if (mem == CQM_MEM_HOST) {
    double2* t;
    CQM_TRY(S.get(&t, ng));
    CQM_CUDA_TRY(cudaMemcpyAsync(t, qhat, ng * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
    dg = t;
    CQM_TRY(S.get(&dq, nq));
  }
  CQM_TRY(inverse_transform(h, dg, dq));
  if (mem == CQM_MEM_HOST)
    CQM_CUDA_TRY(cudaMemcpyAsync(q, dq, nq * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CQM_OK;
}

int cqm_bem_entries(cqm_handle* h, int64_t npairs, const int32_t* I, const int32_t* J,
                    int32_t nfreq, const int32_t* freq, double* out, int32_t mem) {
  if (!h || npairs < 0 || nfreq < 0 || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE))
    return CQM_EINVAL;
  if (npairs == 0 || nfreq == 0) return CQM_OK;
  if (!I || !J || !freq || !out) return CQM_EINVAL;
  Scratch S(&h->alloc);
  const int *dI = I, *dJ = J, *dF = freq;
  double2* dO = (double2*)out;
  if (mem == CQM_MEM_HOST) {
    for (int64_t k = 0; k < npairs; ++k)
      if (I[k] < 0 || I[k] >= h->M || J[k] < 0 || J[k] >= h->M) {
        set_last_error("pair index out of range");
        return CQM_EINVAL;
      }
    for (int f = 0; f < nfreq; ++f)
      if (freq[f] < 0 || freq[f] >= h->L) {
        set_last_error("frequency index out of range");
        return CQM_EINVAL;
      }
    int *tI, *tJ, *tF;
    CQM_TRY(S.get(&tI, npairs));
    CQM_TRY(S.get(&tJ, npairs));
    CQM_TRY(S.get(&tF, nfreq));
    CQM_TRY(S.get(&dO, (size_t)npairs * nfreq));
    CQM_CUDA_TRY(cudaMemcpyAsync(tI, I, npairs * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CQM_CUDA_TRY(cudaMemcpyAsync(tJ, J, npairs * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CQM_CUDA_TRY(cudaMemcpyAsync(tF, freq, nfreq * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    dI = tI; dJ = tJ; dF = tF;
  }
  CQM_TRY(entries_list(h, npairs, dI, dJ, nfreq, dF, dO));
  if (mem == CQM_MEM_HOST)
    CQM_CUDA_TRY(cudaMemcpyAsync(out, dO, (size_t)npairs * nfreq * sizeof(double2),
                                 cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CQM_OK;
}

int cqm_bem_apply(cqm_handle* h, const double* x, double* y, int32_t mem) {
  if (!h || !x || !y || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE)) return CQM_EINVAL;
  const size_t n = (size_t)h->Ls * h->M;
  Scratch S(&h->alloc);
  const double2* dx = (const double2*)x;
  double2* dy = (double2*)y;
  if (mem == CQM_MEM_HOST) {
    double2* t;
    CQM_TRY(S.get(&t, n));
    CQM_CUDA_TRY(cudaMemcpyAsync(t, x, n * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
    dx = t;
    CQM_TRY(S.get(&dy, n));
  }
  CQM_TRY(apply_operator(h, dx, dy));
  if (mem == CQM_MEM_HOST)
    CQM_CUDA_TRY(cudaMemcpyAsync(y, dy, n * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CQM_OK;
}

int cqm_bem_apply_inner(cqm_handle* h, const double* x, double* y, int32_t mem) {
  if (!h || !x || !y || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE)) return CQM_EINVAL;
  const size_t n = (size_t)h->Ls * h->M;
  Scratch S(&h->alloc);
  const double2* dx = (const double2*)x;
  double2* dy = (double2*)y;
  if (mem == CQM_MEM_HOST) {
    double2* t;
    CQM_TRY(S.get(&t, n));
    CQM_CUDA_TRY(cudaMemcpyAsync(t, x, n * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
    dx = t;
    CQM_TRY(S.get(&dy, n));
  }
  CQM_TRY(clear_wait_flag(h));
  CQM_TRY(apply_operator_inner(h, dx, dy));
  if (mem == CQM_MEM_HOST)
    CQM_CUDA_TRY(cudaMemcpyAsync(y, dy, n * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return check_wait_flag(h);
}

int cqm_bem_solve_frequencies(cqm_handle* h, const double* ghat, double* qhat, int32_t mem,
                              cqm_solve_info* info) {
  if (!h || !ghat || !qhat || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE)) return CQM_EINVAL;
  const size_t n = (size_t)h->Ls * h->M;
  Scratch S(&h->alloc);
  const double2* dg = (const double2*)ghat;
  double2* dq = (double2*)qhat;
  if (mem == CQM_MEM_HOST) {
    double2* t;
    CQM_TRY(S.get(&t, n));
    CQM_CUDA_TRY(cudaMemcpyAsync(t, ghat, n * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
    dg = t;
    CQM_TRY(S.get(&dq, n));
  }
  cqm_solve_info loc{};
  int st = gmres_solve(h, dg, dq, info ? info : &loc);
  if (st != CQM_OK && st != CQM_ENOCONV) return st;
  if (mem == CQM_MEM_HOST)
    CQM_CUDA_TRY(cudaMemcpyAsync(qhat, dq, n * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return st;
}

int cqm_bem_solve_mot(cqm_handle* h, const double* rhs, double* density, int32_t mem,
                      cqm_solve_info* info) {
  if (!h || !rhs || !density || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE)) return CQM_EINVAL;
  set_last_error("");
  const size_t nt = (size_t)h->L * h->M;
  Scratch S(&h->alloc);
  const double* db = rhs;
  double* dq = density;
  if (mem == CQM_MEM_HOST) {
    double* t;
    CQM_TRY(S.get(&t, nt));
    CQM_CUDA_TRY(cudaMemcpyAsync(t, rhs, nt * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    db = t;
    CQM_TRY(S.get(&dq, nt));
  }
  cqm_solve_info loc{};
  CQM_TRY(mot_solve(h, db, dq, info ? info : &loc));
  if (mem == CQM_MEM_HOST)
    CQM_CUDA_TRY(cudaMemcpyAsync(density, dq, nt * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CQM_OK;
}

int cqm_bem_apply_double_layer(cqm_handle* h, const double* x, double* y, int32_t mem) {
  if (!h || !x || !y || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE)) return CQM_EINVAL;
  set_last_error("");
  const size_t n = (size_t)h->Ls * h->M;
  Scratch S(&h->alloc);
  const double2* dx = (const double2*)x;
  double2* dy = (double2*)y;
  if (mem == CQM_MEM_HOST) {
    double2* t;
    CQM_TRY(S.get(&t, n));
    CQM_CUDA_TRY(cudaMemcpyAsync(t, x, n * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
    dx = t;
    CQM_TRY(S.get(&dy, n));
  }
  CQM_TRY(dl_apply(h, dx, dy));
  if (mem == CQM_MEM_HOST)
    CQM_CUDA_TRY(cudaMemcpyAsync(y, dy, n * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CQM_OK;
}

int cqm_bem_p1_matrices(cqm_handle* h, double* K1, double* Kp, double* D, int32_t mem) {
  if (!h || !K1 || !Kp || !D || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE)) return CQM_EINVAL;
  set_last_error("");
  const size_t nk = (size_t)h->Ls * h->M * h->nv, nd = (size_t)h->Ls * h->nv * h->nv;
  Scratch S(&h->alloc);
  double2 *dK1 = (double2*)K1, *dKp = (double2*)Kp, *dD = (double2*)D;
  if (mem == CQM_MEM_HOST) {
    CQM_TRY(S.get(&dK1, nk));
    CQM_TRY(S.get(&dKp, nk));
    CQM_TRY(S.get(&dD, nd));
  }
  CQM_TRY(p1_matrices(h, dK1, dKp, dD));
  if (mem == CQM_MEM_HOST) {
    CQM_CUDA_TRY(cudaMemcpyAsync(K1, dK1, nk * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
    CQM_CUDA_TRY(cudaMemcpyAsync(Kp, dKp, nk * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
    CQM_CUDA_TRY(cudaMemcpyAsync(D, dD, nd * sizeof(double2), cudaMemcpyDeviceToHost, h->stream));
  }
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CQM_OK;
}

int cqm_bem_solve_mixed(cqm_handle* h, const int32_t* dmask, const double* gD, const double* gN, double* q,
                        double* u, int32_t mem) {
  if (!h || !dmask || !gD || !gN || !q || !u || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE))
    return CQM_EINVAL;
  set_last_error("");
  const size_t nD = (size_t)h->L * h->nv, nN = (size_t)h->L * h->M;
  Scratch S(&h->alloc);
  const double *dgD = gD, *dgN = gN;
  double *dq = q, *du = u;
  if (mem == CQM_MEM_HOST) {
    double *t1, *t2;
    CQM_TRY(S.get(&t1, nD));
    CQM_TRY(S.get(&t2, nN));
    CQM_CUDA_TRY(cudaMemcpyAsync(t1, gD, nD * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CQM_CUDA_TRY(cudaMemcpyAsync(t2, gN, nN * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    dgD = t1;
    dgN = t2;
    CQM_TRY(S.get(&dq, nN));
    CQM_TRY(S.get(&du, nD));
  }
  CQM_TRY(mixed_solve(h, dmask, dgD, dgN, dq, du));
  if (mem == CQM_MEM_HOST) {
    CQM_CUDA_TRY(cudaMemcpyAsync(q, dq, nN * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CQM_CUDA_TRY(cudaMemcpyAsync(u, du, nD * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CQM_OK;
}

int cqm_bem_solve_dirichlet(cqm_handle* h, const double* g, double* q, int32_t mem, cqm_solve_info* info) {
  if (!h || !g || !q || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE)) return CQM_EINVAL;
  set_last_error("");
  const size_t nt = (size_t)h->L * h->M;
  Scratch S(&h->alloc);
  const double* dg = g;
  double* dq = q;
  if (mem == CQM_MEM_HOST) {
    double* t;
    CQM_TRY(S.get(&t, nt));
    CQM_CUDA_TRY(cudaMemcpyAsync(t, g, nt * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    dg = t;
    CQM_TRY(S.get(&dq, nt));
  }
  cqm_solve_info loc{};
  const int st = dl_solve(h, dg, dq, info ? info : &loc);
  if (st != CQM_OK && st != CQM_ENOCONV) return st;
  if (mem == CQM_MEM_HOST)
    CQM_CUDA_TRY(cudaMemcpyAsync(q, dq, nt * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return st;
}

int cqm_bem_mot_weight(cqm_handle* h, int32_t n, double* W, int32_t mem) {
  if (!h || !W || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE)) return CQM_EINVAL;
  set_last_error("");
  const size_t nn = (size_t)h->M * h->M;
  Scratch S(&h->alloc);
  double* dw = W;
  if (mem == CQM_MEM_HOST) CQM_TRY(S.get(&dw, nn));
  CQM_TRY(mot_weight(h, n, dw));
  if (mem == CQM_MEM_HOST) {
    CQM_CUDA_TRY(cudaMemcpyAsync(W, dw, nn * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  }
  return CQM_OK;
}

int cqm_bem_solve(cqm_handle* h, const double* rhs, double* density, int32_t mem,
                  cqm_solve_info* info) {
  if (!h || !rhs || !density || (mem != CQM_MEM_HOST && mem != CQM_MEM_DEVICE)) return CQM_EINVAL;
  set_last_error("");
  const size_t nt = (size_t)h->L * h->M, nf = (size_t)h->Ls * h->M;
  Scratch S(&h->alloc);
  const double* db = rhs;
  double* dq = density;
  if (mem == CQM_MEM_HOST) {
    double *tb, *tq;
    CQM_TRY(S.get(&tb, nt));
    CQM_TRY(S.get(&tq, nt));
    CQM_CUDA_TRY(cudaMemcpyAsync(tb, rhs, nt * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    db = tb;
    dq = tq;
  }
  double2 *ghat, *qhat;
  CQM_TRY(S.get(&ghat, nf));
  CQM_TRY(S.get(&qhat, nf));
  cudaEvent_t ev[4];
  for (auto& e : ev) cudaEventCreate(&e);
  cudaEventRecord(ev[0], h->stream);
  int st = forward_transform(h, db, ghat);
  cudaEventRecord(ev[1], h->stream);
  cqm_solve_info loc{};
  cqm_solve_info* I = info ? info : &loc;
  if (st == CQM_OK) {
    st = gmres_solve(h, ghat, qhat, I);
  }
  cudaEventRecord(ev[2], h->stream);
  if (st == CQM_OK || st == CQM_ENOCONV) {
    int s2 = inverse_transform(h, qhat, dq);
    if (s2 != CQM_OK) st = s2;
  }
  cudaEventRecord(ev[3], h->stream);
  if (mem == CQM_MEM_HOST && (st == CQM_OK || st == CQM_ENOCONV)) {
    cudaError_t e = cudaMemcpyAsync(density, dq, nt * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); st = CQM_ECUDA; }
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess && st == CQM_OK) {
    set_last_error(cudaGetErrorString(e));
    st = CQM_ECUDA;
  }
  I->t_forward_ms = elapsed(ev[0], ev[1]);
  I->t_inverse_ms = elapsed(ev[2], ev[3]);
  // imaginary parts that conjugate symmetry forces to zero: Im qhat_0 (s_0 real)
  double2 q0 = make_double2(0, 0);
  if (st == CQM_OK || st == CQM_ENOCONV) {
    cudaMemcpy(&q0, qhat, sizeof(double2), cudaMemcpyDeviceToHost);
  }
  I->max_imag = std::fabs(q0.y);
  for (auto& ev1 : ev) cudaEventDestroy(ev1);
  return st;
}

int cqm_bem_get_tree(const cqm_handle* h, int32_t* perm, int32_t* begin, int32_t* end,
                     int32_t* son0, int32_t* son1, int32_t* level, double* lo, double* hi) {
  if (!h) return CQM_EINVAL;
  if (h->n_nodes == 0) {
    set_last_error("no cluster tree (dense mode)");
    return CQM_EINVAL;
  }
  const int n = h->n_nodes;
  cudaStream_t S = h->stream;
  if (perm) CQM_CUDA_TRY(cudaMemcpyAsync(perm, h->perm.p, sizeof(int) * h->M, cudaMemcpyDeviceToHost, S));
  if (begin) CQM_CUDA_TRY(cudaMemcpyAsync(begin, h->node_begin.p, sizeof(int) * n, cudaMemcpyDeviceToHost, S));
  if (end) CQM_CUDA_TRY(cudaMemcpyAsync(end, h->node_end.p, sizeof(int) * n, cudaMemcpyDeviceToHost, S));
  if (son0) CQM_CUDA_TRY(cudaMemcpyAsync(son0, h->node_son0.p, sizeof(int) * n, cudaMemcpyDeviceToHost, S));
  if (son1) CQM_CUDA_TRY(cudaMemcpyAsync(son1, h->node_son1.p, sizeof(int) * n, cudaMemcpyDeviceToHost, S));
  if (level) CQM_CUDA_TRY(cudaMemcpyAsync(level, h->node_level.p, sizeof(int) * n, cudaMemcpyDeviceToHost, S));
  if (lo) CQM_CUDA_TRY(cudaMemcpyAsync(lo, h->node_lo.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, S));
  if (hi) CQM_CUDA_TRY(cudaMemcpyAsync(hi, h->node_hi.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, S));
  CQM_CUDA_TRY(cudaStreamSynchronize(S));
  return CQM_OK;
}

int cqm_bem_get_blocks(const cqm_handle* h, int32_t* near_rc, int32_t* far_rc, int32_t* near_rank,
                       int32_t* far_rank) {
  if (!h) return CQM_EINVAL;
  if (h->n_nodes == 0) {
    set_last_error("no block partition (dense mode)");
    return CQM_EINVAL;
  }
  for (int b = 0; b < h->n_near; ++b) {
    if (near_rc) { near_rc[2 * b] = h->h_near[b].x; near_rc[2 * b + 1] = h->h_near[b].y; }
    if (near_rank) near_rank[b] = b < (int)h->h_near_rank.size() ? h->h_near_rank[b] : 0;
  }
  for (int b = 0; b < h->n_far; ++b) {
    if (far_rc) { far_rc[2 * b] = h->h_far[b].x; far_rc[2 * b + 1] = h->h_far[b].y; }
    if (far_rank) far_rank[b] = b < (int)h->h_far_rank.size() ? h->h_far_rank[b] : 0;
  }
  return CQM_OK;
}

int cqm_bem_get_block_factors(const cqm_handle* h, int32_t kind, int32_t b, int32_t* rank,
                              int32_t* rows, int32_t* cols, double* Cout, double* Dout) {
  if (!h || (kind != 0 && kind != 1)) return CQM_EINVAL;
  const int nb = kind == 0 ? h->n_near : h->n_far;
  if (b < 0 || b >= nb) {
    set_last_error("block index out of range");
    return CQM_EINVAL;
  }
  const std::vector<int>& rk = kind == 0 ? h->h_near_rank : h->h_far_rank;
  if ((int)rk.size() != nb) {
    set_last_error("no MACA factors");
    return CQM_EINVAL;
  }
  int2 rc = kind == 0 ? h->h_near[b] : h->h_far[b];
  int nr = kind == 0 ? h->h_end[rc.x] - h->h_begin[rc.x] : h->p;
  int nc = kind == 0 ? h->h_end[rc.y] - h->h_begin[rc.y] : h->p;
  int r = rk[b];
  if (rank) *rank = r;
  if (rows) *rows = nr;
  if (cols) *cols = nc;
  cudaStream_t S = h->stream;
  const size_t blk = (size_t)nr * nc;
  std::vector<float> ffbuf;
  if (Cout && r > 0) {
    const double2* src = kind == 0 ? h->nearC.p + h->h_near_off[b]
                                   : h->farC.p + (size_t)b * h->rank_cap * blk;
    if (h->factors_ff) {
      ffbuf.resize(4 * blk * r);
      CQM_CUDA_TRY(cudaMemcpyAsync(ffbuf.data(), src, sizeof(double2) * blk * r, cudaMemcpyDeviceToHost, S));
    } else {
      CQM_CUDA_TRY(cudaMemcpyAsync(Cout, src, sizeof(double2) * blk * r, cudaMemcpyDeviceToHost, S));
    }
  }
  if (Dout && r > 0) {
    const double2* src = (kind == 0 ? h->nearD.p : h->farD.p) + (size_t)b * h->rank_cap * h->Ls;
    CQM_CUDA_TRY(cudaMemcpyAsync(Dout, src, sizeof(double2) * h->Ls * r, cudaMemcpyDeviceToHost, S));
  }
  CQM_CUDA_TRY(cudaStreamSynchronize(S));
  for (size_t i = 0; i < ffbuf.size() / 4; ++i) {  // float-float pairs -> hi + lo
    Cout[2 * i] = (double)ffbuf[4 * i] + (double)ffbuf[4 * i + 2];
    Cout[2 * i + 1] = (double)ffbuf[4 * i + 1] + (double)ffbuf[4 * i + 3];
  }
  return CQM_OK;
}

}  // extern "C"

namespace cqm {

ProfScope::ProfScope(cqm_handle* hh, int id) : h(hh) {
  if (!h || !h->prof_on) return;
  cudaEvent_t a, b;
  auto take = [&](cudaEvent_t& e) {
    if (!h->prof_pool.empty()) {
      e = h->prof_pool.back();
      h->prof_pool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
  };
  take(a);
  take(b);
  cudaEventRecord(a, h->stream);
  h->prof_recs.push_back({id, a, b});
  idx = (int)h->prof_recs.size() - 1;
}

ProfScope::~ProfScope() {
  if (idx >= 0) cudaEventRecord(h->prof_recs[idx].b, h->stream);
}

void prof_resolve(cqm_handle* h) {
  if (h->prof_recs.empty()) return;
  cudaEventSynchronize(h->prof_recs.back().b);
  for (auto& r : h->prof_recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    h->prof_launch[r.id] += 1;
    h->prof_ms[r.id] += ms;
    h->prof_pool.push_back(r.a);
    h->prof_pool.push_back(r.b);
  }
  h->prof_recs.clear();
}

void prof_release(cqm_handle* h) {
  prof_resolve(h);
  for (auto e : h->prof_pool) cudaEventDestroy(e);
  h->prof_pool.clear();
}

}  // namespace cqm

extern "C" {

static const char* k_names[CQM_K_COUNT] = {
    "geometry", "tree", "partition", "bases", "dense_assemble", "entries", "maca_slice",
    "maca_pivot", "maca_fibre", "maca_finalize", "near_apply", "leaf_forward", "upsweep",
    "far_coupling", "downsweep", "leaf_backward", "dense_apply", "arnoldi", "gmres_other",
    "forward_dft", "inverse_dft", "rhs", "precond", "near_exact", "far_exact", "expand", "points", "mot_weights", "mot_history",
    "mot_step", "dl_setup", "dl_apply"};

const char* cqm_bem_kernel_name(int32_t id) {
  return (id >= 0 && id < CQM_K_COUNT) ? k_names[id] : "";
}

int cqm_bem_set_wait_limit(cqm_handle* h, int64_t ns, int32_t expire_next) {
  if (!h || ns < 0) return CQM_EINVAL;
  h->wait_limit_ns = ns == 0 ? 1000000000ull : (uint64_t)ns;
  h->wait_probe = expire_next != 0;
  return CQM_OK;
}

int cqm_bem_profile(cqm_handle* h, int32_t enable) {
  if (!h) return CQM_EINVAL;
  prof_resolve(h);
  for (int k = 0; k < CQM_K_COUNT; ++k) {
    h->prof_launch[k] = 0;
    h->prof_ms[k] = 0.0;
  }
  h->prof_on = enable != 0;
  return CQM_OK;
}

int cqm_bem_profile_read(cqm_handle* h, int32_t n, int64_t* launches, double* total_ms) {
  if (!h || n < 0 || (n > 0 && (!launches || !total_ms))) return CQM_EINVAL;
  prof_resolve(h);
  for (int k = 0; k < n; ++k) {
    launches[k] = k < CQM_K_COUNT ? h->prof_launch[k] : 0;
    total_ms[k] = k < CQM_K_COUNT ? h->prof_ms[k] : 0.0;
  }
  return CQM_OK;
}

}  // extern "C"
