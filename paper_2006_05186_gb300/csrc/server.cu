// Serving many scattering problems on one GPU: a request queue, worker
// threads with one CUDA stream each, and admission by estimated device
// footprint.  Every frequency of the decoupled solve is independent (Remark in
// Sec. 6.2) and so is every request; the workers run the ordinary setup
// (Alg. 3) and solve of each request on their own stream, so that kernels of
// different requests overlap on the device while each request computes
// exactly what it would alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "handle.cuh"

namespace cqm {

using Clock = std::chrono::steady_clock;

static double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  int64_t ticket = 0;
  std::vector<double> xyz;
  std::vector<int32_t> tri;
  int32_t nv = 0, nt = 0;
  double dt = 0.0;
  int32_t N = 0, bdf = 2;
  cqm_params params{};
  std::vector<double> rhs;  // (N+1) x nt, or empty: plane-wave pulse
  double dir[3] = {0, 0, 1};
  double width = 0.5, delay = 0.0;
  int64_t bytes = 0;  // reserved at admission
  // result
  bool done = false;
  std::vector<double> density;
  cqm_result_info info{};
  Clock::time_point t_submit, t_admit;
};

}  // namespace cqm

struct cqm_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<cqm::Request>> queue;
  std::unordered_map<int64_t, std::shared_ptr<cqm::Request>> requests;
  int64_t next_ticket = 1;
  int64_t budget = 0, in_use = 0;
  int running = 0;
  bool stop = false;
  int device = 0;
  std::vector<std::thread> workers;
};

namespace cqm {

// Upper estimate of the device bytes of one request (see cqm_bem_estimate_bytes).
static int64_t estimate_bytes(int M, int N, const cqm_params& p, size_t total_dev) {
  const double L = N + 1, Ls = (double)(N + 1) / 2 + 1;
  const double cap = std::min(std::min(p.rank_cap, 64), (int)Ls);
  const double m = M;
  double b = 0.0;
  if (p.mode == CQM_MODE_DENSE) {
    b += Ls * m * m * 16.0;
  } else {
    const double ne = 1000.0 * m;   // near-field entries
    const double nf = 2.5 * m;      // far blocks
    const double nnb = ne / 256.0;  // near blocks
    const double nodes = m / 4.0, leaves = m / 8.0;
    b += cap * ne * 16.0 + nnb * cap * Ls * 16.0;                  // near C, D
    b += nf * cap * 4096.0 * 16.0 + nf * cap * Ls * 24.0;          // far C, D (+ FP32 D)
    b += p.tensor_cores == 1 ? nf * cap * 32768.0 : nf * cap * 4096.0 * 8.0;  // inner far factors
    if (!p.expand_near) b += cap * ne * 8.0 + nnb * cap * Ls * 8.0;  // FP32 near factors
    b += 1.2e6 * m + nf * 4096.0 * 16.0;                           // quadrature point caches
    b += leaves * 1024.0 * Ls * 16.0;                              // preconditioner
    b += (p.gmres_restart + 5.0) * Ls * m * 16.0;                  // GMRES workspace
    b += nodes * 64.0 * Ls * 48.0;                                 // H^2 transforms
    b += 2000.0 * 64.0 * Ls * 24.0;                                // partial tiles
    const double nearx = ne * Ls * 24.0, farx = nf * Ls * 4096.0 * 16.0;
    if (p.expand_near && nearx <= 0.25 * (double)total_dev) b += nearx;
    if (p.expand_far && p.exact_ff && farx <= 0.4 * (double)total_dev) b += farx;
  }
  b += 6.0 * L * m * 8.0 + 64.0 * 1024 * 1024;  // data, transforms, tables
  return (int64_t)b;
}

static bool fits(const cqm_server* s, const Request& r) { return s->in_use + r.bytes <= s->budget; }

static void run_request(cqm_server* s, Request& r, cudaStream_t stream, int worker) {
  r.info.worker = worker;
  r.info.bytes_estimate = r.bytes;
  cqm_mesh mesh{r.nv, r.xyz.data(), r.nt, r.tri.data()};
  cqm_handle* h = nullptr;
  const Clock::time_point t0 = Clock::now();
  int st = cqm_bem_setup(&mesh, r.dt, r.N, r.bdf, &r.params, stream, &h);
  const Clock::time_point t1 = Clock::now();
  r.info.t_setup_ms = ms_between(t0, t1);
  if (st == CQM_OK) {
    r.info.device_bytes = h->info.device_bytes;
    const size_t n = (size_t)(r.N + 1) * r.nt;
    if (r.rhs.empty()) {
      r.rhs.resize(n);
      st = cqm_bem_rhs_plane_wave(h, r.dir, r.width, r.delay, r.rhs.data(), CQM_MEM_HOST);
    }
    if (st == CQM_OK) {
      r.density.assign(n, 0.0);
      st = cqm_bem_solve(h, r.rhs.data(), r.density.data(), CQM_MEM_HOST, &r.info.solve);
    }
  }
  r.info.t_solve_ms = ms_between(t1, Clock::now());
  cqm_bem_destroy(h);
  r.info.status = st;
  (void)s;
}

static void worker_main(cqm_server* s, int worker) {
  cudaSetDevice(s->device);
  cudaStream_t stream = nullptr;
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) stream = nullptr;
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      for (;;) {
        if (s->stop && s->queue.empty()) break;
        auto it = std::find_if(s->queue.begin(), s->queue.end(),
                               [&](const std::shared_ptr<Request>& q) { return fits(s, *q); });
        if (it != s->queue.end()) {
          r = *it;
          s->queue.erase(it);
          s->in_use += r->bytes;
          ++s->running;
          break;
        }
        s->cv_work.wait(lock);
      }
      if (!r) break;
    }
    r->t_admit = Clock::now();
    run_request(s, *r, stream, worker);
    {
      std::lock_guard<std::mutex> lock(s->mu);
      s->in_use -= r->bytes;
      --s->running;
      r->info.t_queue_ms = ms_between(r->t_submit, r->t_admit);
      r->info.t_total_ms = ms_between(r->t_submit, Clock::now());
      r->done = true;
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
  if (stream) {
    cudaStreamSynchronize(stream);
    cudaStreamDestroy(stream);
  }
}

}  // namespace cqm

using namespace cqm;

extern "C" {

int cqm_bem_estimate_bytes(int32_t nt, int32_t N, const cqm_params* params, int64_t* bytes) {
  if (nt < 1 || N < 1 || N > CQM_MAX_STEPS || !bytes) return CQM_EINVAL;
  cqm_params p;
  if (params) p = *params;
  else cqm_params_default(&p);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    total_b = (size_t)1 << 40;
  }
  *bytes = estimate_bytes(nt, N, p, total_b);
  return CQM_OK;
}

int cqm_server_create(int32_t workers, int64_t byte_budget, cqm_server** out) {
  if (!out || workers < 1 || workers > 256 || byte_budget < 0) return CQM_EINVAL;
  *out = nullptr;
  cqm_server* s = new cqm_server();
  CQM_CUDA_TRY(cudaGetDevice(&s->device));
  size_t free_b = 0, total_b = 0;
  CQM_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  s->budget = byte_budget > 0 ? byte_budget : (int64_t)(0.9 * (double)free_b);
  // keep freed blocks in the stream-ordered pool between requests
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  for (int w = 0; w < workers; ++w) s->workers.emplace_back(worker_main, s, w);
  *out = s;
  return CQM_OK;
}

int cqm_bem_submit(cqm_server* s, const cqm_request* req, int64_t* ticket) {
  if (!s || !req || !ticket) return CQM_EINVAL;
  const cqm_mesh& m = req->mesh;
  if (!m.xyz || !m.tri || m.nt < 1 || m.nv < 3 || !(req->dt > 0.0) || req->N < 1 ||
      req->N > CQM_MAX_STEPS || (req->bdf_order != 1 && req->bdf_order != 2)) {
    set_last_error("request: bad mesh, dt, N or bdf_order");
    return CQM_EINVAL;
  }
  for (int64_t k = 0; k < 3 * (int64_t)m.nt; ++k)
    if (m.tri[k] < 0 || m.tri[k] >= m.nv) {
      set_last_error("request: triangle vertex index out of range");
      return CQM_EINVAL;
    }
  auto r = std::make_shared<Request>();
  r->nv = m.nv;
  r->nt = m.nt;
  r->xyz.assign(m.xyz, m.xyz + 3 * (size_t)m.nv);
  r->tri.assign(m.tri, m.tri + 3 * (size_t)m.nt);
  r->dt = req->dt;
  r->N = req->N;
  r->bdf = req->bdf_order;
  if (req->params) {
    r->params = *req->params;
  } else {
    cqm_params_default(&r->params);
    r->params.expand_far = 0;
  }
  r->params.allocator = nullptr;
  r->params.profile = 0;
  if (req->rhs) r->rhs.assign(req->rhs, req->rhs + (size_t)(req->N + 1) * m.nt);
  std::memcpy(r->dir, req->dir, sizeof(r->dir));
  r->width = req->width;
  r->delay = req->delay;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    total_b = (size_t)s->budget;
  }
  r->bytes = estimate_bytes(m.nt, req->N, r->params, total_b);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (r->bytes > s->budget) {
      set_last_error("request needs an estimated " + std::to_string(r->bytes) +
                     " bytes of device memory, more than the server's budget of " +
                     std::to_string(s->budget));
      return CQM_ENOMEM;
    }
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    s->queue.push_back(r);
    s->requests[r->ticket] = r;
    *ticket = r->ticket;
  }
  s->cv_work.notify_all();
  return CQM_OK;
}

int cqm_bem_poll(cqm_server* s, int64_t ticket, int32_t wait, double* density, cqm_result_info* info) {
  if (!s) return CQM_EINVAL;
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->requests.find(ticket);
    if (it == s->requests.end()) {
      set_last_error("unknown ticket " + std::to_string(ticket));
      return CQM_EINVAL;
    }
    r = it->second;
    if (!r->done) {
      if (!wait) return CQM_EPENDING;
      s->cv_done.wait(lock, [&] { return r->done; });
    }
    s->requests.erase(ticket);
  }
  if (density && !r->density.empty()) std::memcpy(density, r->density.data(), r->density.size() * sizeof(double));
  if (info) *info = r->info;
  return r->info.status;
}

int cqm_server_load(cqm_server* s, int64_t* bytes_in_use, int32_t* queued, int32_t* running) {
  if (!s) return CQM_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (bytes_in_use) *bytes_in_use = s->in_use;
  if (queued) *queued = (int32_t)s->queue.size();
  if (running) *running = s->running;
  return CQM_OK;
}

int cqm_server_destroy(cqm_server* s) {
  if (!s) return CQM_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
  return CQM_OK;
}

}  // extern "C"
