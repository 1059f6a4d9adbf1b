// Cluster tree (Def. 2) and block partition (Defs. 3-4, eq. qadm).
//
// Tree: one CTA, level-synchronous, one warp per node of the current level.
// A node's box is the tight box of its triangles' vertices; a node with more
// than n_min triangles splits along the longest box side (ties: x, y, z) at
// the midpoint (lo + hi) * 0.5, a triangle going left iff its centroid
// coordinate is below the midpoint; if a side would be empty the first
// floor(n/2) triangles in (centroid coordinate, index) order go left.  Both
// sons keep the parent's order.  Nodes are numbered breadth-first.
//
// Partition: one CTA walks the block tree level by level (Def. 3): a pair is
// admissible iff dist > 0 and max(diam_r, diam_c) <= eta * dist on boxes
// (eq. qadm; diam = box diagonal, dist = box distance, sums of squares formed
// as ((x^2 + y^2) + z^2) without contraction); admissible pairs are far
// blocks, inadmissible leaf pairs near blocks, the rest split into sons
// (sons(r) x c, r x sons(c) or sons(r) x sons(c)).  The lists are then sorted
// by (row, column).
#include <algorithm>
#include <vector>

#include "handle.cuh"

namespace cqm {

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_isum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct TreeOut {
  int* perm;
  int* tmp;
  int* begin;
  int* end;
  int* son0;
  int* son1;
  int* parent;
  int* level;
  double* lo;
  double* hi;
  int* split;  // per node: number of left triangles (0 = leaf)
  int* counters;  // [0] n_nodes, [1] depth
};

__global__ void __launch_bounds__(1024) k_build_tree(int M, int n_min, int cap,
                                                     const double* __restrict__ xyz,
                                                     const int* __restrict__ tri,
                                                     const double* __restrict__ cen, TreeOut T) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  __shared__ int s_level_begin, s_level_end, s_n_nodes, s_depth;
  for (int i = threadIdx.x; i < M; i += blockDim.x) T.perm[i] = i;
  if (threadIdx.x == 0) {
    T.begin[0] = 0;
    T.end[0] = M;
    T.parent[0] = -1;
    T.level[0] = 0;
    s_level_begin = 0;
    s_level_end = 1;
    s_n_nodes = 1;
    s_depth = 0;
  }
  __syncthreads();
  while (s_level_begin < s_level_end) {
    const int lb = s_level_begin, le = s_level_end;
    for (int node = lb + warp; node < le; node += nwarps) {
      const int b = T.begin[node], e = T.end[node], n = e - b;
      double lo0 = 1e300, lo1 = 1e300, lo2 = 1e300, hi0 = -1e300, hi1 = -1e300, hi2 = -1e300;
      for (int k = b + lane; k < e; k += 32) {
        const int t = T.perm[k];
        for (int v = 0; v < 3; ++v) {
          const double* p = xyz + 3 * tri[3 * t + v];
          lo0 = fmin(lo0, p[0]); lo1 = fmin(lo1, p[1]); lo2 = fmin(lo2, p[2]);
          hi0 = fmax(hi0, p[0]); hi1 = fmax(hi1, p[1]); hi2 = fmax(hi2, p[2]);
        }
      }
      lo0 = warp_min(lo0); lo1 = warp_min(lo1); lo2 = warp_min(lo2);
      hi0 = warp_max(hi0); hi1 = warp_max(hi1); hi2 = warp_max(hi2);
      if (lane == 0) {
        T.lo[3 * node] = lo0; T.lo[3 * node + 1] = lo1; T.lo[3 * node + 2] = lo2;
        T.hi[3 * node] = hi0; T.hi[3 * node + 1] = hi1; T.hi[3 * node + 2] = hi2;
      }
      if (n <= n_min) {
        if (lane == 0) T.split[node] = 0;
        continue;
      }
      const double e0 = hi0 - lo0, e1 = hi1 - lo1, e2 = hi2 - lo2;
      int ax = 0;
      double best = e0;
      if (e1 > best) { ax = 1; best = e1; }
      if (e2 > best) { ax = 2; }
      const double mid = __dmul_rn(__dadd_rn(ax == 0 ? lo0 : (ax == 1 ? lo1 : lo2),
                                             ax == 0 ? hi0 : (ax == 1 ? hi1 : hi2)), 0.5);
      int nl = 0;
      for (int k = b + lane; k < e; k += 32) nl += (cen[3 * T.perm[k] + ax] < mid) ? 1 : 0;
      nl = warp_isum(nl);
      const bool median = (nl == 0 || nl == n);
      if (median) nl = n / 2;
      // stable partition into tmp[b..e)
      int offl = 0, offr = 0;
      for (int k0 = b; k0 < e; k0 += 32) {
        const int k = k0 + lane;
        bool left = false;
        int t = -1;
        if (k < e) {
          t = T.perm[k];
          const double c = cen[3 * t + ax];
          if (!median) {
            left = c < mid;
          } else {
            int rank = 0;
            for (int q = b; q < e; ++q) {
              const int u = T.perm[q];
              const double cu = cen[3 * u + ax];
              rank += (cu < c || (cu == c && u < t)) ? 1 : 0;
            }
            left = rank < nl;
          }
        }
        const unsigned bl = __ballot_sync(0xffffffffu, k < e && left);
        const unsigned br = __ballot_sync(0xffffffffu, k < e && !left);
        const unsigned lt = (1u << lane) - 1u;
        if (k < e) {
          if (left) T.tmp[b + offl + __popc(bl & lt)] = t;
          else T.tmp[b + nl + offr + __popc(br & lt)] = t;
        }
        offl += __popc(bl);
        offr += __popc(br);
      }
      __syncwarp();
      for (int k = b + lane; k < e; k += 32) T.perm[k] = T.tmp[k];
      if (lane == 0) T.split[node] = nl;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int nn = s_n_nodes;
      for (int node = lb; node < le; ++node) {
        const int nl = T.split[node];
        if (nl > 0 && nn + 2 <= cap) {
          const int b = T.begin[node], e = T.end[node];
          T.son0[node] = nn;
          T.son1[node] = nn + 1;
          T.begin[nn] = b; T.end[nn] = b + nl; T.parent[nn] = node; T.level[nn] = T.level[node] + 1;
          T.begin[nn + 1] = b + nl; T.end[nn + 1] = e; T.parent[nn + 1] = node;
          T.level[nn + 1] = T.level[node] + 1;
          nn += 2;
        } else {
          T.son0[node] = -1;
          T.son1[node] = -1;
        }
      }
      s_level_begin = le;
      s_level_end = nn;
      if (nn > le) s_depth = T.level[le];
      s_n_nodes = nn;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    T.counters[0] = s_n_nodes;
    T.counters[1] = s_depth;
  }
}

int build_tree(cqm_handle* h) {
  const int M = h->M;
  const int cap = 2 * M + 1;
  CQM_TRY(h->perm.allocate(h->alloc, M));
  CQM_TRY(h->node_begin.allocate(h->alloc, cap));
  CQM_TRY(h->node_end.allocate(h->alloc, cap));
  CQM_TRY(h->node_son0.allocate(h->alloc, cap));
  CQM_TRY(h->node_son1.allocate(h->alloc, cap));
  CQM_TRY(h->node_parent.allocate(h->alloc, cap));
  CQM_TRY(h->node_level.allocate(h->alloc, cap));
  CQM_TRY(h->node_lo.allocate(h->alloc, 3 * (size_t)cap));
  CQM_TRY(h->node_hi.allocate(h->alloc, 3 * (size_t)cap));
  DArray<int> tmp, split, counters;
  int st = CQM_OK;
  if ((st = tmp.allocate(h->alloc, M)) == CQM_OK && (st = split.allocate(h->alloc, cap)) == CQM_OK &&
      (st = counters.allocate(h->alloc, 4)) == CQM_OK) {
    TreeOut T{h->perm.p, tmp.p, h->node_begin.p, h->node_end.p, h->node_son0.p,
              h->node_son1.p, h->node_parent.p, h->node_level.p, h->node_lo.p, h->node_hi.p,
              split.p, counters.p};
    {
      ProfScope ps_(h, CQM_K_TREE);
      k_build_tree<<<1, 1024, 0, h->stream>>>(M, h->params.n_min, cap, h->xyz.p, h->tri.p, h->cen.p, T);
    }
    cudaError_t e = cudaGetLastError();
    int hc[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc, counters.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      set_last_error(std::string("build_tree: ") + cudaGetErrorString(e));
      st = CQM_ECUDA;
    } else {
      h->n_nodes = hc[0];
      h->depth = hc[1];
    }
  }
  tmp.free(h->alloc);
  split.free(h->alloc);
  counters.free(h->alloc);
  if (st != CQM_OK) return st;
  const int n = h->n_nodes;
  h->h_begin.resize(n); h->h_end.resize(n); h->h_son0.resize(n); h->h_son1.resize(n); h->h_level.resize(n);
  CQM_CUDA_TRY(cudaMemcpyAsync(h->h_begin.data(), h->node_begin.p, n * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaMemcpyAsync(h->h_end.data(), h->node_end.p, n * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaMemcpyAsync(h->h_son0.data(), h->node_son0.p, n * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaMemcpyAsync(h->h_son1.data(), h->node_son1.p, n * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaMemcpyAsync(h->h_level.data(), h->node_level.p, n * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->n_leaves = 0;
  for (int r = 0; r < n; ++r) h->n_leaves += h->h_son0[r] < 0;
  h->level_begin.assign(h->depth + 2, n);
  for (int r = n - 1; r >= 0; --r) h->level_begin[h->h_level[r]] = r;
  h->level_begin[h->depth + 1] = n;
  for (int lv = h->depth; lv >= 0; --lv)
    if (h->level_begin[lv] > h->level_begin[lv + 1]) h->level_begin[lv] = h->level_begin[lv + 1];
  return CQM_OK;
}

// ------------------------------------------------------------- partition ----

__device__ __forceinline__ bool admissible(const double* lo, const double* hi, int r, int c,
                                           double eta) {
  const double* lr = lo + 3 * r;
  const double* hr = hi + 3 * r;
  const double* lc = lo + 3 * c;
  const double* hc = hi + 3 * c;
  const double dr = exact_len(__dsub_rn(hr[0], lr[0]), __dsub_rn(hr[1], lr[1]), __dsub_rn(hr[2], lr[2]));
  const double dc = exact_len(__dsub_rn(hc[0], lc[0]), __dsub_rn(hc[1], lc[1]), __dsub_rn(hc[2], lc[2]));
  double g[3];
  for (int d = 0; d < 3; ++d)
    g[d] = fmax(fmax(__dsub_rn(lc[d], hr[d]), __dsub_rn(lr[d], hc[d])), 0.0);
  const double dist = exact_len(g[0], g[1], g[2]);
  return dist > 0.0 && fmax(dr, dc) <= __dmul_rn(eta, dist);
}

// Block-wide exclusive scan of one int per thread (blockDim.x == 1024).
__device__ __forceinline__ int block_exscan(int v, int* sh, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = sh[lane];
    int z = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    sh[lane] = z - w;
    if (lane == 31) sh[32] = z;
  }
  __syncthreads();
  const int r = sh[warp] + x - v;
  *total = sh[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(1024) k_partition(const double* __restrict__ lo,
                                                    const double* __restrict__ hi,
                                                    const int* __restrict__ son0,
                                                    const int* __restrict__ son1, double eta,
                                                    int2* fa, int2* fb, int fcap, int2* near,
                                                    int ncap, int2* far, int farcap, int* counters) {
  __shared__ int sh[33];
  __shared__ int s_nf, s_nn, s_nfar, s_over;
  if (threadIdx.x == 0) {
    fa[0] = make_int2(0, 0);
    s_nf = 1;
    s_nn = 0;
    s_nfar = 0;
    s_over = 0;
  }
  __syncthreads();
  int2* cur = fa;
  int2* nxt = fb;
  while (s_nf > 0) {
    const int nf = s_nf;
    int next = 0;
    for (int base = 0; base < nf; base += blockDim.x) {
      const int k = base + threadIdx.x;
      int cfar = 0, cnear = 0, ckid = 0;
      int2 rc = make_int2(0, 0);
      bool rl = false, cl = false;
      if (k < nf) {
        rc = cur[k];
        rl = son0[rc.x] < 0;
        cl = son0[rc.y] < 0;
        if (admissible(lo, hi, rc.x, rc.y, eta)) cfar = 1;
        else if (rl && cl) cnear = 1;
        else ckid = (rl || cl) ? 2 : 4;
      }
      int tf, tn, tk;
      const int pf = block_exscan(cfar, sh, &tf);
      const int pn = block_exscan(cnear, sh, &tn);
      const int pk = block_exscan(ckid, sh, &tk);
      if (cfar && s_nfar + pf < farcap) far[s_nfar + pf] = rc;
      if (cnear && s_nn + pn < ncap) near[s_nn + pn] = rc;
      if (ckid) {
        int2 kids[4];
        int nk = 0;
        if (rl) { kids[nk++] = make_int2(rc.x, son0[rc.y]); kids[nk++] = make_int2(rc.x, son1[rc.y]); }
        else if (cl) { kids[nk++] = make_int2(son0[rc.x], rc.y); kids[nk++] = make_int2(son1[rc.x], rc.y); }
        else {
          kids[nk++] = make_int2(son0[rc.x], son0[rc.y]); kids[nk++] = make_int2(son0[rc.x], son1[rc.y]);
          kids[nk++] = make_int2(son1[rc.x], son0[rc.y]); kids[nk++] = make_int2(son1[rc.x], son1[rc.y]);
        }
        for (int q = 0; q < nk; ++q)
          if (next + pk + q < fcap) nxt[next + pk + q] = kids[q];
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        s_nfar += tf;
        s_nn += tn;
        if (s_nfar > farcap || s_nn > ncap || next + tk > fcap) s_over = 1;
      }
      next += tk;
      __syncthreads();
    }
    if (threadIdx.x == 0) s_nf = (next <= fcap && !s_over) ? next : 0;
    __syncthreads();
    int2* t = cur;
    cur = nxt;
    nxt = t;
  }
  if (threadIdx.x == 0) {
    counters[0] = s_nn;
    counters[1] = s_nfar;
    counters[2] = s_over;
  }
}

// Sort a block list by (row, column): count rows, scan, scatter, per-row sort.
__global__ void k_count_rows(int n, const int2* __restrict__ in, int* cnt) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) atomicAdd(&cnt[in[k].x], 1);
}
__global__ void __launch_bounds__(1024) k_scan_rows(int nrows, const int* cnt, int* rowptr, int* cursor) {
  __shared__ int sh[33];
  int carry = 0;
  for (int base = 0; base < nrows; base += blockDim.x) {
    int k = base + threadIdx.x;
    int v = k < nrows ? cnt[k] : 0;
    int tot;
    int x = block_exscan(v, sh, &tot);
    if (k < nrows) { rowptr[k] = carry + x; cursor[k] = carry + x; }
    carry += tot;
  }
  if (threadIdx.x == 0) rowptr[nrows] = carry;
}
__global__ void k_scatter_rows(int n, const int2* __restrict__ in, int* cursor, int2* out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    int2 v = in[k];
    out[atomicAdd(&cursor[v.x], 1)] = v;
  }
}
__global__ void k_sort_rows(int nrows, const int* __restrict__ rowptr, int2* a) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  for (int i = rowptr[r] + 1; i < rowptr[r + 1]; ++i) {
    int2 v = a[i];
    int j = i - 1;
    while (j >= rowptr[r] && a[j].y > v.y) {
      a[j + 1] = a[j];
      --j;
    }
    a[j + 1] = v;
  }
}

static int sort_blocks(cqm_handle* h, int n, int2* raw, DArray<int2>& out, DArray<int>& rowptr) {
  const int nr = h->n_nodes;
  CQM_TRY(out.allocate(h->alloc, std::max(n, 1)));
  CQM_TRY(rowptr.allocate(h->alloc, nr + 1));
  DArray<int> cnt, cursor;
  int st = cnt.allocate(h->alloc, nr);
  if (st == CQM_OK) st = cursor.allocate(h->alloc, nr);
  if (st == CQM_OK) {
    cudaMemsetAsync(cnt.p, 0, sizeof(int) * nr, h->stream);
    if (n > 0) {
      ProfScope ps_(h, CQM_K_PARTITION);
      k_count_rows<<<grid_for(n, 256), 256, 0, h->stream>>>(n, raw, cnt.p);
    }
    {
      ProfScope ps_(h, CQM_K_PARTITION);
      k_scan_rows<<<1, 1024, 0, h->stream>>>(nr, cnt.p, rowptr.p, cursor.p);
    }
    if (n > 0) {
      ProfScope ps_(h, CQM_K_PARTITION);
      k_scatter_rows<<<grid_for(n, 256), 256, 0, h->stream>>>(n, raw, cursor.p, out.p);
    }
    {
      ProfScope ps_(h, CQM_K_PARTITION);
      k_sort_rows<<<grid_for(nr, 128), 128, 0, h->stream>>>(nr, rowptr.p, out.p);
    }
    if (cudaGetLastError() != cudaSuccess) st = CQM_ECUDA;
  }
  cnt.free(h->alloc);
  cursor.free(h->alloc);
  if (st == CQM_ECUDA) set_last_error("sort_blocks launch failed");
  return st;
}

int build_partition(cqm_handle* h) {
  int fcap = std::max(1024, 64 * h->n_nodes), ncap = fcap, farcap = fcap;
  for (int attempt = 0; attempt < 6; ++attempt) {
    DArray<int2> fa, fb, near, far;
    DArray<int> counters;
    int st = fa.allocate(h->alloc, fcap);
    if (st == CQM_OK) st = fb.allocate(h->alloc, fcap);
    if (st == CQM_OK) st = near.allocate(h->alloc, ncap);
    if (st == CQM_OK) st = far.allocate(h->alloc, farcap);
    if (st == CQM_OK) st = counters.allocate(h->alloc, 4);
    int hc[3] = {0, 0, 0};
    if (st == CQM_OK) {
      {
        ProfScope ps_(h, CQM_K_PARTITION);
        k_partition<<<1, 1024, 0, h->stream>>>(h->node_lo.p, h->node_hi.p, h->node_son0.p,
                                               h->node_son1.p, h->params.eta, fa.p, fb.p, fcap,
                                               near.p, ncap, far.p, farcap, counters.p);
      }
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaMemcpyAsync(hc, counters.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) {
        set_last_error(std::string("partition: ") + cudaGetErrorString(e));
        st = CQM_ECUDA;
      }
    }
    if (st == CQM_OK && !hc[2]) {
      h->n_near = hc[0];
      h->n_far = hc[1];
      st = sort_blocks(h, h->n_near, near.p, h->near_rc, h->near_rowptr);
      if (st == CQM_OK) st = sort_blocks(h, h->n_far, far.p, h->far_rc, h->far_rowptr);
      if (st == CQM_OK) {
        h->h_near.resize(h->n_near);
        h->h_far.resize(h->n_far);
        cudaMemcpyAsync(h->h_near.data(), h->near_rc.p, sizeof(int2) * h->n_near, cudaMemcpyDeviceToHost, h->stream);
        cudaMemcpyAsync(h->h_far.data(), h->far_rc.p, sizeof(int2) * h->n_far, cudaMemcpyDeviceToHost, h->stream);
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) st = CQM_ECUDA;
      }
    }
    fa.free(h->alloc); fb.free(h->alloc); near.free(h->alloc); far.free(h->alloc);
    counters.free(h->alloc);
    if (st != CQM_OK) return st;
    if (!hc[2]) return CQM_OK;
    fcap *= 4; ncap *= 4; farcap *= 4;
  }
  set_last_error("block partition exceeded its list capacity");
  return CQM_ECAPACITY;
}

}  // namespace cqm

namespace cqm {

// The tree kernel on buffers the caller provides (scratch included); used by
// the entry point that allocates no device memory.
int launch_tree_kernel(int M, int n_min, int cap, const double* xyz, const int* tri,
                       const double* cen, int* perm, int* tmp, int* begin, int* end, int* son0,
                       int* son1, int* parent, int* level, double* lo, double* hi, int* split,
                       int* counters, cudaStream_t stream) {
  TreeOut T{perm, tmp, begin, end, son0, son1, parent, level, lo, hi, split, counters};
  k_build_tree<<<1, 1024, 0, stream>>>(M, n_min, cap, xyz, tri, cen, T);
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

}  // namespace cqm
