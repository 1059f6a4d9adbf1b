// Far-field coupling of the inner operator on the tcgen05 tensor cores, with
// the frequencies on the MMA's M dimension (eq. lrfinal for all frequencies):
//
//   yhat_r[mu][l] += sum_{b=(r,c)} sum_t d_{b,t}[l] Z_{b,t}[mu][l],
//   Z_{b,t} = C_{b,t} xhat_c  (64 x 64 times 64 x Ls, complex).
//
// Z does not depend on d_t, so the operand xhat_c is formed once per block
// and the rank terms of the block stream past it; d_t[l] scales row l of Z^T,
// which is one value per TMEM lane, in the epilogue.  In real arithmetic, with
// A = [Re xhat_c^T | Im xhat_c^T] (128 frequencies x K = 128) and
// B = [Re C_t | Im C_t] (64 rows x K = 128):
//   Re Z^T = A[:, :64] Re C^T - A[:, 64:] Im C^T   (B's second K half negated),
//   Im Z^T = A[:, :64] Im C^T + A[:, 64:] Re C^T   (B's K halves swapped).
// Two consecutive rank terms t, t + 1 of a block share A, so their B operands
// are stacked into one of N = 128 rows: per pair of terms, two GEMMs of
// M = 128, N = 128, K = 128 (the tensor pipe takes about as long for an MMA of
// N = 64 as for one of N = 128).  The last term of a block of odd rank runs
// alone with N = 64.  Operands are split as hi + lo in bf16 and the products
// hi*hi + hi*lo + lo*hi are accumulated in fp32 (about 2^-17 per product; the
// inner operator only steers GMRES, whose restarts recompute the residual in
// float-float).  The trailing terms of a block that stay below a set fraction
// of the largest far term at every frequency (k_tc2_single_from) take the
// hi*hi product alone, and their lo planes are not copied: a single bf16
// product rounds such a term to ~2^-8 of itself, below the other errors.
//
// Layout and roles (one CTA per work item: a row cluster and a run of its far
// blocks; 1 CTA per SM, which owns the 512 TMEM columns):
//   TMEM columns [0, 256): A, two buffers of 128 (bf16 hi 64 + lo 64; lane l
//     holds frequency l0 + l, two bf16 per column, lower K in the low half);
//   TMEM columns [256, 512): accumulators, slot 0 for Re Z^T and slot 1 for
//     Im Z^T of one pair (128 columns each: mu of term t, then mu of t + 1).
//   shared memory: a ring of NSTAGE stages of 64 KB, [hi t | hi t+1 | lo t |
//     lo t+1], each plane (16 KB) bulk-copied from the term's precomputed
//     32 KB image in HBM (warp 13); a plane is 64 rows x 128 bf16 of
//     [Re C_t | Im C_t] in the canonical K-major layout without swizzle (core
//     matrices of 8 rows x 16 bytes, K-adjacent ones 128 bytes apart, 8-row
//     groups 2048 bytes apart), so the two hi (lo) planes of a stage are one
//     operand of 128 rows.
//   warps 8-11 build A for each block from xhat_c (one lane per frequency);
//   warp 12 (one thread) issues 24 MMAs (8 for a single-product pair) into
//     slot 0 and as many into slot 1 per pair and frees each B stage,
//     accumulator slot and A buffer with tcgen05.commit;
//   warps 0-7 (two per TMEM lane quadrant, 32 mu each) read each slot (one
//     lane per frequency), multiply by d_t[l] and d_{t+1}[l] (loaded two pairs
//     ahead) and keep the row's sum over all terms in registers, then write
//     the item's partial tile, which the per-row reduction adds in item order.
//     CTA k takes the items at launch positions k, k + grid, ... (launched with
//     one CTA per item, the hardware schedules the items as SMs free up); the
//     launch order puts the largest items first, so that the small ones fill
//     the end of the schedule.
// Frequencies go in chunks of 128 lanes (the last one padded); when Ls mod 128
// is 1 to TAIL_MAX the remaining frequencies are applied from an FP32 table of
// the expanded couplings S_b(l) = sum_t d_t[l] C_t instead (k_far_tail_f32).
// Every wait of the main loop has the handle's time limit; on expiry the kernel
// records it, stops issuing work, lets issued copies and MMAs drain, frees its
// tensor memory and returns (the drain waits keep the one-second default).
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "handle.cuh"
#include "umma.cuh"

namespace cqm {

namespace {
constexpr int TP = 64;                 // Chebyshev points per cluster (m = 4)
constexpr int NSTAGE = 3;              // B stages
constexpr uint32_t BIMG = 32768;       // bytes of one term's B image in HBM (hi + lo planes)
constexpr uint32_t BPLANE = 16384;     // one plane: 64 rows x 128 bf16
constexpr uint32_t BSTAGE = 65536;     // one stage: the planes of a pair of terms
constexpr uint32_t B_SBO = 2048;       // 8-row groups
constexpr uint32_t B_LBO = 128;        // K-adjacent core matrices
constexpr int NTHREADS = 448;          // warps 0-7 epilogue, 8-11 A, 12 MMA, 13 loader
constexpr int W_A0 = 8, W_MMA = 12, W_LOAD = 13;
constexpr int NEPI = 8;                // epilogue warps: two per TMEM lane quadrant
constexpr int MUE = TP / 2;            // mu columns per epilogue warp
constexpr uint32_t TCOLS = 512;
constexpr uint32_t ACC0 = 256;         // first accumulator column
constexpr int ERR_TIMEOUT = 1;
constexpr size_t SMEM = (size_t)NSTAGE * BSTAGE + 1024;
}  // namespace

constexpr int TC2_TAIL_MAX = 4;

// Byte offset of element (row, k) in one plane of a B image.
__host__ __device__ constexpr uint32_t bimg_off(int row, int k) {
  return (uint32_t)((row >> 3) * B_SBO + (k >> 3) * B_LBO + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void split_bf16(float x, uint16_t& hi, uint16_t& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  hi = __bfloat16_as_ushort(h);
  lo = __bfloat16_as_ushort(l);
}

// B images of every rank term: image (b, t) at (first[b] + t) * BIMG bytes,
// element (mu, k) = Re C_t[mu][k] (k < 64) or Im C_t[mu][k - 64], split into
// the hi and lo planes.  One block per (term slot, block) on a one-dimensional
// grid of nt slots per block.
__global__ void __launch_bounds__(256) k_tc2_images(int cap, int nt, const int* __restrict__ rank,
                                                    const int64_t* __restrict__ first,
                                                    const double2* __restrict__ C,
                                                    unsigned char* __restrict__ img) {
  const int b = (int)(blockIdx.x / nt), t = (int)(blockIdx.x - (unsigned)b * nt);
  if (t >= rank[b]) return;
  const double2* Ct = C + ((size_t)b * cap + t) * TP * TP;
  unsigned char* dst = img + (size_t)(first[b] + t) * BIMG;
  for (int e = threadIdx.x; e < TP * 128; e += blockDim.x) {
    const int mu = e >> 7, k = e & 127;
    const double2 c = Ct[mu * TP + (k & 63)];
    uint16_t hi, lo;
    split_bf16((float)(k < 64 ? c.x : c.y), hi, lo);
    const uint32_t o = bimg_off(mu, k);
    *(uint16_t*)(dst + o) = hi;
    *(uint16_t*)(dst + BPLANE + o) = lo;
  }
}

// Sizes of the far rank terms for the choice of their product count:
// n_t(l) = ||C_t||_F |d_t(l)| is the size of term t of block b at frequency l.
// One CTA per block writes ||C_t||_F and raises ref[l] to the largest n_t(l)
// of the block (ref holds the bits of non-negative floats, which order as
// integers).
__global__ void __launch_bounds__(256) k_tc2_term_sizes(int Ls, int cap, const int* __restrict__ rank,
                                                        const double2* __restrict__ C,
                                                        const double2* __restrict__ D, float* __restrict__ cn,
                                                        unsigned int* __restrict__ ref) {
  __shared__ float cs[64];
  __shared__ double red[8];
  const int b = blockIdx.x, rk = rank[b];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = 0; t < rk; ++t) {
    const double2* Ct = C + ((size_t)b * cap + t) * TP * TP;
    double a = 0.0;
    for (int e = threadIdx.x; e < TP * TP; e += blockDim.x) a += Ct[e].x * Ct[e].x + Ct[e].y * Ct[e].y;
    for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[w] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int v = 0; v < 8; ++v) tot += red[v];
      cs[t] = (float)sqrt(tot);
      cn[(size_t)b * cap + t] = cs[t];
    }
    __syncthreads();
  }
  for (int l = threadIdx.x; l < Ls; l += blockDim.x) {
    float mx = 0.f;
    for (int t = 0; t < rk; ++t) {
      const double2 d = D[((size_t)b * cap + t) * Ls + l];
      mx = fmaxf(mx, cs[t] * (float)hypot(d.x, d.y));
    }
    atomicMax(&ref[l], __float_as_uint(mx));
  }
}

// First term of each far block from which its pairs take one product: the
// block's trailing terms with n_t(l) <= ratio * ref[l] at every frequency l,
// ref[l] the largest term of any far block at l (so the rounding of a single
// bf16 product, ~2^-8 of such a term, is measured against the far field's
// scale at that frequency).  t1[b] is the first such term, rounded up to the
// next pair (even t); rank[b] when none (or ratio = 0).  One CTA per block;
// *count gets the number of single-product terms.
__global__ void __launch_bounds__(256) k_tc2_single_from(int Ls, int cap, double ratio,
                                                         const int* __restrict__ rank,
                                                         const double2* __restrict__ D,
                                                         const float* __restrict__ cn,
                                                         const unsigned int* __restrict__ ref,
                                                         int* __restrict__ t1, int* __restrict__ count) {
  __shared__ unsigned int rho[64];
  const int b = blockIdx.x, rk = rank[b];
  for (int t = threadIdx.x; t < rk; t += blockDim.x) rho[t] = 0u;
  __syncthreads();
  for (int l = threadIdx.x; l < Ls; l += blockDim.x) {
    const float r = __uint_as_float(ref[l]);
    if (!(r > 0.f)) continue;
    for (int t = 0; t < rk; ++t) {
      const double2 d = D[((size_t)b * cap + t) * Ls + l];
      atomicMax(&rho[t], __float_as_uint(cn[(size_t)b * cap + t] * (float)hypot(d.x, d.y) / r));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int f = rk;
    if (ratio > 0.0)
      while (f > 0 && (double)__uint_as_float(rho[f - 1]) <= ratio) --f;
    f = min(rk, (f + 1) & ~1);
    t1[b] = f;
    if (rk > f) atomicAdd(count, rk - f);
  }
}

// Expanded couplings of the tail frequencies, nu-major:
// S[(b * ntail + f) * 4096 + nu * 64 + mu] = sum_t d_t[l0 + f] C_t[mu][nu]
// (FP32 from the FP64 factors).
__global__ void __launch_bounds__(256) k_tc2_tail_table(int Ls, int cap, int l0, int ntail,
                                                        const int* __restrict__ rank,
                                                        const double2* __restrict__ C,
                                                        const double2* __restrict__ D,
                                                        float2* __restrict__ S) {
  const int b = blockIdx.x;
  const int rk = rank[b];
  for (int e = threadIdx.x; e < TP * TP * ntail; e += blockDim.x) {
    const int f = e / (TP * TP), en = e - f * TP * TP;
    const int nu = en / TP, mu = en - nu * TP;
    double2 acc = make_double2(0.0, 0.0);
    for (int t = 0; t < rk; ++t)
      cfma(acc, C[((size_t)b * cap + t) * TP * TP + mu * TP + nu], D[((size_t)b * cap + t) * Ls + l0 + f]);
    S[((size_t)b * ntail + f) * TP * TP + en] = make_float2((float)acc.x, (float)acc.y);
  }
}

// Tail frequencies: yhat_r(l)[mu] += sum over the far blocks (r, c) of row r of
// sum_nu S_b(l)[mu][nu] xhat_c(l)[nu].  One CTA per (far row, tail
// frequency); warp w takes the row's blocks w, w + 8, ... (lane owns mu = lane
// and lane + 32, coalesced reads of the nu-major table); the warps' sums are
// added in warp order.
__global__ void __launch_bounds__(256) k_far_tail_f32(int Ls, int l0, int ntail,
                                                      const int* __restrict__ rows,
                                                      const int* __restrict__ rowptr,
                                                      const int2* __restrict__ rc,
                                                      const float2* __restrict__ S,
                                                      const float2* __restrict__ xhat,
                                                      float2* __restrict__ yhat,
                                                      const int* __restrict__ act) {
  __shared__ float2 red[8][TP];
  const int k = blockIdx.x / ntail, f = blockIdx.x - k * ntail, l = l0 + f;
  if (act && !act[l]) return;  // a converged frequency (act may be null)
  const int r = rows[k];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
  for (int bi = rowptr[r] + w; bi < rowptr[r + 1]; bi += 8) {
    const float2* xc = xhat + (size_t)rc[bi].y * TP * Ls + l;
    const float2 x0 = xc[(size_t)lane * Ls], x1 = xc[(size_t)(lane + 32) * Ls];
    const float2* Sb = S + ((size_t)bi * ntail + f) * TP * TP;
#pragma unroll 8
    for (int nu = 0; nu < TP; ++nu) {
      const float2 xv = make_float2(__shfl_sync(0xffffffffu, nu < 32 ? x0.x : x1.x, nu & 31),
                                    __shfl_sync(0xffffffffu, nu < 32 ? x0.y : x1.y, nu & 31));
      cfma(a0, Sb[nu * TP + lane], xv);
      cfma(a1, Sb[nu * TP + lane + 32], xv);
    }
  }
  red[w][lane] = a0;
  red[w][lane + 32] = a1;
  __syncthreads();
  if (w == 0) {
    float2 s0 = red[0][lane], s1 = red[0][lane + 32];
    for (int v = 1; v < 8; ++v) {
      s0 = cadd(s0, red[v][lane]);
      s1 = cadd(s1, red[v][lane + 32]);
    }
    float2* yr = yhat + (size_t)r * TP * Ls + l;
    yr[(size_t)lane * Ls] = cadd(yr[(size_t)lane * Ls], s0);
    yr[(size_t)(lane + 32) * Ls] = cadd(yr[(size_t)(lane + 32) * Ls], s1);
  }
}

// Position in the sequence (item, chunk, block, pair of terms t, t + 1) of
// one CTA: items blockIdx.x, blockIdx.x + gridDim.x, ...; blocks of rank 0
// skipped; done() once the items are exhausted.
struct Seq {
  int ii, ch, bi, t;
  int b0, b1;
  int n_items, stride, nch;
  const int4* items;
  const int* order;  // launch position -> item (largest items first)
  const int* rank;
  __device__ void start(const int4* items_, const int* order_, int n_items_, int nch_, const int* rank_) {
    items = items_; order = order_; n_items = n_items_; nch = nch_; rank = rank_;
    stride = gridDim.x;
    ii = blockIdx.x;
    t = 0;
    enter();
    skip();
  }
  __device__ void enter() {  // first block of item ii
    ch = 0;
    if (ii < n_items) {
      const int4 it = items[order[ii]];
      b0 = it.y;
      b1 = it.z;
    } else {
      b0 = b1 = 0;
    }
    bi = b0;
  }
  __device__ void skip() {
    while (ii < n_items) {
      while (ch < nch) {
        while (bi < b1 && rank[bi] == 0) ++bi;
        if (bi < b1) return;
        ++ch;
        bi = b0;
      }
      ii += stride;
      enter();
    }
  }
  __device__ bool done() const { return ii >= n_items; }
  // the unit holds terms t and t + 1 (false: t is a block's last, odd term)
  __device__ bool two() const { return t + 1 < rank[bi]; }
  // advance by one pair; returns true if the block (or chunk, or item) changed
  __device__ bool next() {
    t += 2;
    if (t < rank[bi]) return false;
    t = 0;
    ++bi;
    skip();
    return true;
  }
  __device__ bool same_block(const Seq& o) const { return ii == o.ii && ch == o.ch && bi == o.bi; }
};

// d_{t+j}[l] (j = 0, 1) of the pair at q for this lane's frequency of q's
// chunk (0 past the end and for the missing second term)
__device__ __forceinline__ float2 term_d(const Seq& q, int j, const float2* __restrict__ Df, int cap, int Ls,
                                         int qd, int lane) {
  if (q.done() || (j && !q.two())) return make_float2(0.f, 0.f);
  const int l = 128 * q.ch + 32 * qd + lane;
  return l < Ls ? __ldg(Df + ((size_t)q.bi * cap + q.t + j) * Ls + l) : make_float2(0.f, 0.f);
}

__global__ void __launch_bounds__(NTHREADS, 1)
    k_far_coupling_tc2(int Ls, int nch, int cap, int n_items, const int4* __restrict__ items,
                       const int* __restrict__ order, const int2* __restrict__ blocks, const int* __restrict__ rank,
                       const int64_t* __restrict__ first, const int* __restrict__ t1,
                       const unsigned char* __restrict__ img,
                       const float2* __restrict__ Df, const float2* __restrict__ xhat,
                       float2* __restrict__ part, int* __restrict__ err, uint64_t lim, int probe) {
  using namespace umma;
  extern __shared__ unsigned char smraw[];
  __shared__ __align__(8) uint64_t b_full[NSTAGE], b_empty[NSTAGE];
  __shared__ __align__(8) uint64_t a_full[2], a_empty[2];
  __shared__ __align__(8) uint64_t c_full[2], c_empty[2];
  __shared__ __align__(8) uint64_t fin_bar, probe_bar;
  __shared__ uint32_t tmem_sh;
  __shared__ volatile int abort_sh;
  __shared__ volatile int never_sh;
  unsigned char* ring = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&a_full[s], 4);  // one arrival per A warp
      mbar_init(&a_empty[s], 1);
      mbar_init(&c_full[s], 1);
      mbar_init(&c_empty[s], NEPI);  // one arrival per epilogue warp
    }
    mbar_init(&fin_bar, 1);
    mbar_init(&probe_bar, 1);
    abort_sh = 0;
    never_sh = 0;
    mbar_init_fence();
  }
  if (warp == W_MMA) tmem_alloc(&tmem_sh, TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  // failure-path check armed from the host: a wait on a barrier nothing completes
  if (probe && blockIdx.x == 0 && warp == W_MMA) mbar_wait(&probe_bar, 0u, &abort_sh, err, ERR_TIMEOUT, lim);

  uint32_t n_issued = 0;  // loader: images copied
  if (warp == W_MMA) {
    // -------------------------------------------------------------- MMA issue
    constexpr uint32_t ID2 = idesc_bf16(128, 128, false), ID2N = idesc_bf16(128, 128, true);
    constexpr uint32_t ID1 = idesc_bf16(128, 64, false), ID1N = idesc_bf16(128, 64, true);
    Seq q;
    q.start(items, order, n_items, nch, rank);
    uint32_t ib = 0, ia = 0;  // pairs issued, blocks entered
    bool first_pair = true;
    while (!q.done()) {
      const int s = (int)(ib % NSTAGE), ab = (int)(ia & 1u);
      const bool two = q.two(), last_pair = q.t + 2 >= rank[q.bi];
      const int npr = q.t >= t1[q.bi] ? 1 : 3;  // products: hi*hi (+ hi*lo + lo*hi)
      const uint32_t id = two ? ID2 : ID1, idn = two ? ID2N : ID1N;
      const uint32_t a_hi = tmem + 128u * ab, a_lo = a_hi + 64u;
      const uint32_t bh = smem_u32(ring + (size_t)s * BSTAGE), bl = bh + 2u * BPLANE;
      bool ok = mbar_wait(&b_full[s], (ib / NSTAGE) & 1u, &abort_sh, err, ERR_TIMEOUT, lim);
      if (first_pair) ok = mbar_wait(&a_full[ab], (ia >> 1) & 1u, &abort_sh, err, ERR_TIMEOUT, lim) && ok;
      // slot 0 (Re Z^T), then slot 1 (Im Z^T); each is free once the epilogue
      // has read the previous pair's
#pragma unroll
      for (int sl = 0; sl < 2; ++sl) {
        if (ib >= 1) ok = mbar_wait(&c_empty[sl], (ib - 1) & 1u, &abort_sh, err, ERR_TIMEOUT, lim) && ok;
        ok = __all_sync(0xffffffffu, ok);
        tc_fence_after();
        if (lane == 0) {
          if (ok) {
            const uint32_t z = tmem + ACC0 + 128u * sl;
            // products hi*hi, hi*lo, lo*hi over K = 128 in 8 steps of 16
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
              if (pr >= npr) break;
              const uint32_t aa = pr == 2 ? a_lo : a_hi;
              const uint32_t bb = pr == 1 ? bl : bh;
#pragma unroll
              for (int ks = 0; ks < 8; ++ks) {
                const uint32_t acc = (pr == 0 && ks == 0) ? 0u : 1u;
                if (sl == 0)
                  mma_bf16_ts(z, aa + 8u * ks, sdesc_lbo_sbo(bb + 256u * ks, B_LBO, B_SBO), ks < 4 ? id : idn,
                              acc);
                else
                  mma_bf16_ts(z, aa + 8u * ks, sdesc_lbo_sbo(bb + 256u * ((ks + 4) & 7), B_LBO, B_SBO), id,
                              acc);
              }
            }
          }
          mma_commit(&c_full[sl]);
        }
        __syncwarp();
      }
      if (lane == 0) {
        mma_commit(&b_empty[s]);
        if (last_pair) mma_commit(&a_empty[ab]);
      }
      __syncwarp();
      ++ib;
      const bool newblock = q.next();
      if (newblock) ++ia;
      first_pair = newblock;
    }
  } else if (warp == W_LOAD) {
    // ------------------------------------------------------------ B loader
    if (lane == 0) {
      Seq q;
      q.start(items, order, n_items, nch, rank);
      for (; !q.done(); q.next(), ++n_issued) {
        const int s = (int)(n_issued % NSTAGE);
        if (n_issued >= NSTAGE &&
            !mbar_wait(&b_empty[s], (n_issued / NSTAGE - 1) & 1u, &abort_sh, err, ERR_TIMEOUT, lim))
          break;
        const bool two = q.two(), lo = q.t < t1[q.bi];  // single-product pairs read no lo planes
        unsigned char* st = ring + (size_t)s * BSTAGE;
        const unsigned char* src = img + (size_t)(first[q.bi] + q.t) * BIMG;  // [hi t | lo t | hi t+1 | lo t+1]
        mbar_arrive_expect_tx(&b_full[s], (two ? 2u : 1u) * (lo ? 2u : 1u) * BPLANE);
        bulk_g2s(st, src, BPLANE, &b_full[s]);
        if (lo) bulk_g2s(st + 2u * BPLANE, src + BPLANE, BPLANE, &b_full[s]);
        if (two) {
          bulk_g2s(st + BPLANE, src + 2u * BPLANE, BPLANE, &b_full[s]);
          if (lo) bulk_g2s(st + 3u * BPLANE, src + 3u * BPLANE, BPLANE, &b_full[s]);
        }
      }
    }
    __syncwarp();
  } else if (warp >= W_A0 && warp < W_A0 + 4) {
    // ------------------------------------------------------------ A builders
    const int qd = warp & 3;
    const uint32_t trow = tmem + ((uint32_t)(32 * qd) << 16);
    Seq q;
    q.start(items, order, n_items, nch, rank);
    uint32_t ia = 0;
    while (!q.done()) {
      const int ab = (int)(ia & 1u);
      if (ia >= 2) mbar_wait(&a_empty[ab], ((ia >> 1) - 1) & 1u, &abort_sh, err, ERR_TIMEOUT, lim);
      const bool go = !__any_sync(0xffffffffu, abort_sh != 0);
      if (go) {
        tc_fence_after();
        const int l = 128 * q.ch + 32 * qd + lane;
        const float2* xc = xhat + (size_t)blocks[q.bi].y * TP * Ls + l;
        // K order: 0..63 Re xhat[nu], 64..127 Im xhat[nu]; two bf16 per column
#pragma unroll 1
        for (int c8 = 0; c8 < 4; ++c8) {  // nu = 16 c8 .. 16 c8 + 15: 8 columns of Re, 8 of Im
          float2 xv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            xv[j] = l < Ls ? __ldg(xc + (size_t)(16 * c8 + j) * Ls) : make_float2(0.f, 0.f);
#pragma unroll
          for (int part = 0; part < 2; ++part) {  // 0: Re (K 0..63), 1: Im (K 64..127)
            uint32_t vh[8], vl[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const float x0 = part ? xv[2 * j].y : xv[2 * j].x;
              const float x1 = part ? xv[2 * j + 1].y : xv[2 * j + 1].x;
              uint16_t h0, l0v, h1, l1v;
              split_bf16(x0, h0, l0v);
              split_bf16(x1, h1, l1v);
              vh[j] = (uint32_t)h0 | ((uint32_t)h1 << 16);
              vl[j] = (uint32_t)l0v | ((uint32_t)l1v << 16);
            }
            const uint32_t col = 128u * ab + 32u * part + 8u * c8;
            tmem_st8(trow + col, vh);
            tmem_st8(trow + col + 64u, vl);
          }
        }
        tmem_wait_st();
        tc_fence_before();
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&a_full[ab]);
      ++ia;
      // skip to the next block (or chunk, or item)
      const Seq cur = q;
      while (!q.done() && q.same_block(cur)) q.next();
    }
  } else if (warp < NEPI) {
    // ------------------------------------------------------------- epilogue
    const int qd = warp & 3, mu0 = MUE * (warp >> 2);  // lane quadrant, first mu
    const uint32_t trow = tmem + ((uint32_t)(32 * qd) << 16);
    float yr[MUE], yi[MUE];
#pragma unroll
    for (int mu = 0; mu < MUE; ++mu) yr[mu] = yi[mu] = 0.f;
    Seq q, qp;
    q.start(items, order, n_items, nch, rank);
    qp = q;
    // d_t, d_{t+1} of the next two pairs, loaded ahead of their accumulators
    float2 da0 = term_d(qp, 0, Df, cap, Ls, qd, lane), db0 = term_d(qp, 1, Df, cap, Ls, qd, lane);
    if (!qp.done()) qp.next();
    float2 da1 = term_d(qp, 0, Df, cap, Ls, qd, lane), db1 = term_d(qp, 1, Df, cap, Ls, qd, lane);
    if (!qp.done()) qp.next();
    uint32_t ic = 0;  // pairs consumed
    for (int ii = blockIdx.x; ii < n_items; ii += gridDim.x) {
      for (int ch = 0; ch < nch; ++ch) {
        while (!q.done() && q.ii == ii && q.ch == ch) {
          const bool two = q.two();
          const float2 da = da0, db = db0;
          da0 = da1;
          db0 = db1;
          da1 = term_d(qp, 0, Df, cap, Ls, qd, lane);
          db1 = term_d(qp, 1, Df, cap, Ls, qd, lane);
          if (!qp.done()) qp.next();
#pragma unroll
          for (int sl = 0; sl < 2; ++sl) {
            bool ok = mbar_wait(&c_full[sl], ic & 1u, &abort_sh, err, ERR_TIMEOUT, lim);
            ok = __all_sync(0xffffffffu, ok);
            tc_fence_after();
            if (ok) {
              // slot 0 holds Re Z^T: y += d Re z; slot 1 holds Im Z^T: y += i d Im z
              const float war = sl ? -da.y : da.x, wai = sl ? da.x : da.y;
              const float wbr = sl ? -db.y : db.x, wbi = sl ? db.x : db.y;
              const uint32_t z = trow + ACC0 + 128u * sl + (uint32_t)mu0;
#pragma unroll
              for (int m0 = 0; m0 < MUE; m0 += 16) {
                uint32_t va[16], vb[16];
                tmem_ld16(z + (uint32_t)m0, va);
                if (two) tmem_ld16(z + 64u + (uint32_t)m0, vb);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  const float a = __uint_as_float(va[j]);
                  yr[m0 + j] = fmaf(war, a, yr[m0 + j]);
                  yi[m0 + j] = fmaf(wai, a, yi[m0 + j]);
                }
                if (two) {
#pragma unroll
                  for (int j = 0; j < 16; ++j) {
                    const float bq = __uint_as_float(vb[j]);
                    yr[m0 + j] = fmaf(wbr, bq, yr[m0 + j]);
                    yi[m0 + j] = fmaf(wbi, bq, yi[m0 + j]);
                  }
                }
              }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&c_empty[sl]);
          }
          ++ic;
          q.next();
        }
        // the item's partial tile of this chunk (zero for an item without terms)
        const int l = 128 * ch + 32 * qd + lane;
        if (l < Ls) {
          float2* dst = part + ((size_t)order[ii] * TP + mu0) * Ls + l;
#pragma unroll
          for (int mu = 0; mu < MUE; ++mu) dst[(size_t)mu * Ls] = make_float2(yr[mu], yi[mu]);
        }
#pragma unroll
        for (int mu = 0; mu < MUE; ++mu) yr[mu] = yi[mu] = 0.f;
      }
    }
  }
  // ------------------------------------------------------------------ teardown
  __syncthreads();
  if (warp == W_LOAD && lane == 0) {
    // every copy issued has landed before the CTA's shared memory is released
    const uint32_t from = n_issued > NSTAGE ? n_issued - NSTAGE : 0;
    for (uint32_t u = from; u < n_issued; ++u)
      mbar_wait(&b_full[u % NSTAGE], (u / NSTAGE) & 1u, &never_sh, err, ERR_TIMEOUT);
  }
  if (warp == W_MMA) {
    // every MMA issued has finished before TMEM is released
    if (lane == 0) mma_commit(&fin_bar);
    __syncwarp();
    mbar_wait(&fin_bar, 0u, &never_sh, err, ERR_TIMEOUT);
    tc_fence_after();
    __syncwarp();
    tmem_dealloc(tmem, TCOLS);
  }
}

// Chunks of 128 frequencies on the tensor cores and the tail frequencies
// applied from the expanded FP32 table.
static void tc2_split(int Ls, int& nch, int& l_tail, int& ntail) {
  const int rem = Ls % 128;
  if (Ls > 128 && rem >= 1 && rem <= TC2_TAIL_MAX) {
    nch = Ls / 128;
    l_tail = 128 * nch;
    ntail = rem;
  } else {
    nch = (Ls + 127) / 128;
    l_tail = Ls;
    ntail = 0;
  }
}

int setup_tc2(cqm_handle* h) {
  CQM_CUDA_TRY(cudaFuncSetAttribute(k_far_coupling_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)SMEM));
  int dev = 0;
  CQM_CUDA_TRY(cudaGetDevice(&dev));
  CQM_CUDA_TRY(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev));
  return CQM_OK;
}

// B images and tail table from the FP64 factors (before they become
// float-float pairs).
int build_tc2(cqm_handle* h) {
  if (h->n_far == 0) return CQM_OK;
  std::vector<int64_t> first(h->n_far + 1, 0);
  for (int b = 0; b < h->n_far; ++b) first[b + 1] = first[b] + h->h_far_rank[b];
  CQM_TRY(h->tc2_first.allocate(h->alloc, h->n_far + 1));
  CQM_CUDA_TRY(cudaMemcpyAsync(h->tc2_first.p, first.data(), sizeof(int64_t) * (h->n_far + 1),
                               cudaMemcpyHostToDevice, h->stream));
  CQM_TRY(h->tc2_img.allocate(h->alloc, (size_t)std::max<int64_t>(1, first[h->n_far]) * BIMG));
  {
    ProfScope ps_(h, CQM_K_EXPAND);
    const int nt = std::max(1, h->info.rank_max);
    k_tc2_images<<<(unsigned)nt * (unsigned)h->n_far, 256, 0, h->stream>>>(
        h->rank_cap, nt, h->far_rank.p, h->tc2_first.p, h->farC.p, h->tc2_img.p);
  }
  CQM_CHECK_LAUNCH();
  // t1 of every block, the number of single-product terms, ref[Ls] and the
  // norms ||C_t||_F (n_far x cap), all 4-byte words
  const size_t nw = (size_t)h->n_far + 1 + h->Ls + (size_t)h->n_far * h->rank_cap;
  CQM_TRY(h->tc2_t1.allocate(h->alloc, nw));
  int* cnt = h->tc2_t1.p + h->n_far;
  unsigned int* ref = (unsigned int*)(cnt + 1);
  float* cn = (float*)(ref + h->Ls);
  CQM_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * (1 + h->Ls), h->stream));
  {
    ProfScope ps_(h, CQM_K_EXPAND);
    k_tc2_term_sizes<<<h->n_far, 256, 0, h->stream>>>(h->Ls, h->rank_cap, h->far_rank.p, h->farC.p, h->farD.p,
                                                      cn, ref);
    k_tc2_single_from<<<h->n_far, 256, 0, h->stream>>>(h->Ls, h->rank_cap, h->params.tc_single_ratio,
                                                       h->far_rank.p, h->farD.p, cn, ref, h->tc2_t1.p, cnt);
  }
  CQM_CHECK_LAUNCH();
  int n_single = 0;
  CQM_CUDA_TRY(cudaMemcpyAsync(&n_single, cnt, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  int nch, l_tail, ntail;
  tc2_split(h->Ls, nch, l_tail, ntail);
  if (ntail > 0) {
    CQM_TRY(h->tc2_tail.allocate(h->alloc, (size_t)h->n_far * ntail * TP * TP));
    ProfScope ps_(h, CQM_K_EXPAND);
    k_tc2_tail_table<<<h->n_far, 256, 0, h->stream>>>(h->Ls, h->rank_cap, l_tail, ntail, h->far_rank.p,
                                                     h->farC.p, h->farD.p, h->tc2_tail.p);
    CQM_CHECK_LAUNCH();
  }
  CQM_CUDA_TRY(cudaStreamSynchronize(h->stream));  // `first` goes out of scope
  h->info.tc_single_terms = n_single;
  return CQM_OK;
}

// Writes the item partial tiles of frequencies [0, l_tail) and adds the tail
// frequencies to yhat_f directly; returns the first tail frequency.
int far_coupling_tc2(cqm_handle* h, int* l_tail_out) {
  int nch, l_tail, ntail;
  tc2_split(h->Ls, nch, l_tail, ntail);
  ProfScope ps_(h, CQM_K_FAR_COUPLING);  // one timed unit: the chunks and the tail
  {
    k_far_coupling_tc2<<<h->n_far_items, NTHREADS, SMEM, h->stream>>>(
        h->Ls, nch, h->rank_cap, h->n_far_items, h->far_items.p, h->far_order.p, h->far_rc.p, h->far_rank.p,
        h->tc2_first.p, h->tc2_t1.p, h->tc2_img.p, h->farD_f.p, h->xhat_f.p, h->part_f.p, h->flag.p + 1, h->wait_limit_ns,
        h->wait_probe ? 1 : 0);
    h->wait_probe = false;  // one-shot
  }
  CQM_CHECK_LAUNCH();
  if (ntail > 0) {
    const int nfr = (int)h->h_far_rows.size();
    k_far_tail_f32<<<(unsigned)(nfr * ntail), 256, 0, h->stream>>>(
        h->Ls, l_tail, ntail, h->d_far_rows.p, h->far_rowptr.p, h->far_rc.p, h->tc2_tail.p,
        h->xhat_f.p, h->yhat_f.p, h->inner_active);
    CQM_CHECK_LAUNCH();
  }
  *l_tail_out = l_tail;
  return CQM_OK;
}

}  // namespace cqm
