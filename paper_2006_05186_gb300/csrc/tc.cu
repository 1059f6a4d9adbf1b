// Far-field coupling of the inner operator on the fifth-generation tensor
// cores (tcgen05, accumulator in TMEM).
//
// yhat_r[mu][l] += sum_{b=(r,c)} sum_t sum_nu C_{b,t}[mu][nu] d_{b,t}[l] xhat_c[nu][l]
// (eq. lrfinal for all frequencies at once).  In real arithmetic each rank term
// (b, t) is one GEMM with M = 128, K = 128 and N = the frequency columns:
//   [Re y; Im y] += [[Re C, -Im C], [Im C, Re C]] [Re x~; Im x~],  x~ = d_t (.) xhat_c,
// and a work item (a row cluster and a run of its far blocks) sums all of its
// (b, t) in one TMEM accumulator.  Every operand is split as hi (rounded to
// tf32) + lo, and the three products lo*hi + hi*lo + hi*hi are accumulated in
// fp32, which carries each operand to 2^-21 (the inner operator is fp32-class;
// the FP64-accurate residual is computed apart).
//
// One CTA per work item.  Each K-slab covers 16 Chebyshev indices nu (their
// real and imaginary parts: 32 real-form K).  Warp 13 runs ahead and copies
// each slab's 16 x 64 block of C (stored nu-major, 8 KB contiguous) into a
// ring of 8 staging buffers with bulk asynchronous copies; warps 1-4 build the
// slab's A (the real form of C) from there row by row straight into tensor
// memory, one TMEM lane per row; warps 5-12 build B = x~ in shared memory in
// the canonical K-major layout, with the d_t values loaded three slabs ahead.
// A ring of 4 slabs is guarded by mbarriers; one thread of warp 0 issues
// 4 x 3 MMAs per slab (A from TMEM, B from shared memory) and frees the slab
// with tcgen05.commit; warps 1-4 finally copy the accumulator from TMEM into
// the item's partial tile, which the per-row reduction adds in item order (as
// for the SIMT kernel).  Every wait is bounded in time; on expiry the kernel
// records an error in *err, stops issuing work, lets issued copies and MMAs
// drain, frees TMEM and returns.  The time limit of the waits of the main
// loop is the handle's (cqm_bem_set_wait_limit); the drain at the end waits
// for copies and MMAs already issued, with the default limit of one second.
#include <algorithm>

#include "handle.cuh"
#include "umma.cuh"

namespace cqm {

namespace {
constexpr int TP = 64;          // Chebyshev points per cluster (m = 4)
constexpr int NSTAGE = 4;       // slabs in the MMA ring
constexpr int NCS = 8;          // C staging buffers (8 KB each)
constexpr uint32_t CSLAB = 16u * TP * 8u;  // bytes of one slab of C: 16 nu x 64 mu complex fp32
constexpr int NA = 128;         // A producer threads (warps 1..4): one TMEM lane (row) each
constexpr int NBP = 256;        // B producer threads (warps 5..12)
constexpr int LOADER = 13;      // warp that issues the C copies
constexpr int NTHREADS = 32 * (LOADER + 1);
constexpr uint32_t TCOLS = 512;       // TMEM columns: accumulator [0, 256), A ring [256, 512)
constexpr uint32_t ACOL = 256;        // first column of the A ring; 64 per slab (hi 32, lo 32)
constexpr int ERR_TIMEOUT = 1;

template <int NT>
struct TcCfg {
  static constexpr int NC = 16 * NT;                       // frequency columns per chunk (MMA N)
  static constexpr uint32_t B_PLANE = (uint32_t)NC * 128u;  // NC rows x 32 tf32
  static constexpr uint32_t STAGE = 2 * B_PLANE;
  static constexpr size_t SMEM_RING = (size_t)NSTAGE * STAGE + (size_t)NCS * CSLAB + 1024;
  // at least 116 KB: one CTA per SM, which owns all 512 TMEM columns
  static constexpr size_t SMEM = SMEM_RING > 118784 ? SMEM_RING : 118784;
};

// Position in the slab sequence (block b, nu slab j, rank term t), blocks of
// rank 0 skipped; bi == end once the sequence is exhausted.
struct SlabPos {
  int bi, j, tt;
  __device__ void start(int b0, int end, const int* rank) {
    bi = b0;
    j = tt = 0;
    while (bi < end && rank[bi] == 0) ++bi;
  }
  __device__ void next(int end, const int* rank) {
    if (++tt == rank[bi]) {
      tt = 0;
      if (++j == 4) {
        j = 0;
        do ++bi; while (bi < end && rank[bi] == 0);
      }
    }
  }
};

__device__ __forceinline__ void st_split4(unsigned char* hi, unsigned char* lo, uint32_t off, float a,
                                          float b, float c, float d) {
  float4 h, l;
  umma::split_tf32(a, h.x, l.x);
  umma::split_tf32(b, h.y, l.y);
  umma::split_tf32(c, h.z, l.z);
  umma::split_tf32(d, h.w, l.w);
  *(float4*)(hi + off) = h;
  *(float4*)(lo + off) = l;
}
}  // namespace

template <int NT>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_far_coupling_tc(int Ls, int cap, const int4* __restrict__ items, const int2* __restrict__ blocks,
                      const int* __restrict__ rank, const float2* __restrict__ Cf,
                      const float2* __restrict__ Df, const float2* __restrict__ xhat,
                      float2* __restrict__ part, int* __restrict__ err, uint64_t lim,
                      int probe) {
  using namespace umma;
  using K = TcCfg<NT>;
  constexpr int NC = K::NC;
  constexpr int NB = (4 * NC + NBP - 1) / NBP;  // B items per producer thread and slab
  extern __shared__ unsigned char smraw[];
  __shared__ __align__(8) uint64_t full_bar[NSTAGE];
  __shared__ __align__(8) uint64_t empty_bar[NSTAGE];
  __shared__ __align__(8) uint64_t cfull_bar[NCS];
  __shared__ __align__(8) uint64_t cempty_bar[NCS];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ __align__(8) uint64_t fin_bar;
  __shared__ __align__(8) uint64_t probe_bar;  // never completed (failure-path check)
  __shared__ uint32_t tmem_sh;
  __shared__ volatile int abort_sh;
  __shared__ volatile int never_sh;
  unsigned char* ring = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  unsigned char* cstage = ring + (size_t)NSTAGE * K::STAGE;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4 it = items[blockIdx.x];  // (row, first block, end block, -)

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full_bar[s], (NA + NBP) / 32);  // one arrival per producer warp
      mbar_init(&empty_bar[s], 1);
    }
    for (int s = 0; s < NCS; ++s) {
      mbar_init(&cfull_bar[s], 1);
      mbar_init(&cempty_bar[s], NA / 32);
    }
    mbar_init(&done_bar, 1);
    mbar_init(&fin_bar, 1);
    mbar_init(&probe_bar, 1);
    abort_sh = 0;
    never_sh = 0;
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_sh, TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;

  // Check of the failure path, armed from the host: the first CTA waits on a
  // barrier that nothing completes; the wait runs out after `lim` and the
  // whole CTA takes the abort path below.
  if (probe && blockIdx.x == 0 && warp == 0) mbar_wait(&probe_bar, 0u, &abort_sh, err, ERR_TIMEOUT, lim);

  int nwork = 0;  // rank terms of the item; none leaves the tile zero
  for (int bi = it.y; bi < it.z; ++bi) nwork += rank[bi];

  // Slabs in the order (block b, nu slab j, rank term t) in every role.
  uint32_t use = 0;
  int chunk = 0;
  uint32_t c_issued = 0;  // loader: C copies issued so far
  for (int l0 = 0; l0 < Ls; l0 += NC, ++chunk) {
    if (warp == 0) {
      // ---------------------------------------------------------------- MMA
      constexpr uint32_t idesc = idesc_tf32(128, NC);
      uint32_t acc = 0;
      for (int k = 0; k < 4 * nwork; ++k, ++use) {
        const int s = (int)(use % NSTAGE);
        const bool ok = mbar_wait(&full_bar[s], (use / NSTAGE) & 1u, &abort_sh, err, ERR_TIMEOUT, lim);
        tc_fence_after();
        if (ok && lane == 0) {
          const uint32_t a_hi = tmem + ACOL + 64u * s, a_lo = a_hi + 32u;
          const uint32_t b_hi = smem_u32(ring + (size_t)s * K::STAGE), b_lo = b_hi + K::B_PLANE;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            mma_tf32_ts(tmem, a_lo + 8u * ks, sdesc(b_hi + 256u * ks), idesc, acc);
            mma_tf32_ts(tmem, a_hi + 8u * ks, sdesc(b_lo + 256u * ks), idesc, 1u);
            mma_tf32_ts(tmem, a_hi + 8u * ks, sdesc(b_hi + 256u * ks), idesc, 1u);
            acc = 1u;
          }
          mma_commit(&empty_bar[s]);
        }
        __syncwarp();
      }
      if (lane == 0 && nwork > 0) mma_commit(&done_bar);
      __syncwarp();
    } else if (warp == LOADER) {
      // ------------------------------------------------------------- loader
      if (lane == 0) {
        SlabPos sp;
        sp.start(it.y, it.z, rank);
        for (; sp.bi < it.z; sp.next(it.z, rank), ++c_issued) {
          const int sc = (int)(c_issued % NCS);
          if (c_issued >= NCS &&
              !mbar_wait(&cempty_bar[sc], (c_issued / NCS - 1) & 1u, &abort_sh, err, ERR_TIMEOUT, lim))
            break;
          mbar_arrive_expect_tx(&cfull_bar[sc], CSLAB);
          bulk_g2s(cstage + (size_t)sc * CSLAB,
                   Cf + ((size_t)sp.bi * cap + sp.tt) * TP * TP + (size_t)(16 * sp.j) * TP, CSLAB,
                   &cfull_bar[sc]);
        }
      }
      __syncwarp();
    } else if (warp <= 4) {
      // -------------------------------------------------------- A producers
      // Row m = 32 (warp % 4) + lane of the real form: m < 64 gives Re y_mu,
      // [Re C | -Im C]; m >= 64 gives Im y_mu, [Im C | Re C] (mu = m mod 64).
      const int q = warp & 3, m = 32 * q + lane, mu = m & 63;
      const bool im = m >= 64;
      const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + ACOL;
      for (int k = 0; k < 4 * nwork; ++k, ++use) {
        const int sc = (int)(use % NCS);
        float2 c[16];
        const bool cok = mbar_wait(&cfull_bar[sc], (use / NCS) & 1u, &abort_sh, err, ERR_TIMEOUT, lim);
        if (cok) {
          const float2* cs = (const float2*)(cstage + (size_t)sc * CSLAB) + mu;
#pragma unroll
          for (int v = 0; v < 16; ++v) c[v] = cs[v * TP];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&cempty_bar[sc]);
        const int s = (int)(use % NSTAGE);
        const uint32_t round = use / NSTAGE;
        if (round > 0) mbar_wait(&empty_bar[s], (round - 1) & 1u, &abort_sh, err, ERR_TIMEOUT, lim);
        if (!__any_sync(0xffffffffu, abort_sh != 0)) {
          tc_fence_after();
          uint32_t hi[16], lo[16];
          // K 0..15: Re C (Re rows) or Im C (Im rows) of nu = 16 j + k
#pragma unroll
          for (int v = 0; v < 16; ++v) {
            float h, l;
            split_tf32(im ? c[v].y : c[v].x, h, l);
            hi[v] = __float_as_uint(h);
            lo[v] = __float_as_uint(l);
          }
          tmem_st16(trow + 64u * s, hi);
          tmem_st16(trow + 64u * s + 32u, lo);
          // K 16..31: -Im C (Re rows) or Re C (Im rows)
#pragma unroll
          for (int v = 0; v < 16; ++v) {
            float h, l;
            split_tf32(im ? c[v].x : -c[v].y, h, l);
            hi[v] = __float_as_uint(h);
            lo[v] = __float_as_uint(l);
          }
          tmem_st16(trow + 64u * s + 16u, hi);
          tmem_st16(trow + 64u * s + 48u, lo);
          tmem_wait_st();
          tc_fence_before();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&full_bar[s]);
      }
    } else {
      // -------------------------------------------------------- B producers
      // The 16 rows of xhat_c of slab j are loaded once per (b, j) and reused
      // for every t; d_t is loaded three slabs ahead (register chain).
      const int pb = tid - 32 - NA;
      auto load_d = [&](const SlabPos& sp, float2 (&dv)[NB]) {
        if (sp.bi >= it.z) return;
        const float2* Dt = Df + ((size_t)sp.bi * cap + sp.tt) * Ls;
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          const int e = pb + NBP * i;
          const int lg = l0 + e % NC;
          dv[i] = (e < 4 * NC && lg < Ls) ? Dt[lg] : make_float2(0.f, 0.f);
        }
      };
      auto load_x = [&](const SlabPos& sp, float2 (&xv)[NB][4]) {
        const float2* xc = xhat + (size_t)blocks[sp.bi].y * TP * Ls;
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          const int e = pb + NBP * i;
          const int qq = e / NC, lg = l0 + e - qq * NC;
          const bool in = e < 4 * NC && lg < Ls;
#pragma unroll
          for (int v = 0; v < 4; ++v)
            xv[i][v] = in ? xc[(size_t)(16 * sp.j + 4 * qq + v) * Ls + lg] : make_float2(0.f, 0.f);
        }
      };
      SlabPos cur, ahead;
      cur.start(it.y, it.z, rank);
      ahead = cur;
      float2 d0[NB], d1[NB], d2[NB], xv[NB][4];
      if (cur.bi < it.z) load_x(cur, xv);
      load_d(ahead, d0);
      if (ahead.bi < it.z) ahead.next(it.z, rank);
      load_d(ahead, d1);
      if (ahead.bi < it.z) ahead.next(it.z, rank);
      load_d(ahead, d2);
      if (ahead.bi < it.z) ahead.next(it.z, rank);
      for (; cur.bi < it.z; ++use) {
        const int s = (int)(use % NSTAGE);
        const uint32_t round = use / NSTAGE;
        if (round > 0) mbar_wait(&empty_bar[s], (round - 1) & 1u, &abort_sh, err, ERR_TIMEOUT, lim);
        if (!abort_sh) {
          unsigned char* Bhi = ring + (size_t)s * K::STAGE;
          unsigned char* Blo = Bhi + K::B_PLANE;
          // row l, Re x~ at K group qq, Im x~ at K group 4 + qq
#pragma unroll
          for (int i = 0; i < NB; ++i) {
            const int e = pb + NBP * i;
            if (e < 4 * NC) {
              const int qq = e / NC, l = e - qq * NC;
              float re[4], imv[4];
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                re[v] = fmaf(d0[i].x, xv[i][v].x, -d0[i].y * xv[i][v].y);
                imv[v] = fmaf(d0[i].x, xv[i][v].y, d0[i].y * xv[i][v].x);
              }
              st_split4(Bhi, Blo, core_off(l, 4 * qq), re[0], re[1], re[2], re[3]);
              st_split4(Bhi, Blo, core_off(l, 16 + 4 * qq), imv[0], imv[1], imv[2], imv[3]);
            }
          }
          fence_async_shared();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&full_bar[s]);
        cur.next(it.z, rank);
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          d0[i] = d1[i];
          d1[i] = d2[i];
        }
        load_d(ahead, d2);
        if (ahead.bi < it.z) ahead.next(it.z, rank);
        if (cur.bi < it.z && cur.tt == 0) load_x(cur, xv);
      }
    }
    // ------------------------------------------- epilogue: TMEM -> partial tile
    if (warp >= 1 && warp <= 4) {
      const int qd = warp & 3;  // TMEM lanes 32 qd .. 32 qd + 31 belong to this warp
      const int m = 32 * qd + lane, mu = m & 63, im = m >> 6;
      bool ok = nwork > 0 && mbar_wait(&done_bar, (uint32_t)chunk & 1u, &abort_sh, err, ERR_TIMEOUT, lim);
      ok = __all_sync(0xffffffffu, ok);
      tc_fence_after();
      float* dst = (float*)(part + ((size_t)blockIdx.x * TP + mu) * Ls) + im;
      for (int c0 = 0; c0 < NC; c0 += 16) {
        uint32_t v[16];
        if (ok) {
          tmem_ld16(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)c0, v);
          tmem_wait_ld();
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0u;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int l = l0 + c0 + i;
          if (l < Ls) dst[2 * l] = __uint_as_float(v[i]);
        }
      }
      tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
  }
  // ------------------------------------------------------------------ teardown
  if (warp == LOADER && lane == 0) {
    // every copy issued has landed before the CTA's shared memory is released
    const uint32_t first = c_issued > NCS ? c_issued - NCS : 0;
    for (uint32_t u = first; u < c_issued; ++u)
      mbar_wait(&cfull_bar[u % NCS], (u / NCS) & 1u, &never_sh, err, ERR_TIMEOUT);
  }
  if (warp == 0) {
    // every MMA this thread issued has finished before TMEM is released
    if (lane == 0) mma_commit(&fin_bar);
    __syncwarp();
    mbar_wait(&fin_bar, 0u, &never_sh, err, ERR_TIMEOUT);
    tc_fence_after();
    __syncwarp();
    tmem_dealloc(tmem, TCOLS);
  }
}

static int nt_for(int Ls) {
  const int nchunk = (Ls + 159) / 160;
  const int per = (Ls + nchunk - 1) / nchunk;
  return std::max(1, std::min(10, (per + 15) / 16));
}

int setup_tc_kernels(cqm_handle* h) {
#define TC_SETUP(N)                                                                                \
  CQM_CUDA_TRY(cudaFuncSetAttribute(k_far_coupling_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                    (int)TcCfg<N>::SMEM));
  TC_SETUP(1) TC_SETUP(2) TC_SETUP(3) TC_SETUP(4) TC_SETUP(5)
  TC_SETUP(6) TC_SETUP(7) TC_SETUP(8) TC_SETUP(9) TC_SETUP(10)
#undef TC_SETUP
  return CQM_OK;
}

int far_coupling_tc(cqm_handle* h) {
  const int n = h->n_far_items;
  ProfScope ps_(h, CQM_K_FAR_COUPLING);
#define TC_CASE(N)                                                                                 \
  case N:                                                                                          \
    k_far_coupling_tc<N><<<n, NTHREADS, TcCfg<N>::SMEM, h->stream>>>(                              \
        h->Ls, h->rank_cap, h->far_items.p, h->far_rc.p, h->far_rank.p, h->farC_f.p, h->farD_f.p,  \
        h->xhat_f.p, h->part_f.p, h->flag.p + 1, h->wait_limit_ns, h->wait_probe ? 1 : 0);            \
    break;
  switch (nt_for(h->Ls)) {
    TC_CASE(1) TC_CASE(2) TC_CASE(3) TC_CASE(4) TC_CASE(5)
    TC_CASE(6) TC_CASE(7) TC_CASE(8) TC_CASE(9) TC_CASE(10)
    default: break;
  }
#undef TC_CASE
  h->wait_probe = false;  // one-shot
  CQM_CHECK_LAUNCH();
  return CQM_OK;
}

}  // namespace cqm
