// Internal state of a cqm_handle and the entry points of each module.
#pragma once

#include <vector>

#include "common.cuh"
#include "quad.cuh"

struct cqm_handle {
  cqm::Allocator alloc;
  cudaStream_t stream = nullptr;
  cqm_params params{};
  int M = 0, nv = 0, N = 0, L = 0, Ls = 0, bdf = 2;
  double dt = 0.0, R = 0.0;

  // geometry (Sec. 3.2: flat triangles)
  cqm::DArray<int> tri;
  cqm::DArray<double> xyz, P, area, cen, diam;
  cqm::DArray<int> flag;  // device status word (degenerate input, capacity, ...)
  // time limit of the bounded device waits of the pipelined kernels (ns)
  uint64_t wait_limit_ns = 1000000000ull;
  bool wait_probe = false;  // next pipelined launch makes one wait that runs out

  // quadrature tables
  cqm::DArray<double4> near_pt, ss_pt[3];
  cqm::DArray<double> ss_w[3];
  cqm::Quad quad{};
  cqm::DArray<double> exp_t2;
  cqm::DArray<double2> exp_cs;
  cqm::DArray<float2> exp_t2_ff;  // the same tables as float-float pairs
  cqm::DArray<float4> exp_cs_ff;

  // CQM frequencies s_l, l = 0..L-1 (eq. cqm_freq)
  cqm::DArray<double2> s;
  std::vector<double2> s_host;

  // dense representation: V[l][i][j], l < Ls
  cqm::DArray<double2> Vd;

  // cluster tree (Def. 2), breadth-first numbering
  int n_nodes = 0, n_leaves = 0, depth = 0;
  cqm::DArray<int> perm, node_begin, node_end, node_son0, node_son1, node_parent, node_level;
  cqm::DArray<double> node_lo, node_hi;  // n_nodes x 3
  std::vector<int> level_begin;          // host: first node of each level (+ sentinel)
  std::vector<int> h_begin, h_end, h_son0, h_son1, h_level;

  // block partition (Defs. 3-4), sorted by (row, column)
  int n_near = 0, n_far = 0;
  cqm::DArray<int2> near_rc, far_rc;
  cqm::DArray<int> near_rowptr, far_rowptr;  // CSR over row clusters (n_nodes + 1)
  std::vector<int2> h_near, h_far;

  // cluster bases (Sec. 4.2, Alg. 1): Chebyshev nodes, leaf matrices, transfers
  int m = 4, p = 64;
  cqm::DArray<double> cheb;      // n_nodes x 3 x m
  cqm::DArray<double> Uleaf;     // per position i (tree order): p values -> M x p
  cqm::DArray<double> Etr;       // per node (non-root): 3 x m x m 1-D transfer factors

  // MACA factors (Alg. 2, eq. lrfinal); rank slots of capacity rank_cap per block
  int rank_cap = 32;
  cqm::DArray<int> near_rank, far_rank;
  cqm::DArray<int64_t> near_off;      // C slot base per near block (complex entries)
  cqm::DArray<double2> nearC, nearD;  // C: sum_b cap * #r #c ; D: n_near x cap x Ls
  cqm::DArray<double2> farC, farD;    // C: n_far x cap x p x p ; D: n_far x cap x Ls
  std::vector<int> h_near_rank, h_far_rank;
  std::vector<int64_t> h_near_off;
  // near-field quadrature points cached for the MACA slices and fibres
  int64_t n_points = 0;
  std::vector<int64_t> h_block_points;  // cached near points of each block (0 for lower blocks)
  cqm::DArray<int64_t> pt_off;
  cqm::DArray<int> pt_cnt;
  cqm::DArray<double> pt_r, pt_c;  // FP64 r and c; with maca_ff the same bytes hold
                                   // float-float d = r - r0 and c
  cqm::DArray<double> pt_r0;       // maca_ff: distance bound r0 of each pair
  // maca_ff: far blocks' kernel points (Chebyshev pairs), float-float d and c,
  // entry (mu, nu) of block b at b p^2 + mu p + nu, bound r0 per block
  cqm::DArray<float2> fpt_d, fpt_c;
  cqm::DArray<double> fpt_r0;
  bool cache_far_points = false;

  // apply plan: leaf clusters and row clusters owning far blocks
  std::vector<int> h_leaves, h_far_rows;
  cqm::DArray<int> d_leaves, d_far_rows;
  // balanced work items (row, first block, end block) of the contractions,
  // with per-row item ranges; partial tiles are reduced per row in item order
  int n_far_items = 0, n_near_items = 0;
  cqm::DArray<int4> far_items, near_items;
  cqm::DArray<int> far_order;  // far items by decreasing work (launch order of the coupling)
  cqm::DArray<int> far_item_ptr, near_item_ptr;
  cqm::DArray<float2> part_f;
  cqm::DArray<double2> part_d;

  // leaf block-diagonal preconditioner: P[leaf][i][j][l]
  bool use_precond = false;
  cqm::DArray<double2> Pinv;

  // FP32 copy of the operator (inner iterations of mixed precision)
  bool use_f32 = false;
  bool factors_ff = false;  // nearC / farC hold float-float pairs (hi re, hi im, lo re, lo im)
  bool farC_f_transposed = false;  // farC_f tiles stored nu-major (tensor-core coupling)
  // expanded near field: block b, frequency l, entry (i, j) at
  // nearV_off[b] + (l #c + j) #r + i; nearV holds FP64 values, or float-float
  // pairs when nearV_ff, and nearV_f their FP32 values
  bool near_expanded = false;
  bool expand_near_ok = false;  // expand_near and the table fits (a quarter of the device)
  bool nearV_ff = false;  // nearV holds float-float pairs (expanded after factors_to_ff)
  cqm::DArray<double2> nearV;
  cqm::DArray<float2> nearV_f;
  cqm::DArray<int64_t> nearV_off;
  std::vector<int64_t> h_nearV_off;
  // expanded far couplings (float-float pairs) for the FP64-accurate apply:
  // block b, frequency l, entry (mu, nu) at (b Ls + l) p^2 + nu p + mu
  bool far_expanded = false;
  cqm::DArray<double2> farS;
  cqm::DArray<float2> nearC_f, nearD_f, farC_f, farD_f, xhat_f, yhat_f;
  cqm::DArray<float2> x32;  // FP32 copy of the inner apply's input (expanded near field)
  // frequencies still iterating while GMRES applies the inner operator (null
  // otherwise): the kernels of the inner apply that work per frequency or per
  // chunk of 32 skip the others, whose results GMRES does not read
  const int* inner_active = nullptr;
  // frequencies whose residual a GMRES restart recomputes (null otherwise):
  // the FP64-accurate apply's expanded streams and sweeps skip the others
  // (converged at an earlier restart: their solution has not changed since)
  const int* exact_active = nullptr;
  // bf16 images of the far factors for the tensor-core coupling (32 KB per rank
  // term, term t of block b at tc2_first[b] + t) and the FP32 expanded
  // couplings of its tail frequencies
  cqm::DArray<int64_t> tc2_first;
  cqm::DArray<unsigned char> tc2_img;
  // first term of each far block from which the pairs take one product
  cqm::DArray<int> tc2_t1;
  cqm::DArray<float2> tc2_tail;
  int n_sm = 1;  // multiprocessors of the handle's device (persistent grids)
  cqm::DArray<float> Uleaf_f, Etr_f;

  // solver workspace
  cqm::DArray<double2> xhat, yhat;  // n_nodes x p x Ls (far field transforms)

  // marching on in time (mot.cu), built on the first call that needs it:
  // transformed MACA fibres dhat_t[n] (eq. fastdft), (b cap + t) L + n, of the
  // near and far blocks; explicit cluster bases (rows of every node from
  // Ue_off[r], p per row); the inverse of the dense step-0 weight Vhat_0 in
  // tree order (M x M, row-major)
  bool mot_ready = false;
  cqm::DArray<double2> mot_dn, mot_df;
  cqm::DArray<float4> mot_dn_ff, mot_df_ff;  // the same as float-float pairs (history sums)
  cqm::DArray<double> mot_Ue, mot_Ainv;
  cqm::DArray<int64_t> mot_Ue_off;
  double mot_setup_ms = 0.0;

  // double layer (dlayer.cu), built on the first call that needs it: the
  // near-field table (the expanded near-field layout, FP64) and the leaf
  // column basis W (M x p, tree order)
  bool dl_ready = false;
  cqm::DArray<double2> dl_table;
  cqm::DArray<int64_t> dl_off;
  cqm::DArray<double> dl_W;

  cqm_setup_info info{};

  // per-launch kernel timing (cqm_bem_profile)
  bool prof_on = false;
  struct ProfRec { int id; cudaEvent_t a, b; };
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  int64_t prof_launch[CQM_K_COUNT] = {};
  double prof_ms[CQM_K_COUNT] = {};
};

namespace cqm {

// geometry.cu
int build_geometry(cqm_handle* h, const cqm_mesh* mesh);
int build_frequencies(cqm_handle* h);
int rhs_plane_wave(cqm_handle* h, const double dir[3], double width, double delay, double* d_rhs);

// transform.cu
int forward_transform(cqm_handle* h, const double* d_b, double2* d_ghat);
int inverse_transform(cqm_handle* h, const double2* d_qhat, double* d_q);
int forward_transform_cols(cqm_handle* h, int ncol, const double* d_b, double2* d_ghat);
int inverse_transform_cols(cqm_handle* h, int ncol, const double2* d_qhat, double* d_q);
// mixed boundary conditions, dense mode: q (N+1 x nt) on Gamma_D, u (N+1 x nv) on Gamma_N's space
int mixed_solve(cqm_handle* h, const int* dmask, const double* gD, const double* gN, double* q, double* u);

// entries.cu
int build_quad_tables(cqm_handle* h);
int entries_list(cqm_handle* h, int64_t npairs, const int* d_I, const int* d_J, int nfreq,
                 const int* d_freq, double2* d_out);
int assemble_dense(cqm_handle* h);
int apply_dense(cqm_handle* h, const double2* x, double2* y);

// cluster.cu
int build_tree(cqm_handle* h);
int launch_tree_kernel(int M, int n_min, int cap, const double* xyz, const int* tri,
                       const double* cen, int* perm, int* tmp, int* begin, int* end, int* son0,
                       int* son1, int* parent, int* level, double* lo, double* hi, int* split,
                       int* counters, cudaStream_t stream);
int build_partition(cqm_handle* h);

// h2.cu
int build_bases(cqm_handle* h);
int apply_compressed(cqm_handle* h, const double2* x, double2* y);
int apply_compressed_f32(cqm_handle* h, const double2* x, double2* y);
int build_f32_copy(cqm_handle* h);

// apply32.cu (register-tiled FP32 contractions of the inner operator)
int setup_f32_kernels(cqm_handle* h);
int near_apply_f32(cqm_handle* h, const double2* x, double2* y);
int far_coupling_f32(cqm_handle* h);
int far_coupling_generic_f32(cqm_handle* h);

// tc.cu (tensor-core far coupling of the inner operator, TF32, tensor_cores = 2)
int setup_tc_kernels(cqm_handle* h);
int far_coupling_tc(cqm_handle* h);
// tc2.cu (tensor-core far coupling of the inner operator, bf16, tensor_cores = 1)
int setup_tc2(cqm_handle* h);
int build_tc2(cqm_handle* h);  // from the FP64 far factors, before factors_to_ff
int far_coupling_tc2(cqm_handle* h, int* l_tail);

// ff.cu (float-float contractions of the FP64-accurate apply)
int setup_ff(cqm_handle* h);
int near_apply_ff(cqm_handle* h, const double2* x, double2* y);
int far_coupling_ff(cqm_handle* h);
int factors_to_ff(cqm_handle* h);  // after every FP64 reader of the C factors at setup

// near_dense.cu (expanded near field)
// dense Galerkin matrices with P1 functions (mixed boundary conditions), device
int p1_matrices(cqm_handle* h, double2* K1, double2* Kp, double2* D);
int build_near_expanded(cqm_handle* h);  // after the near MACA, before factors_to_ff
int near_apply_expanded(cqm_handle* h, const double2* x, double2* y, bool fp64);
// ff.cu (expanded far couplings of the FP64-accurate apply)
int build_far_expanded(cqm_handle* h);  // after factors_to_ff; stays factored if it does not fit
int far_apply_expanded_ff(cqm_handle* h);
int build_near_expanded_ff(cqm_handle* h);  // after factors_to_ff
int near_apply_expanded_ff(cqm_handle* h, const double2* x, double2* y);

// maca.cu
int build_maca(cqm_handle* h);
int build_work_items(cqm_handle* h);

// precond.cu
int build_precond(cqm_handle* h);
// act (may be null): frequencies to compute (the others are left untouched)
int apply_precond(cqm_handle* h, const double2* v, double2* z, const int* act = nullptr);

// gmres.cu
int gmres_solve(cqm_handle* h, const double2* d_b, double2* d_x, cqm_solve_info* info);

// mot.cu (marching on in time with the compressed CQM weights)
int mot_prepare(cqm_handle* h);
int mot_weight(cqm_handle* h, int n, double* d_W);  // dense Vhat_n, original numbering
int mot_solve(cqm_handle* h, const double* d_b, double* d_q, cqm_solve_info* info);
void mot_release(cqm_handle* h);

// dlayer.cu (double layer, direct Dirichlet formulation)
int dl_apply(cqm_handle* h, const double2* x, double2* y);  // y_l = K_l x_l, l < Ls
int dl_solve(cqm_handle* h, const double* d_g, double* d_q, cqm_solve_info* info);
void dl_release(cqm_handle* h);
// near_dense.cu / h2.cu pieces the double layer shares
int near_apply_table(cqm_handle* h, const double2* T, const int64_t* off, const double2* x, double2* y);
int apply_far_columns(cqm_handle* h, const double* Wleaf, const double2* x, double2* y);

// Kernel timing scope: records an event pair around the launches it encloses.
struct ProfScope {
  cqm_handle* h;
  int idx = -1;
  ProfScope(cqm_handle* hh, int id);
  ~ProfScope();
};
void prof_resolve(cqm_handle* h);
void prof_release(cqm_handle* h);

// flag[1]: a kernel's bounded wait expired (it recorded the error and returned).
// Reads the word after the stream's work so far and clears it; CQM_ETIMEOUT if
// it was set.  clear_wait_flag resets it before a call's first launch.
int check_wait_flag(cqm_handle* h);
int clear_wait_flag(cqm_handle* h);

// operator dispatch: FP64 operator, and the operator of the inner GMRES
// iterations (its FP32 copy when mixed precision is on)
inline int apply_operator(cqm_handle* h, const double2* x, double2* y) {
  return h->params.mode == CQM_MODE_DENSE ? apply_dense(h, x, y) : apply_compressed(h, x, y);
}
inline int apply_operator_inner(cqm_handle* h, const double2* x, double2* y) {
  if (h->params.mode != CQM_MODE_DENSE && h->use_f32) return apply_compressed_f32(h, x, y);
  return apply_operator(h, x, y);
}

}  // namespace cqm
