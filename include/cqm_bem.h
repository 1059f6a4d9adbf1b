/*
 * cqm_bem.h -- C ABI of libcqmbem, a GB300 (sm_103a) implementation of the
 * frequency-domain convolution-quadrature boundary element method for the
 * acoustic single layer.
 *
 * The method (D. Seibel, "Boundary Element Methods for the Wave Equation based
 * on Hierarchical Matrices and Adaptive Cross Approximation"):
 *   - CQM frequencies s_l = chi(R zeta^l) / dt, zeta = exp(2 pi i / L),
 *     L = N + 1 (Sec. 3.1, eq. cqm_freq);
 *   - per frequency, the P0 Galerkin single layer
 *     V_l[i,j] = int_{tau_i} int_{tau_j} exp(-s_l |x-y|) / (4 pi |x-y|)
 *     (Sec. 3.2, eq. fundsol);
 *   - optionally compressed as an H^2 matrix with Chebyshev interpolation
 *     (Sec. 4, Alg. 1) and, block by block, in frequency by multivariate
 *     adaptive cross approximation (Sec. 5.1, Alg. 2; Alg. 3, eq. lrfinal);
 *   - the decoupled solve of the Remark in Sec. 6.2: transform the data to
 *     the frequencies, solve V_l qhat_l = ghat_l for every l (GMRES on the
 *     GPU), transform back with the R-scaled inverse DFT (eq. omega_n).
 *
 * Conventions shared by every call:
 *   - All arrays are plain pointers.  Arrays that cross the boundary as
 *     complex numbers are interleaved (re, im) float64 pairs.
 *   - Where a call takes `mem`, CQM_MEM_HOST means the pointers are host
 *     memory (pinned or pageable) and CQM_MEM_DEVICE means device memory of
 *     the handle's device.  Host buffers are copied inside the call.
 *   - The caller owns every buffer it passes; the handle owns all device
 *     state it allocates (geometry, tree, bases, compressed blocks, solver
 *     workspace) and frees it in cqm_bem_destroy.
 *   - Calls on one handle must not run concurrently (a handle is bound to
 *     one CUDA stream).  Different handles are independent.
 *   - Every call returns a status code; nothing aborts, exits or traps.
 *     cqm_bem_strerror() names a code; cqm_bem_last_error() gives the
 *     detail message of the most recent failure on the calling thread.
 *   - Calls that return host data synchronise the handle's stream.
 */
#ifndef CQM_BEM_H
#define CQM_BEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define CQM_OK        0
#define CQM_EINVAL    1   /* bad argument: N < 1, dt <= 0, bdf not 1/2, bad indices, degenerate triangle, NULL */
#define CQM_ENOMEM    2   /* device allocation failed (HBM admission) */
#define CQM_ENOCONV   3   /* GMRES reached its iteration cap; outputs and info are still written */
#define CQM_ETIMEOUT  4   /* a bounded device wait gave up */
#define CQM_ECUDA     5   /* a CUDA runtime error; see cqm_bem_last_error() */
#define CQM_ECAPACITY 6   /* a fixed device capacity (rank slots, block lists) was exceeded */
#define CQM_EPENDING  7   /* a submitted request is still queued or running (cqm_bem_poll) */

/* Largest step count N: the transforms hold 24 (N + 1) bytes of twiddle and
 * R-power tables in one CTA's shared memory (at most 227 KB). */
#define CQM_MAX_STEPS 9000

/* Operator representations. */
#define CQM_MODE_DENSE  0 /* dense V_l for every solved frequency (Sec. 3.2) */
#define CQM_MODE_H2MACA 1 /* near field + H^2 far field, both MACA-compressed in frequency (eq. lrfinal) */

/* Memory kinds of caller buffers. */
#define CQM_MEM_HOST   0
#define CQM_MEM_DEVICE 1

/* Surface mesh: nv vertices (xyz, nv x 3, float64) and nt flat triangles
 * (tri, nt x 3, int32 vertex indices, outward counter-clockwise).  Copied at
 * setup; the caller's arrays may be freed afterwards. */
typedef struct cqm_mesh {
  int32_t nv;
  const double* xyz;
  int32_t nt;
  const int32_t* tri;
} cqm_mesh;

/* Optional device allocator.  alloc returns device memory of at least `bytes`
 * bytes usable on `stream` (NULL on failure); free releases it.  When absent,
 * the library uses cudaMallocAsync / cudaFreeAsync on the handle's stream. */
typedef struct cqm_allocator {
  void* ctx;
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
} cqm_allocator;

/* Parameters (cqm_params_default fills the values in brackets). */
typedef struct cqm_params {
  int32_t mode;           /* CQM_MODE_*                                   [CQM_MODE_H2MACA] */
  double R;               /* CQM radius; <= 0 means (1e-10)^(1/(2L))      [0]   */
  int32_t g_sing;         /* Gauss points per direction, singular pairs    [5]   */
  int32_t g_near;         /* Gauss points per direction, near-singular     [5]   */
  double near_ratio;      /* near-singular iff centroid distance < ratio * max longest edge [2.0] */
  int32_t n_min;          /* cluster leaf size                             [32]  */
  double eta;             /* admissibility parameter (eq. qadm)            [1.0] */
  int32_t cheb_m;         /* Chebyshev points per axis, p = m^3 (m <= 4)   [4]   */
  double aca_eps;         /* MACA stopping tolerance (Alg. 2)              [1e-6] */
  int32_t rank_cap;       /* rank slots reserved per block (1..64)         [32]  */
  int32_t gmres_restart;  /* Krylov dimension per cycle                    [50]  */
  int32_t gmres_max_iter; /* total Arnoldi steps cap                       [3000] */
  double gmres_tol;       /* residual target ||r_l|| <= tol max(||ghat_l||, 1e-6 max_k ||ghat_k||):
                             every frequency weighs the same in the time steps [1e-13] */
  int32_t profile;        /* nonzero: time every kernel launch with CUDA events [0] */
  int32_t precond;        /* H2MACA: right-precondition GMRES with the inverses of the
                             leaf diagonal near blocks, per frequency     [1]   */
  int32_t inner_fp32;     /* H2MACA: Arnoldi steps apply an FP32 copy of the operator;
                             every restart recomputes the FP64 residual,
                             so results keep FP64 accuracy                [1]   */
  double inner_rtol;      /* with inner_fp32: a cycle ends once its residual
                             estimate fell by this factor                 [1e-5] */
  int32_t tensor_cores;   /* H2MACA with inner_fp32, m = 4: far coupling of the inner
                             operator on the tcgen05 tensor cores.  1: bf16 hi/lo
                             three-product split, frequencies on the MMA rows, the
                             C factors streamed as precomputed images, d_t applied
                             to each term's TMEM accumulator; 2: TF32 three-product
                             split with d_t folded into the B operand;
                             0 = FP32 SIMT                                 [1]   */
  int32_t cache_quadrature; /* H2MACA: keep every near-field quadrature point (r and
                             weight / (4 pi r)) in device memory for the MACA
                             slices and fibres (16 bytes per point)       [1]   */
  int32_t exact_ff;       /* H2MACA: the FP64-accurate apply (residuals) runs its
                             near-field and coupling contractions in float-float
                             arithmetic (~48 bits) on the FP32 pipes, and the C
                             factors are held as float-float pairs after setup;
                             0 = FP64                                     [1]   */
  int32_t expand_near;    /* H2MACA: after the MACA, expand every near block per
                             frequency (sum_t C_t d_t, FP64 with an FP32 copy,
                             Ls x #near entries x 24 bytes) and apply the near
                             field from it, if that takes at most a quarter of
                             the device memory; 0 = apply it from the factors [1] */
  int32_t expand_far;     /* H2MACA with exact_ff: expand every far coupling per
                             frequency (sum_t C_t d_t, float-float, Ls x p^2 x 16
                             bytes per far block) for the FP64-accurate apply,
                             if that takes at most 40% of the device memory and
                             the allocation succeeds; 0 = keep it factored [1]   */
  int32_t maca_ff;        /* H2MACA with cache_quadrature: the MACA slices and fibres
                             evaluate the kernel at the cached points in float-float
                             (~47 bits) on the FP32 pipes, exp(-s r0) of each pair's
                             distance bound in FP64; 0 = FP64 throughout   [1]   */
  const cqm_allocator* allocator; /* NULL: stream-ordered CUDA pool        [NULL] */
  double tc_single_ratio; /* with tensor_cores = 1: the trailing rank terms of a far
                             block whose size ||C_t||_F |d_t(l)| is at most this
                             fraction of the largest far term at every frequency l
                             take one bf16 product (hi*hi) instead of the
                             three-product split, and their lo planes are not read;
                             the rounding of a term this small (~2^-8 of it) stays
                             below the inner operator's other errors.  Only the
                             inner iterations see it (restarts are FP64-accurate).
                             0 = three products throughout                 [1e-3] */
} cqm_params;

/* Setup product summary. */
typedef struct cqm_setup_info {
  int32_t nt, nv, N, L, Ls;     /* triangles, vertices, steps, frequencies, solved frequencies */
  int32_t mode;
  int32_t n_nodes, n_leaves;    /* cluster tree (0 in dense mode) */
  int32_t n_near, n_far;        /* blocks of the partition (0 in dense mode) */
  int64_t near_entries;         /* sum #r #c over near blocks */
  int64_t far_coupling;         /* sum p^2 over far blocks */
  int64_t rank_sum_near, rank_sum_far;
  int32_t rank_max;
  double R;
  int64_t device_bytes;         /* device memory held by the handle */
  double t_geometry_ms, t_tree_ms, t_bases_ms, t_assembly_ms; /* stage times (CUDA events) */
  int64_t near_rank_entries;    /* sum over near blocks of rank * #r * #c */
  int32_t near_expanded;        /* 1 if the near field is held expanded per frequency */
  int32_t far_expanded;         /* 1 if the far couplings of the FP64-accurate apply are */
  /* Kernel evaluations c exp(-s r) of the MACA (Alg. 2), near and far blocks:
   * every slice evaluates all quadrature points of its block at one frequency
   * (p^2 Chebyshev pairs for a far block), every fibre the points of its pivot
   * pair at all Ls frequencies.  Slices are counted exactly (the ranks times
   * the block's points); fibres with each block's mean points per pair. */
  int64_t maca_slice_evals, maca_fibre_evals;
  /* tensor_cores = 1: far rank terms that take the single-product MMAs
   * (tc_single_ratio), out of rank_sum_far */
  int64_t tc_single_terms;
} cqm_setup_info;

/* Per-solve summary. */
typedef struct cqm_solve_info {
  int32_t iterations;           /* Arnoldi steps taken (lockstep over frequencies) */
  int32_t restarts;
  int32_t converged;            /* frequencies meeting gmres_tol */
  int32_t Ls;
  double max_rel_residual;      /* max_l ||ghat_l - V_l qhat_l|| / n_l (true residual, FP64), with
                                   n_l = max(||ghat_l||, 1e-6 max_k ||ghat_k||) */
  double max_imag;              /* max |Im q_n[i]| before taking the real part */
  double t_forward_ms, t_gmres_ms, t_inverse_ms;
  /* Arnoldi work: sum over steps and active frequencies of the basis vectors
   * the step orthogonalises against (j + 1 at step j), and of 1. */
  int64_t arnoldi_vectors, arnoldi_freq_steps;
  /* FP64-accurate operator applies of the restarts after the first, in
   * frequencies: each recomputes the residual of the frequencies not converged
   * at an earlier restart. */
  int64_t restart_freq_applies;
} cqm_solve_info;

typedef struct cqm_handle cqm_handle;

/* Fill `p` with the defaults above.  Returns CQM_EINVAL for p == NULL. */
int cqm_params_default(cqm_params* p);

/* Build the operator for a mesh (Alg. 3: cluster, cluster bases, partition,
 * MACA per block -- or the dense V_l in CQM_MODE_DENSE).
 * dt > 0 time step, 1 <= N <= CQM_MAX_STEPS steps (L = N + 1 frequencies), bdf_order 1 or 2
 * (chi of BDF-k: sum_{j=1..k} (1 - z)^j / j).  cuda_stream is a cudaStream_t
 * (NULL: the legacy default stream).  On success *out owns the device state.
 * Errors: CQM_EINVAL (arguments, mesh indices, zero-area triangles),
 * CQM_ENOMEM, CQM_ECAPACITY (rank_cap exceeded), CQM_ECUDA. */
int cqm_bem_setup(const cqm_mesh* mesh, double dt, int32_t N, int32_t bdf_order,
                  const cqm_params* params, void* cuda_stream, cqm_handle** out);

/* Solve for the time-step densities.
 * rhs:     (N+1) x nt float64, row n = b_n[i] = int_{tau_i} u_inc(x, t_n) dS
 *          (Galerkin data of V q = u_inc).
 * density: (N+1) x nt float64, row n = q_n.
 * Both in `mem` memory.  info may be NULL.  Steps: forward R-scaled DFT,
 * batched GMRES over the floor(L/2)+1 solved frequencies (conjugate symmetry
 * gives the rest), inverse R-scaled DFT (eq. omega_n).
 * Errors: CQM_EINVAL, CQM_ENOCONV (results still written), CQM_ECUDA. */
int cqm_bem_solve(cqm_handle* h, const double* rhs, double* density, int32_t mem,
                  cqm_solve_info* info);

/* Solve the same problem by marching on in time, the paper's own time
 * stepping (Sec. 3.2: sum_{k<=n} Vhat_{n-k} q_k = b_n, step by step), with the
 * compressed weights: the MACA fibres are transformed to the CQM weights'
 * time index (eq. fastdft), Vhat_n = Re sum_t C_t dhat_t[n] per block, and
 * the history of each step is sum_t C_t (sum_{k<n} dhat_t[n-k] q_k) per block
 * (eq. fastrhs; far blocks through their cluster bases).  Vhat_0 is
 * assembled densely once and inverted once (FP64 blocked Gauss-Jordan; the
 * paper factorises it once by LU); each step applies its inverse.  The result
 * equals the decoupled solve of cqm_bem_solve up to O(R^L) and is exactly
 * causal.  H2MACA mode only.  The first call builds the weights (held by the
 * handle: (n_near + n_far) rank_cap L transformed fibres and M^2 doubles).
 * rhs, density: (N+1) x nt float64 in `mem` memory.  info (may be NULL):
 * iterations = N + 1 steps, t_gmres_ms = the march, t_forward_ms = the weight
 * construction of this call (0 once built).  All FP64.
 * Errors: CQM_EINVAL (NULL, dense mode), CQM_ENOMEM, CQM_ECUDA. */
int cqm_bem_solve_mot(cqm_handle* h, const double* rhs, double* density, int32_t mem,
                      cqm_solve_info* info);

/* The CQM weight Vhat_n (eq. dft) of the compressed operator as a dense
 * nt x nt float64 matrix in the caller's numbering (row-major), n = 0..N:
 * Re sum_t C_t dhat_t[n] per near block, U_r (Re sum_t C_t dhat_t[n]) U_c^T
 * per far block (eq. fastdft).  Inspection call of the marching-on-in-time
 * path.  W in `mem` memory.  Errors: CQM_EINVAL (n out of range, dense
 * mode), CQM_ENOMEM, CQM_ECUDA. */
int cqm_bem_mot_weight(cqm_handle* h, int32_t n, double* W, int32_t mem);

/* The direct formulation of the sound-soft (Dirichlet) problem (Sec. 7.2,
 * eq. cqmdir; Sec. 2.2 for the double layer K), decoupled in frequency as in
 * the Remark of Sec. 6.2: V_l qhat_l = (-1/2 M + K_l) ghat_l with M the P0
 * mass matrix diag |tau_i|, then the inverse transform.  g: (N+1) x nt float64,
 * row n = the P0 (L^2-projection) coefficients of the Dirichlet data at t_n;
 * q: (N+1) x nt float64, the Neumann data (normal derivative along the outward
 * normal).  Both in `mem` memory.  K_l has the single layer's quadrature rules
 * (test i, trial j, no symmetrisation; identical pairs vanish on flat
 * triangles); its near field is evaluated once per solved frequency (held by
 * the handle after the first call: near entries x Ls complex), its far field
 * is U_r S_b W_c^T with the single layer's compressed couplings and the column
 * basis W_c = int n . grad L_c.  The solve is the single layer's batched GMRES
 * (info as for cqm_bem_solve).  H2MACA mode only.
 * Errors: CQM_EINVAL, CQM_ENOMEM, CQM_ENOCONV (results written), CQM_ECUDA. */
int cqm_bem_solve_dirichlet(cqm_handle* h, const double* g, double* q, int32_t mem,
                            cqm_solve_info* info);

/* y_l = K_l x_l for the Ls solved frequencies (the double layer of
 * cqm_bem_solve_dirichlet).  x, y: Ls x nt complex in `mem` memory. */
int cqm_bem_apply_double_layer(cqm_handle* h, const double* x, double* y, int32_t mem);

/* Galerkin matrices with piecewise linear functions for mixed boundary
 * conditions (Sec. 2.3 eq. wavegalform; the matrices K_l, K'_l, D_l of
 * Sec. 3.2 with the spaces of constants per triangle and of vertex hats),
 * dense, at the Ls solved frequencies of the handle:
 *   K1[l][m][v] = <phi0_m, K_l phi1_v>   (Ls x nt x nv), double layer, P1 trial;
 *   Kp[l][v][i] = <phi1_v, K'_l phi0_i>  (Ls x nv x nt), adjoint double layer;
 *   D[l][u][v]  = <phi1_u, D_l phi1_v>   (Ls x nv x nv), hypersingular operator in
 *                 Maue's form int int G [curl phi_u . curl phi_v + s^2 (n_x . n_y) phi_u phi_v].
 * Complex, interleaved (re, im) float64, row-major, in `mem` memory, owned by
 * the caller; overwritten.  The single layer's quadrature rules (test
 * triangle first, no symmetrisation), outward normals of counter-clockwise
 * triangles, FP64.  Dense: O(nt^2 Ls) work and the sizes above (meant for
 * small meshes and checks).  Either mode.
 * Errors: CQM_EINVAL (NULL, mem), CQM_ENOMEM (host-memory outputs need device
 * staging of the same size), CQM_ECUDA. */
int cqm_bem_p1_matrices(cqm_handle* h, double* K1, double* Kp, double* D, int32_t mem);

/* Mixed boundary conditions (Sec. 2.3 eq. wavegalform; Sec. 3.2 eq.
 * cqmgalapx, decoupled in frequency like cqm_bem_solve): Dirichlet data on the
 * triangles with dmask[m] != 0 (Gamma_D), Neumann data on the others
 * (Gamma_N).  dmask: nt int32 (host).  gD: (N+1) x nv float64, vertex values
 * of the Dirichlet data (only the vertices of Gamma_D's triangles are used);
 * gN: (N+1) x nt float64, P0 coefficients of the Neumann data (only Gamma_N's
 * triangles are used).  Results: q (N+1) x nt, the Neumann data on Gamma_D
 * (0 on Gamma_N); u (N+1) x nv, the Dirichlet data in the hats of the
 * vertices that touch no Gamma_D triangle (0 at the others).  All in `mem`
 * memory.  Per solved frequency the dense system
 *   [ V_DD -K1_DN ; Kp_ND D_NN ] [qhat ; uhat] =
 *   [ (-1/2 I + K1) gDhat - V gNhat ; (-1/2 I' - Kp) gNhat - D gDhat ]
 * (the matrices of cqm_bem_p1_matrices, I the P0 x P1 mass matrix) by
 * Gaussian elimination with partial pivoting on the GPU, then the inverse
 * transform.  CQM_MODE_DENSE only (the dense V_l).
 * Errors: CQM_EINVAL (NULL, mem, not the dense mode, no unknowns), CQM_ENOMEM,
 * CQM_ECUDA. */
int cqm_bem_solve_mixed(cqm_handle* h, const int32_t* dmask, const double* gD, const double* gN, double* q,
                        double* u, int32_t mem);

/* Galerkin data of the plane-wave pulse u(x,t) = exp(-((t - delay - d.x)/width)^2)
 * at t_n = n dt, n = 0..N, with Radon's 7-point rule per triangle.
 * dir: 3 doubles (host, normalised inside).  rhs: (N+1) x nt float64 in `mem`. */
int cqm_bem_rhs_plane_wave(cqm_handle* h, const double dir[3], double width, double delay,
                           double* rhs, int32_t mem);

/* Time limit, in nanoseconds, of every bounded device wait of the handle's
 * pipelined kernels (the mbarrier waits of the tensor-core far coupling);
 * 0 restores the default of one second.  A wait that runs out makes its
 * kernel record the expiry, stop issuing work, let what it issued finish,
 * free its tensor memory and return; the GMRES loop stops at its next check
 * and the call returns CQM_ETIMEOUT (cqm_bem_last_error names the limit).
 * The handle stays usable: the next call starts with the expiry cleared.
 * expire_next != 0 arms a one-shot check of that path: in the next launch of
 * the pipelined kernel one thread first waits on a barrier that nothing
 * completes, so that this wait runs out after `ns` (nothing faults or hangs;
 * the expiry is reported as above).
 * Errors: CQM_EINVAL (NULL, ns < 0).  (Sec. 6.2 names no device waits; this
 * is the failure path of the solver's pipelined kernels.) */
int cqm_bem_set_wait_limit(cqm_handle* h, int64_t ns, int32_t expire_next);

/* Release everything the handle owns.  NULL is accepted. */
int cqm_bem_destroy(cqm_handle* h);

/* Static description of a status code. */
const char* cqm_bem_strerror(int status);

/* Detail of the last failure on this thread ("" if none). */
const char* cqm_bem_last_error(void);

/* ---- Inspection calls (host outputs; used to check each step) ---------- */

/* Summary of the setup product. */
int cqm_bem_get_info(const cqm_handle* h, cqm_setup_info* out);

/* The L frequencies s_l (eq. cqm_freq): out = 2 L doubles (re, im). */
int cqm_bem_get_frequencies(const cqm_handle* h, double* out);

/* Cluster tree (Def. 2), nodes numbered breadth-first.  Any output may be
 * NULL.  perm: nt int32 (triangle at each position); begin/end/son0/son1/level:
 * n_nodes int32 (son = -1 for leaves); lo/hi: n_nodes x 3 float64 boxes. */
int cqm_bem_get_tree(const cqm_handle* h, int32_t* perm, int32_t* begin, int32_t* end,
                     int32_t* son0, int32_t* son1, int32_t* level, double* lo, double* hi);

/* Block partition (Defs. 3-4): near (n_near x 2) and far (n_far x 2) cluster
 * pairs sorted by (row, column); ranks of their MACA factors. Any may be NULL. */
int cqm_bem_get_blocks(const cqm_handle* h, int32_t* near_rc, int32_t* far_rc,
                       int32_t* near_rank, int32_t* far_rank);

/* MACA factors of one block (eq. maca): kind 0 = near, 1 = far; b = index in
 * the sorted list.  C: rank x rows x cols complex (rows/cols in tree order:
 * triangles perm[begin..end) for near blocks, Chebyshev multi-indices for far
 * blocks); D: rank x Ls complex (D[t][l] = d_t[l]).  Either may be NULL.
 * With exact_ff the C entries are returned as hi + lo of their float-float
 * pairs (about 48 significant bits of the FP64 values the MACA computed). */
int cqm_bem_get_block_factors(const cqm_handle* h, int32_t kind, int32_t b,
                              int32_t* rank, int32_t* rows, int32_t* cols,
                              double* C, double* D);

/* Galerkin entries V_l[I[k], J[k]] computed directly by the quadrature
 * kernel at the frequencies l = freq[f] (0 <= freq[f] < L).
 * out: npairs x nfreq complex.  I, J, freq, out in `mem` memory. */
int cqm_bem_entries(cqm_handle* h, int64_t npairs, const int32_t* I, const int32_t* J,
                    int32_t nfreq, const int32_t* freq, double* out, int32_t mem);

/* Apply the handle's operator: y_l = V_l x_l for the Ls solved frequencies.
 * x, y: Ls x nt complex in `mem` memory (row l = frequency l). */
int cqm_bem_apply(cqm_handle* h, const double* x, double* y, int32_t mem);

/* Apply the operator of the inner GMRES iterations (the FP32 copy of the
 * compressed operator when inner_fp32 is on; otherwise the same as
 * cqm_bem_apply).  x, y: Ls x nt complex in `mem` memory. */
int cqm_bem_apply_inner(cqm_handle* h, const double* x, double* y, int32_t mem);

/* Solve V_l qhat_l = ghat_l for the Ls solved frequencies (batched GMRES).
 * ghat, qhat: Ls x nt complex in `mem` memory. */
int cqm_bem_solve_frequencies(cqm_handle* h, const double* ghat, double* qhat, int32_t mem,
                              cqm_solve_info* info);

/* R-scaled transforms alone: forward ghat_l = sum_n R^n b_n zeta^{n l}
 * ((N+1) x nt real -> Ls x nt complex) and inverse (eq. omega_n, with
 * conjugate symmetry; Ls x nt complex -> (N+1) x nt real). */
int cqm_bem_forward_transform(cqm_handle* h, const double* b, double* ghat, int32_t mem);
int cqm_bem_inverse_transform(cqm_handle* h, const double* qhat, double* q, int32_t mem);

/* ---- Kernel timing ------------------------------------------------------ */

/* Kernel classes timed by the profiler (index into cqm_bem_profile_read). */
#define CQM_K_GEOMETRY       0
#define CQM_K_TREE           1
#define CQM_K_PARTITION      2
#define CQM_K_BASES          3    /* cluster bases, FP32 and float-float factor copies */
#define CQM_K_DENSE_ASSEMBLE 4
#define CQM_K_ENTRIES        5
#define CQM_K_MACA_SLICE     6
#define CQM_K_MACA_PIVOT     7
#define CQM_K_MACA_FIBRE     8
#define CQM_K_MACA_FINALIZE  9
#define CQM_K_NEAR_APPLY     10   /* near field of the inner (FP32) apply, or of the FP64 apply without inner_fp32 */
#define CQM_K_LEAF_FORWARD   11
#define CQM_K_UPSWEEP        12
#define CQM_K_FAR_COUPLING   13   /* far coupling of the inner (FP32) apply, or of the FP64 apply without inner_fp32 */
#define CQM_K_DOWNSWEEP      14
#define CQM_K_LEAF_BACKWARD  15
#define CQM_K_DENSE_APPLY    16
#define CQM_K_ARNOLDI        17
#define CQM_K_GMRES_OTHER    18
#define CQM_K_FORWARD_DFT    19
#define CQM_K_INVERSE_DFT    20
#define CQM_K_RHS            21
#define CQM_K_PRECOND        22
#define CQM_K_NEAR_EXACT     23   /* near field of the FP64-accurate apply (residuals) */
#define CQM_K_FAR_EXACT      24   /* far coupling of the FP64-accurate apply (residuals) */
#define CQM_K_EXPAND         25   /* expanded tables and tensor-core operand images (setup) */
#define CQM_K_POINTS         26   /* near-field quadrature point cache and far kernel points (setup) */
#define CQM_K_MOT_WEIGHTS    27   /* marching on in time: transformed fibres, Vhat_0 and its inverse */
#define CQM_K_MOT_HISTORY    28   /* marching on in time: history sum of each step (near and far) */
#define CQM_K_MOT_STEP       29   /* marching on in time: step solve, H2 transforms of the new density */
#define CQM_K_DL_SETUP       30   /* double layer: near-field table and leaf column basis */
#define CQM_K_DL_APPLY       31   /* double layer: near field of an apply (the far field counts as H2 steps) */
#define CQM_K_COUNT          32

/* Turn per-launch event timing on (nonzero) or off; either way the counters
 * are reset.  Timing adds one event pair per launch on the handle's stream. */
int cqm_bem_profile(cqm_handle* h, int32_t enable);

/* Launch counts and summed device time (ms, CUDA events on the launching
 * stream) of the first n kernel classes since the last reset; synchronises
 * the stream.  launches and total_ms hold n entries each. */
int cqm_bem_profile_read(cqm_handle* h, int32_t n, int64_t* launches, double* total_ms);

/* Name of a kernel class ("" when out of range). */
const char* cqm_bem_kernel_name(int32_t id);

/* ---- Cluster tree without device allocation ----------------------------- */

/* The paper has no counterpart to this call; it exists for callers of this
 * library that may not call cudaMalloc (code inside another runtime that
 * reserved the device memory up front, code on a path where an allocation,
 * which can synchronise the device, is not allowed, or code whose memory is
 * partitioned at start-up).
 *
 * Builds the same cluster tree as cqm_bem_setup (same splitting rule and
 * breadth-first numbering) for a mesh already in device memory, without
 * allocating: the kernel's scratch lives in a fixed array of about 2.3 MB
 * that the library reserves on every GPU that loads it, for the life of the
 * process.  Meshes of at most CQM_TREE_NOALLOC_MAX_TRIANGLES triangles;
 * larger ones are rejected with CQM_EINVAL.
 *
 * xyz: nv x 3 float64, tri: nt x 3 int32 (device).  Outputs (device, owned by
 * the caller): perm (nt), and per node begin, end, son0, son1 (-1 for
 * leaves), parent (-1 for the root), level, each with room for 2 nt - 1
 * entries, lo and hi (3 per node).  n_nodes (host) receives the node count.
 * cuda_stream: a cudaStream_t (NULL: the legacy default stream); the call
 * synchronises it before returning.
 *
 * The first call on a device looks the scratch address up (once per device,
 * with that device current); make that first call before any stream capture.
 * The address is kept for the life of the process: it assumes the device's
 * primary context is not torn down in between (after a cudaDeviceReset on
 * that device the cached address is stale and must not be used).
 * Work: one CTA of 1024 threads builds the whole tree.  A node whose
 * centroids all fall on one side of its box midpoint is split at the median,
 * ranking each element against the whole node (quadratic in the node size),
 * so a degenerate mesh near the size limit can keep one SM busy for seconds.
 * Every call shares the one scratch array per device, so calls whose work
 * overlaps on the GPU (other threads, other streams) race: serialise them.
 * Errors: CQM_EINVAL (NULL, sizes, vertex indices out of range -- checked on
 * the device before any indexed read), CQM_ECUDA. */
#define CQM_TREE_NOALLOC_MAX_TRIANGLES 65536
int cqm_cluster_tree_noalloc(const double* xyz, int32_t nv, const int32_t* tri, int32_t nt,
                             int32_t n_min, int32_t* perm, int32_t* begin, int32_t* end,
                             int32_t* son0, int32_t* son1, int32_t* parent, int32_t* level,
                             double* lo, double* hi, int32_t* n_nodes, void* cuda_stream);

/* ---- Serving: many scattering problems on one GPU ---------------------- */

/* The decoupled solve treats each frequency independently (Sec. 6.2), and
 * each scattering problem is independent of the others; a server runs many
 * problems concurrently on one GPU.  Each worker thread owns a CUDA stream and
 * runs setup (Alg. 3) and solve of one request at a time, so requests that
 * arrive while others are on the GPU start as soon as a worker and device
 * memory are free, and their kernels overlap on the device.  Requests are
 * admitted by their estimated device footprint (cqm_bem_estimate_bytes)
 * against the server's byte budget, first fit in arrival order; a request
 * runs with the same kernels and parameters it would have alone, so its
 * result is the same alone and in the mix.  Device memory comes from the
 * stream-ordered CUDA pool (a request's params.allocator is ignored). */
typedef struct cqm_server cqm_server;

/* One scattering problem.  mesh, rhs: copied at submit.  rhs: (N+1) x nt
 * host float64 Galerkin data, or NULL to use the plane-wave pulse
 * (dir, width, delay as in cqm_bem_rhs_plane_wave).  params: NULL = defaults
 * with expand_far = 0 (the expanded far table trades a large footprint for a
 * faster residual; a server favours concurrency). */
typedef struct cqm_request {
  cqm_mesh mesh;
  double dt;
  int32_t N, bdf_order;
  const cqm_params* params;
  const double* rhs;
  double dir[3];
  double width, delay;
} cqm_request;

/* Result of a request (filled by cqm_bem_poll). */
typedef struct cqm_result_info {
  int32_t status;               /* status of setup and solve */
  int32_t worker;               /* worker thread that ran it */
  int64_t bytes_estimate;       /* reserved at admission */
  int64_t device_bytes;         /* held by the handle after setup */
  double t_queue_ms;            /* submit -> admitted */
  double t_setup_ms, t_solve_ms;
  double t_total_ms;            /* submit -> done */
  cqm_solve_info solve;
} cqm_result_info;

/* Upper estimate of the device memory of a request: every rank slot of the
 * factors, their FP32 and bf16 copies, the quadrature point cache of the
 * setup, the preconditioner, the solver workspace and the expanded tables the
 * setup would admit.  Per triangle it uses bounds of the partition of closed
 * surfaces with leaves of n_min triangles (at most 1000 near-field entries
 * and 2.5 far blocks per triangle).  Errors: CQM_EINVAL. */
int cqm_bem_estimate_bytes(int32_t nt, int32_t N, const cqm_params* params, int64_t* bytes);

/* workers >= 1 threads on the current device; byte_budget > 0 bytes of
 * device memory for admitted requests, or 0 for 90% of the free memory.
 * Errors: CQM_EINVAL, CQM_ECUDA. */
int cqm_server_create(int32_t workers, int64_t byte_budget, cqm_server** out);

/* Queue a request; *ticket identifies it.  Returns CQM_ENOMEM (and queues
 * nothing) when its estimate exceeds the whole budget, CQM_EINVAL for bad
 * arguments (checked as in cqm_bem_setup). */
int cqm_bem_submit(cqm_server* s, const cqm_request* req, int64_t* ticket);

/* Result of a request.  wait = 0 returns CQM_EPENDING while it is queued or
 * running; wait != 0 blocks until it is done.  When done: density (host,
 * (N+1) x nt, may be NULL) and info (may be NULL) are filled, the request is
 * released, and the return value is its status.  Unknown ticket: CQM_EINVAL. */
int cqm_bem_poll(cqm_server* s, int64_t ticket, int32_t wait, double* density, cqm_result_info* info);

/* Bytes reserved by admitted requests now, and requests queued or running. */
int cqm_server_load(cqm_server* s, int64_t* bytes_in_use, int32_t* queued, int32_t* running);

/* Wait for every submitted request, stop the workers and free the server
 * (results not polled are dropped).  NULL is accepted. */
int cqm_server_destroy(cqm_server* s);

#ifdef __cplusplus
}
#endif
#endif /* CQM_BEM_H */
