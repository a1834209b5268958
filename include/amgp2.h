/*
 * amgp2 -- graph-based algebraic multigrid for hierarchical-P2 finite element
 * systems (H. Yang, arXiv:1503.01287), single-GPU CUDA implementation.
 *
 * The library solves the linear systems of Sec. 2.4 of the paper,
 *   SPD (Eq. ellipticeqn):    A u = f,   A = [K_ll K_ql^T; K_ql K_qq]
 *   saddle (Eq. mixedeqn):    [A B^T; B -C] [u; p] = [f; g]
 * with the AMG of Sec. 3 (Algorithm 1; coarsening on the separate graphs of
 * K_ll and K_qq, Sec. 3.2; prolongation P = diag(I, J[, H]), Eqs.
 * disprolongmat / mixprolongmat; Galerkin coarse operators P^T K P; block
 * Jacobi / block Gauss-Seidel / segregated Gauss-Seidel smoothers, Sec. 3.3)
 * as the preconditioner of CG (SPD) or flexible GMRES (saddle), stopping on
 * ||b - K x_k||_2 / ||b||_2 <= tol from x_0 = 0 (Sec. 4.2).
 *
 * Conventions shared by every entry point:
 *  - Unknowns are grouped in nodes of 3 components (u_x, u_y, u_z), stored
 *    interleaved: unknown 3*i + c is component c of node i.  Nodes are ordered
 *    vertices ("linear" DOF) before edges ("quadratic" DOF), Eq. ellipticeqn.
 *  - A is 3x3-block CSR: a_rowptr[n_nodes+1], a_col[nnzb] (ascending within a
 *    row, diagonal block present), a_val[9*nnzb] with each block row-major.
 *    Its pattern is the structural one (node pairs sharing an element), kept
 *    even where values are zero: coarsening and colouring read only the pattern.
 *  - B (saddle kinds) is 1x3-block CSR with one row per pressure unknown:
 *    b_rowptr[n_pres+1], b_col[b_nnz] (velocity node ids), b_val[3*b_nnz].
 *  - C (saddle kinds) is scalar CSR n_pres x n_pres; its pattern is the P1
 *    (vertex) graph and is required also for Stokes, where its values are 0.
 *  - Dirichlet nodes are identity rows of A with zero off-diagonal blocks in
 *    their row and column and zero right-hand side (tag AMG_NODE_DIRICHLET).
 *  - Return codes: AMG_OK (0) on success, AMG_NOT_CONVERGED (1) when the
 *    iteration limit is reached (x then holds the last iterate, stats are
 *    filled), negative values on errors; amg_last_error() gives the message.
 *  - Nothing is thrown across the ABI.  All calls are host calls; device
 *    work is ordered on the CUDA stream given to amg_setup.
 */
#ifndef AMGP2_H
#define AMGP2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- enums */

/* Problem kinds of Sec. 2.1: Eqs. veclap, elasdis, elasmix, stokesmix. */
enum amg_kind {
  AMG_VECTOR_LAPLACE = 0,
  AMG_ELASTICITY = 1,
  AMG_MIXED_ELASTICITY = 2,
  AMG_STOKES = 3
};

/* Node tags (Sec. 2.3: vertex DOF of V_L, edge DOF of V_Q); bit-or Dirichlet. */
enum amg_node_tag {
  AMG_NODE_VERTEX = 0,
  AMG_NODE_EDGE = 1,
  AMG_NODE_DIRICHLET = 0x10
};

/* Smoothers of Sec. 3.3. */
enum amg_smoother {
  AMG_SMOOTHER_GS = 0,      /* symmetric multicolour 3x3-block Gauss-Seidel     */
  AMG_SMOOTHER_JACOBI = 1,  /* damped 3x3-block Jacobi (omega, default 0.5)     */
  AMG_SMOOTHER_SGS = 2,     /* segregated Gauss-Seidel for saddle systems       */
  AMG_SMOOTHER_BS = 3,      /* Braess-Sarazin type for saddle systems, Eqs.
                               (bssm) / (bssmpre): x += K^{-1} (b - K x) with
                               K^ = [A^ B^T; B B A^{-1} B^T - S^], A^ = 2 diag(A),
                               S^{-1} one V(1,1)-cycle (damped scalar Jacobi 0.5)
                               of the graph AMG on S = C + B A^{-1} B^T through
                               the pressure prolongations H, direct solve on the
                               coarsest pressure level                          */
  AMG_SMOOTHER_VANKA = 4    /* multiplicative Vanka, Eq. (locpatchsm): patch k =
                               pressure unknown k and the velocity nodes of row
                               k of B; x += omega [A_k B_k^T; B_k -C_kk]^{-1} r_k
                               (omega 0.7) over the patches of one colour of the
                               patch overlap graph, residual updated between
                               colours (ascending before, descending after the
                               coarse correction); at most 512 unknowns a patch */
};

enum amg_precision {
  AMG_FP64 = 0,             /* cycle in FP64                                    */
  AMG_FP32 = 1,             /* cycle in FP32, outer Krylov and coarsest in FP64
                               (the Krylov operator products in FP32 pairs by
                               default, amg_options.outer_pair)                 */
  AMG_FP32_BF16 = 2,        /* AMG_FP32 with the operator values of levels >= 1
                               stored in BF16 (rounded to nearest even from the
                               FP64 Galerkin values, converted to FP32 in the
                               kernels); level 0, D^{-1}, P and the pressure
                               parts stay FP32                                  */
  AMG_FP32_PAIR = 3         /* not a cycle precision: amg_level_apply and
                               amg_time_level_op on level 0 of an FP32 handle
                               with outer_pair run the Krylov operator's
                               FP32-pair kernel (see amg_options.outer_pair;
                               amg_level_apply adds the saddle blocks in FP64) */
};

enum amg_krylov {
  AMG_KRYLOV_AUTO = 0,      /* PCG (FP64 cycle) / flexible CG (FP32 cycle) for
                               SPD kinds, flexible GMRES for saddle kinds      */
  AMG_KRYLOV_PCG = 1,
  AMG_KRYLOV_FCG = 2,
  AMG_KRYLOV_FGMRES = 3,
  AMG_KRYLOV_NONE = 4       /* stand-alone AMG: repeated Algorithm 1            */
};

enum amg_status {
  AMG_OK = 0,
  AMG_NOT_CONVERGED = 1,
  AMG_ERR_INVALID = -1,     /* bad argument or malformed matrix                 */
  AMG_ERR_CUDA = -2,        /* a CUDA call failed                               */
  AMG_ERR_BREAKDOWN = -3,   /* zero/NaN pivot or non-finite residual            */
  AMG_ERR_TIMEOUT = -4,     /* a bounded device loop hit its limit              */
  AMG_ERR_NOMEM = -5,       /* device allocation failed                         */
  AMG_ERR_UNSUPPORTED = -6  /* option combination not provided                  */
};

/* --------------------------------------------------------------- structs */

typedef struct amg_matrix {
  int32_t n_nodes;          /* velocity nodes; 3 unknowns each                  */
  int32_t n_pres;           /* pressure unknowns; 0 for the SPD kinds           */
  int64_t nnzb;             /* 3x3 blocks of A                                  */
  const int32_t* a_rowptr;
  const int32_t* a_col;
  const double* a_val;      /* 9 * nnzb, row-major blocks                       */
  int64_t b_nnz;
  const int32_t* b_rowptr;
  const int32_t* b_col;
  const double* b_val;      /* 3 * b_nnz                                        */
  int64_t c_nnz;
  const int32_t* c_rowptr;
  const int32_t* c_col;
  const double* c_val;
  int32_t device_ptrs;      /* 1: all arrays (and node_tags) are device memory  */
} amg_matrix;

typedef struct amg_options {
  int32_t smoother;         /* amg_smoother; default GS (SPD) / SGS (saddle)    */
  int32_t m_pre;            /* pre-smoothing steps, Algorithm 1 (default 1)     */
  int32_t m_post;           /* post-smoothing steps (default 1)                 */
  int32_t nu;               /* recursive calls per level: 1 V-cycle, 2 W-cycle  */
  int32_t cycles;           /* cycles per preconditioner application (1 or 2)   */
  int32_t precision;        /* amg_precision (default FP64)                     */
  int32_t krylov;           /* amg_krylov (default AUTO)                        */
  int32_t max_levels;       /* levels 0..max_levels-1 (default 5)               */
  int32_t coarse_dofs;      /* stop coarsening at <= this many unknowns (300)   */
  int32_t gmres_restart;    /* FGMRES(m) restart length (default 50, at most 318) */
  int32_t separate;         /* 1: separate K_ll / K_qq graphs (Sec. 3.2.1);
                               0: graph of the whole matrix (Table 2, row 3)    */
  int32_t max_iterations;   /* Krylov iteration limit (default 1000)            */
  int32_t use_graphs;       /* 1: replay each Krylov iteration as a CUDA graph  */
  int32_t cluster_from;     /* coarse levels from this level down run as one
                               thread-block-cluster launch: -1 chosen by timing
                               at setup (default), 0 never, k >= 1 from level k */
  int32_t cycle_kernel;     /* 0: chosen by timing at setup (default); 1: one
                               launch per operation (with the cluster levels);
                               2: the whole cycle as one persistent cooperative
                               launch with grid barriers.  With the Vanka
                               smoother both are forced to per-operation
                               launches (cluster_from 0, cycle_kernel 1)        */
  double omega;             /* block Jacobi damping (default 0.5)               */
  double omega_p;           /* sGS pressure step omega (default 0.125)          */
  int32_t batch_tile;       /* amg_solve_batched: tile of the SpMM row kernels
                               and of the colour kernels, -1 chosen per level by
                               timing the SpMM (default; the colour kernels take
                               the same tile); t =
                               0..7 forces (lane groups per row, blocks
                               unrolled) = (1,2), (2,2), (1,4), (2,4), (4,2),
                               (8,2), (4,4), (8,4) on the colour kernels and
                               tile t mod 4 on the SpMM row kernels             */
  int32_t gs_cluster;       /* multicolour Gauss-Seidel sweep of a level whose
                               iterate, right-hand side and row offsets fit in
                               shared memory (SPD kinds, up to about 5000 nodes
                               in FP32, 2800 in FP64): -1
                               chosen per level by timing at setup (default),
                               0 one launch per colour, k = 1, 2, 4, 8 or 16:
                               the whole sweep in one cluster of k CTAs         */
  int32_t outer_pair;       /* FP32-cycle Krylov solves (CG for SPD kinds, the
                               velocity block of FGMRES for saddle kinds, whose
                               B and C parts stay FP64): 1 (default)
                               the Krylov operator products K p in FP32-pair
                               arithmetic -- every FP64 value and direction entry
                               held as two floats hi + lo, each product formed
                               exactly with an FMA, sums compensated (TwoSum),
                               about 2^-48 relative while the values and the
                               direction's entries lie between about 1e-30 and
                               1e38 in magnitude; 0 in FP64.  The residual
                               reported at exit is always recomputed in FP64     */
  int32_t post_order;       /* colour order of the post-smoothing sweeps of the
                               Gauss-Seidel and Vanka smoothers: -1 (default)
                               the pre-smoothing (ascending) order for the
                               stand-alone AMG iteration (krylov =
                               AMG_KRYLOV_NONE; Sec. 4.2, Tables 4 and 8) and
                               the reverse (descending) order for the Krylov
                               methods, which keeps the preconditioner
                               symmetric for CG; 0 reverse; 1 same           */
  int32_t gs_flow;          /* multicolour Gauss-Seidel sweep of a coloured level
                               as one cooperative launch in dataflow order (each
                               row waits on per-node flags of the neighbours it
                               reads new values from): -1 chosen per level by
                               timing at setup (default), 0 never, 1 on every
                               coloured level with the lanes per row of the
                               one-launch-per-colour kernel (bitwise its
                               results)                                       */
  int32_t gs_stream;        /* one-launch-per-colour Gauss-Seidel kernels as
                               grid-stride loops over a grid of k CTAs per SM,
                               each warp loading its next rows' blocks while it
                               updates the current ones: -1 k and the lanes per
                               row chosen per level by timing at setup
                               (default; 0 where one group of lanes per row is
                               faster), 0 never, k = 1..8 forced (lanes per
                               row as tuned for the chain)                     */
  int32_t gs_tma;           /* FP32 one-launch-per-colour Gauss-Seidel kernel
                               with the block values and columns of a CTA's rows
                               staged in shared memory by bulk (TMA) copies
                               issued before the wait on the previous colour:
                               -1 with its lanes per row where it beats the
                               register-prefetch kernel, chosen per level by
                               timing at setup (default), 0 never, 1 on every
                               coloured FP32 level with the chain's lanes per
                               row (bitwise its results)                       */
} amg_options;

#define AMG_MAX_LEVELS 8

typedef struct amg_stats {
  int32_t iterations;       /* Krylov iterations (operator applications)       */
  int32_t converged;
  int32_t n_levels;
  int32_t pad0;
  double rel_residual;      /* recursive residual estimate at exit              */
  double true_rel_residual; /* ||b - K x|| / ||b|| recomputed at exit           */
  double setup_ms;
  double solve_ms;
  int64_t kernel_launches;  /* kernels launched by the last amg_solve           */
  int32_t level_nodes[AMG_MAX_LEVELS];
  int32_t level_pres[AMG_MAX_LEVELS];
  int64_t level_nnzb[AMG_MAX_LEVELS];
  int32_t level_colours[AMG_MAX_LEVELS];
  int32_t level_group[AMG_MAX_LEVELS];  /* lanes per block row chosen at setup       */
  int32_t cluster_from;     /* cycle variant in use: first level of the cluster
                               sub-cycle (0: none)                              */
  int32_t cycle_kernel;     /* 1: one launch per operation, 2: persistent cycle */
  int32_t level_gs_cluster[AMG_MAX_LEVELS];  /* CTAs of the one-cluster sweep
                               (0: one launch per colour)                       */
  int32_t level_gs_flow[AMG_MAX_LEVELS];     /* lanes per row of the one-launch
                               dataflow sweep (0: not used on the level)        */
  int32_t level_gs_stream[AMG_MAX_LEVELS];   /* CTAs per SM of the grid-stride
                               colour kernel (0: one group of lanes per row)    */
  int32_t level_gs_tma[AMG_MAX_LEVELS];      /* 1: the level's colour kernel is
                               the TMA-staged one                               */
} amg_stats;

typedef struct amg_level_info {
  int32_t n_nodes;
  int32_t n_pres;
  int64_t nnzb;
  int64_t p_nnz;            /* entries of the node prolongation to level+1      */
  int64_t h_nnz;            /* entries of the pressure prolongation             */
  int64_t b_nnz;
  int64_t c_nnz;
  int32_t n_colours;
  int32_t is_coarsest;
} amg_level_info;

/* What amg_level_copy returns (always to host memory). */
enum amg_level_item {
  AMG_Q_A_ROWPTR = 0,   /* int32  [n_nodes+1]                                   */
  AMG_Q_A_COL = 1,      /* int32  [nnzb]                                        */
  AMG_Q_A_VAL = 2,      /* double [9*nnzb], row-major blocks                    */
  AMG_Q_TAGS = 3,       /* int32  [n_nodes]                                     */
  AMG_Q_CF_STATE = 4,   /* int32  [n_nodes]  1 = C, 2 = F (not on coarsest)     */
  AMG_Q_P_ROWPTR = 5,   /* int32  [n_nodes+1]                                   */
  AMG_Q_P_COL = 6,      /* int32  [p_nnz]   coarse node ids                     */
  AMG_Q_P_VAL = 7,      /* double [p_nnz]   node weights (x I_3)                */
  AMG_Q_COLOUR = 8,     /* int32  [n_nodes] greedy colour of each node          */
  AMG_Q_DINV = 9,       /* double [9*n_nodes] inverses of diagonal blocks       */
  AMG_Q_B_ROWPTR = 10,  /* int32  [n_pres+1]                                    */
  AMG_Q_B_COL = 11,
  AMG_Q_B_VAL = 12,     /* double [3*b_nnz]                                     */
  AMG_Q_C_ROWPTR = 13,
  AMG_Q_C_COL = 14,
  AMG_Q_C_VAL = 15,
  AMG_Q_PCF_STATE = 16, /* int32 [n_pres] pressure C/F state                    */
  AMG_Q_H_ROWPTR = 17,
  AMG_Q_H_COL = 18,
  AMG_Q_H_VAL = 19,
  AMG_Q_COARSE_INV = 20, /* double [m*m] generalised inverse of the coarsest K,
                           m = 3*n_nodes + n_pres (coarsest level only)         */
  AMG_Q_S_ROWPTR = 21,  /* int32 [n_pres+1] Braess-Sarazin S = C + B A^{-1} B^T
                           of the level (non-coarsest saddle levels, smoother
                           AMG_SMOOTHER_BS); its nnz is S_ROWPTR[n_pres]        */
  AMG_Q_S_COL = 22,
  AMG_Q_S_VAL = 23      /* double [nnz]                                         */
};

typedef struct amg_handle amg_handle;

/* ------------------------------------------------------------ entry points */

/* Fills *opt with the defaults listed in amg_options. */
void amg_default_options(amg_options* opt);

/*
 * amg_setup -- the AMG setup phase of Sec. 3.2 on the GPU.
 *
 * Copies A (and B, C) to the device, then per level: coarsening graph (K_ll and
 * K_qq patterns, or the whole pattern when opt->separate = 0; the P1 pattern of
 * C for the pressure), greedy maximal independent set in increasing node index
 * (C/F split), prolongation rows (C: 1, F: 1/k on its k C-neighbours, Eqs.
 * disprolongmat / mixprolongmat), Galerkin product P^T K P, first-fit greedy
 * colouring in increasing node index, inverses of the 3x3 diagonal blocks.
 * Coarsening stops when a level has <= opt->coarse_dofs unknowns or
 * opt->max_levels levels exist; the coarsest matrix is factorised by LU with
 * complete pivoting stopped at its numerical rank (Algorithm 1, step 6).
 *
 *   mat        the system; all arrays host or all device (mat->device_ptrs).
 *   node_tags  int32 [n_nodes], amg_node_tag values; same memory kind as mat.
 *   kind       amg_kind.
 *   opt        options, or NULL for the defaults.
 *   stream     cudaStream_t; NULL makes the handle create and own a stream.
 *   out        receives the new handle; NULL on failure.
 * Ownership: inputs are copied; the caller keeps its arrays.  The handle owns
 * every device allocation and is released with amg_free.
 * Errors: AMG_ERR_INVALID for malformed input (missing diagonal block, column
 * out of range, non-finite values), AMG_ERR_NOMEM, AMG_ERR_CUDA,
 * AMG_ERR_TIMEOUT (a bounded setup loop hit its limit).
 */
int amg_setup(const amg_matrix* mat, const int32_t* node_tags, int32_t kind,
              const amg_options* opt, void* stream, amg_handle** out);

/*
 * amg_solve -- solve K x = b to ||b - K x||_2 / ||b||_2 <= rel_tol from x = 0
 * (stopping rule of Sec. 4.2) with AMG-preconditioned CG / flexible CG (SPD
 * kinds) or flexible GMRES (saddle kinds).  For Stokes the pressure is
 * returned with zero mean in the P1 mass weighting.
 *   b, x        3*n_nodes + n_pres doubles; device pointers when
 *               device_ptrs = 1, else host pointers (copied in and out inside
 *               the call).  b and x must not alias.
 *   stats       optional, filled on return.
 * The call synchronises its stream before returning.
 */
int amg_solve(amg_handle* h, const double* b, double* x, double rel_tol, int32_t device_ptrs,
              amg_stats* stats);

/*
 * amg_set_pressure_weights -- Stokes only: weights w_i (normally int phi_i dx of
 * the P1 pressure basis) defining the pressure normalisation sum_i w_i p_i = 0
 * applied to every preconditioned vector and to the result.  Without this call
 * the weights are all 1.  w: n_pres doubles, host or device (device_ptrs).
 */
int amg_set_pressure_weights(amg_handle* h, const double* w, int32_t device_ptrs);

/*
 * amg_solve_batched -- several SPD problems (each set up by amg_setup, kinds
 * AMG_VECTOR_LAPLACE / AMG_ELASTICITY, any sizes), each with n_rhs right-hand
 * sides, solved together: the multi-right-hand-side form of amg_solve.  The
 * cycle kernels work on all right-hand sides of a problem at once (block-row
 * times 16-column block: SpMM), each right-hand side runs its own flexible CG
 * with the stopping rule of amg_solve, and every problem runs as one CUDA
 * graph launch on its own handle's stream (an initial block and a device-side
 * loop with its own stopping test), all of them side by side.  How many of the
 * streams run concurrently is bounded by the process's hardware work queues:
 * set CUDA_DEVICE_MAX_CONNECTIONS (e.g. 32) before the CUDA context exists.
 *   handles     n_problems distinct handles (their precision and options apply);
 *               a handle listed twice is rejected with AMG_ERR_INVALID.
 *   n_rhs       1..16 right-hand sides per problem.
 *   B, X        per problem: device pointers to n_rhs vectors of 3*n_nodes
 *               doubles, vector r at offset r*3*n_nodes; X receives the
 *               solutions (x0 = 0).
 *   stats       NULL or an array of n_problems; solve_ms is the device time of
 *               the whole batch (from before the first launch to after the last
 *               problem, on the first handle's stream), iterations the loop count
 *               (the slowest right-hand side),
 *               true_rel_residual the worst right-hand side.
 * Returns AMG_OK when every right-hand side converged, AMG_NOT_CONVERGED when
 * some stopped at max_iterations.  Synchronises every handle's stream.
 */
int amg_solve_batched(amg_handle* const* handles, int32_t n_problems, int32_t n_rhs,
                      const double* const* B, double* const* X, double rel_tol,
                      amg_stats* stats);

/* Releases the handle and all its device memory.  NULL is accepted. */
void amg_free(amg_handle* h);

/* Message of the last error of this handle, or of the calling thread's last
 * failed call when h is NULL.  The string stays valid until the next call. */
const char* amg_last_error(const amg_handle* h);

/* ---------------------------------------------- inspection (parity tests) */

/* Sizes of level `level` of the hierarchy (0 = finest). */
int amg_level_info_get(const amg_handle* h, int32_t level, amg_level_info* info);

/* Copies one array of level `level` (see amg_level_item) into host memory of
 * `capacity` bytes.  AMG_ERR_INVALID if the item does not exist on that level
 * or capacity is too small. */
int amg_level_copy(const amg_handle* h, int32_t level, int32_t item, void* host_dst,
                   int64_t capacity);

/* One application of the preconditioner, z = M^{-1} r (opt->cycles cycles of
 * Algorithm 1 from zero), in the precision chosen at setup.  r and z are device
 * pointers of 3*n_nodes + n_pres doubles.  Synchronises the stream; returns
 * AMG_ERR_TIMEOUT if a bounded device wait of the cycle gave up. */
int amg_apply_preconditioner(amg_handle* h, const double* r, double* z);

/*
 * amg_apply_preconditioner_noalloc -- the same z = M^{-1} r as
 * amg_apply_preconditioner, for callers that cannot let a library call allocate
 * device memory: applications whose framework allocator (a caching allocator, a
 * memory pool sized at start-up) already holds nearly all of the device memory,
 * so that a cudaMalloc inside the call fails or forces the framework to give
 * memory back; and loops with a latency budget, where cudaMalloc and cudaFree may
 * synchronise the whole device.  amg_apply_preconditioner allocates its two
 * staging vectors on its first call; this variant never does.  The paper has no
 * counterpart; this is a property of the library interface.
 *   r, z   device pointers of 3*n_nodes + n_pres doubles (the caller owns them).
 * The input and output are staged in one static device array of the library
 * (2 x 1,310,720 doubles = 20 MiB, held on every GPU that loads the library until
 * the process exits), so the level-0 problem must satisfy
 * 4*n_nodes + n_pres <= 1,310,720; larger problems get AMG_ERR_INVALID with a
 * message giving both sizes.  No cudaMalloc, cudaFree or allocating library
 * routine is called.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the array: calls whose GPU work overlaps (several
 * handles, streams or threads at once) race on it and must be serialised by the
 * caller.  The array keeps the last call's contents; both staged vectors are
 * rewritten completely by every call.  Synchronises the handle's stream and
 * returns AMG_ERR_TIMEOUT if a bounded device wait of the cycle gave up.
 */
int amg_apply_preconditioner_noalloc(amg_handle* h, const double* r, double* z);

/* y = K_l x on level `level` with the library's FP64 (precision = AMG_FP64) or
 * FP32 (AMG_FP32, values rounded to float, accumulated in float) kernels, or on
 * level 0 the Krylov operator's FP32-pair kernel (AMG_FP32_PAIR); x and y are
 * device pointers of 3*n_nodes + n_pres doubles. */
int amg_level_apply(amg_handle* h, int32_t level, int32_t precision, const double* x,
                    double* y);

/* One smoothing sweep of level `level` (Sec. 3.3) on device vectors x (in/out)
 * and b of 3*n_nodes + n_pres doubles, in FP64: direction 0 = colours (or Vanka
 * patch colours) ascending, 1 = descending.  Synchronises the stream; returns
 * AMG_ERR_TIMEOUT if a bounded device wait gave up. */
int amg_level_smooth(amg_handle* h, int32_t level, int32_t direction, double* x,
                     const double* b);

/* The same sweep in `precision`: AMG_FP64 as amg_level_smooth, or AMG_FP32 on a
 * handle set up with precision AMG_FP32: x and b are rounded to float and the
 * sweep runs the FP32 cycle's kernels and launch variants (the ones its solves
 * time) on the level's FP32 values; x is returned widened to double. */
int amg_level_smooth_precision(amg_handle* h, int32_t level, int32_t direction,
                               int32_t precision, double* x, const double* b);

/* ------------------------------------------------------------ measurement */

enum amg_level_op {
  AMG_OP_APPLY = 0,      /* y = K_l x                                            */
  AMG_OP_RESIDUAL = 1,   /* r = b - K_l x                                        */
  AMG_OP_SMOOTH = 2,     /* one pre-smoothing sweep (all colours for GS)         */
  AMG_OP_RESTRICT = 3,   /* b_{l+1} = P^T r                                      */
  AMG_OP_PROLONG = 4,    /* x_l += P x_{l+1}                                     */
  AMG_OP_PRECOND = 5     /* one preconditioner application (level ignored)       */
};

/*
 * amg_time_level_op -- device time of one level operation of the cycle, for
 * roofline measurements.  Runs `warmup` untimed then `reps` timed repetitions
 * of `op` on level `level` in `precision` (AMG_FP64 / AMG_FP32; AMG_FP32_PAIR
 * for AMG_OP_APPLY on level 0) on the handle's
 * work vectors, between two CUDA events recorded on the handle's stream;
 * *ms_per_rep receives the mean.  *launches_per_rep receives the kernel
 * launches of one repetition (e.g. the colour count of a GS sweep).
 * The work vectors' contents are overwritten.
 */
int amg_time_level_op(amg_handle* h, int32_t op, int32_t level, int32_t precision, int32_t reps,
                      int32_t warmup, double* ms_per_rep, int32_t* launches_per_rep);


/* ------------------------------------------- learned weights (small network)
 *
 * Three multipliers per level change the cycle; all 1 is the plain method of
 * Sec. 3.3:
 *   ws  relaxation: the block Jacobi damping omega, the Gauss-Seidel step and
 *       the sGS velocity step of the level are multiplied by ws;
 *   wc  coarse-grid correction: x_l += wc * P x_{l+1} (Algorithm 1, step 13);
 *   wp  sGS pressure step of the level: omega_p is multiplied by wp (saddle
 *       kinds).
 * The paper has no counterpart: this part is an addition of the library.  A
 * network of two hidden layers of 64 (ReLU) maps 13 statistics of one level and
 * the level below it (amg_level_features) and a candidate (ws, wc, log2 wp) for
 * that level to the predicted log10 of the ratio of the convergence factor with
 * that level's multipliers changed (the others plain) to the plain factor.
 * amg_learn_weights evaluates it on a fixed grid of candidates for every level,
 * keeps each level's best, and falls back by measurement: the combination stays
 * only if a probe solve converges faster per iteration than with the plain
 * weights, else the level with the largest predicted gain alone is probed, else
 * the plain weights stay.
 */
#define AMG_N_FEATURES 13
#define AMG_MLP_INPUTS 16      /* features, ws, wc, log2 wp                   */
#define AMG_MLP_HIDDEN 64
#define AMG_MLP_NPARAM 5313    /* W1[64][16] b1[64] W2[64][64] b2[64] W3[64] b3 */
#define AMG_WS_MIN 0.6
#define AMG_WS_MAX 1.6
#define AMG_GRID_NWS 11
#define AMG_WC_MIN 0.8
#define AMG_WC_MAX 1.9
#define AMG_GRID_NWC 12
#define AMG_WP_LOG2_MIN (-1.0)
#define AMG_WP_LOG2_MAX 2.0
#define AMG_GRID_NWP 7

typedef struct amg_learned {
  double weights[3];        /* ws, wc, wp of level 0 after the call             */
  double predicted;         /* sum over levels of the network's output at each
                               level's chosen candidate                         */
  double rho_plain;         /* probe convergence factor, plain weights          */
  double rho_learned;       /* probe convergence factor of the weights that were
                               probed last against the plain ones               */
  int32_t fell_back;        /* 1: the plain weights were kept                   */
  int32_t n_candidates;     /* grid points per level                            */
  int32_t probe_iterations_plain;
  int32_t probe_iterations_learned;
  double level_weights[3 * AMG_MAX_LEVELS];  /* (ws, wc, wp) per level in use     */
  double level_predicted[AMG_MAX_LEVELS];    /* network output at each level's
                                                 choice (0 on the coarsest)      */
  int32_t n_levels;
  int32_t pad0;
} amg_learned;

/*
 * amg_features -- the network's 13 inputs for this hierarchy (host doubles):
 *   [0]      log10(3 n_nodes + n_pres) / 7
 *   [1..5]   level 0, over its non-Dirichlet nodes i (D_i the diagonal block,
 *            Frobenius norms): mean log10(|D_i| |D_i^-1|); standard deviation
 *            of log10 |D_i|; mean of sum_{j!=i} |A_ij| / |D_i|; and over its
 *            F nodes: mean share sum_{j in S_i} |A_ij| / sum_{j!=i} |A_ij|
 *            and mean |S_i| / 8, S_i the C nodes in the pattern of row i of P
 *            (the C-neighbours of i in the coarsening graph)
 *   [6..10]  the same for level 1 (0 when absent; the last two are 0 on the
 *            coarsest level)
 *   [11]     saddle kinds: mean over pressure rows of C_kk / S_D,kk with S_D the
 *            sGS scaling diag(C + B (D/omega)^-1 B^T); 0 otherwise
 *   [12]     1 for saddle kinds, 0 for SPD kinds
 */
int amg_features(amg_handle* h, double* features);

/*
 * amg_level_features -- the network's 13 inputs for non-coarsest level `level`
 * (host doubles), with the statistics of amg_features above:
 *   [0]      log10(3 n_l + n_pres,l) / 7
 *   [1..5]   the five statistics of level l
 *   [6..9]   the first four statistics of level l + 1
 *   [10]     l / 4
 *   [11]     saddle kinds: the pressure mean of level l (as [11] above)
 *   [12]     1 for saddle kinds, 0 for SPD kinds
 * AMG_ERR_INVALID for the coarsest level or a level that does not exist.
 */
int amg_level_features(amg_handle* h, int32_t level, double* features);

/* Sets (ws, wc, wp) = w[0..2] on every level (host doubles, finite, > 0). */
int amg_set_weights(amg_handle* h, const double* w);

/* Sets (ws, wc, wp) = w[3 l .. 3 l + 2] on levels l < n_levels (host doubles,
 * finite, > 0); levels from n_levels on get the plain weights. */
int amg_set_level_weights(amg_handle* h, const double* w, int32_t n_levels);

/* Copies the per-level weights, 4 doubles per level (ws, wc, wp, 1), to host. */
int amg_get_weights(const amg_handle* h, double* w, int32_t capacity);

/*
 * amg_learn_weights -- chooses each level's (ws, wc, wp) with the trained network
 * theta (host floats, AMG_MLP_NPARAM, layout above): per non-coarsest level, the
 * argmin of the network over the grid ws in [AMG_WS_MIN, AMG_WS_MAX]
 * (AMG_GRID_NWS points) x wc (AMG_GRID_NWC) x log2 wp (AMG_GRID_NWP, saddle
 * kinds; wp = 1 otherwise); then probe solves of K x = K y (y pseudo-random, zero
 * on Dirichlet nodes) to a relative residual of 1e-8: plain weights, the
 * combination, and if the combination is not faster the level with the largest
 * predicted gain alone.  Weights are kept only if their factor
 * rel_residual^(1/iterations) is smaller than the plain one.  out receives the
 * decision.  Later amg_solve calls use the weights in place.
 */
int amg_learn_weights(amg_handle* h, const float* theta, amg_learned* out);

/*
 * The network's kernels, on device memory (FP32 master weights, BF16 tensor-core
 * products with FP32 accumulation), ordered on `stream` (cudaStream_t, NULL =
 * legacy default stream); none synchronises.
 *   amg_mlp_forward   y[i] = net(theta, x[16 i .. 16 i + 15]), i < n
 *   amg_mlp_gradient  grad = d/dtheta of loss, loss = sum_i (y_i - t_i)^2 / n
 *                     (grad: AMG_MLP_NPARAM floats, loss: 1 float, both
 *                     overwritten)
 *   amg_mlp_backward  grad = sum_i dy[i] d y_i / d theta for per-sample upstream
 *                     gradients dy (n floats; the gradient of any loss of the
 *                     outputs, e.g. a ranking loss over each problem's
 *                     candidates); grad is overwritten
 *   amg_mlp_adam      one Adam step (beta 0.9 / 0.999, eps 1e-8) of step
 *                     number `step` >= 1 with learning rate lr; m and v are
 *                     the moment buffers (zero before step 1)
 */
int amg_mlp_forward(const float* theta, const float* x, int32_t n, float* y, void* stream);
int amg_mlp_gradient(const float* theta, const float* x, const float* t, int32_t n, float* grad,
                     float* loss, void* stream);
int amg_mlp_backward(const float* theta, const float* x, const float* dy, int32_t n,
                     float* grad, void* stream);
int amg_mlp_adam(float* theta, const float* grad, float* m, float* v, int32_t step, float lr,
                 void* stream);

#ifdef __cplusplus
}
#endif

#endif /* AMGP2_H */
