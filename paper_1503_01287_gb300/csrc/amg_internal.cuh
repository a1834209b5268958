// Internal declarations of the amgp2 CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "amgp2.h"

namespace amgp2 {

// ------------------------------------------------------------------------ errors

struct Error {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what, const char* file, int line);
// opt-in dynamic shared memory of a kernel, once per device
void max_dynamic_smem(const void* func, int bytes);

#define AMG_CUDA(x) ::amgp2::check_cuda((x), #x, __FILE__, __LINE__)
#define AMG_LAUNCH_CHECK() ::amgp2::check_cuda(cudaGetLastError(), "kernel launch", __FILE__, __LINE__)

// ------------------------------------------------------------------------ device buffers

template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    release();
    n = count;
    if (count) AMG_CUDA(cudaMalloc(&p, count * sizeof(T)));
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  size_t bytes() const { return n * sizeof(T); }
  operator T*() const { return p; }
};

// ------------------------------------------------------------------------ hierarchy

// One level of the scalar hierarchy of S = C + B A^{-1} B^T that the Braess-Sarazin
// smoother of a saddle level cycles on (S_0 on the saddle level's pressure
// unknowns, S_{k+1} = H^T S_k H through the pressure prolongations below it).
struct SLevel {
  int n = 0;            // pressure unknowns
  int64_t nnz = 0;
  DBuf<int> rowptr, col;
  DBuf<double> val, dinv;   // dinv: 1 / S_kk (0 where S_kk = 0)
  DBuf<float> val32, dinv32;
  DBuf<double> x64, b64, r64;
  DBuf<float> x32, b32, r32;
};

// One level of the hierarchy.  A is kept as 9 value planes (plane e holds entry
// (e/3, e%3) of every block), so that consecutive threads reading consecutive
// blocks read consecutive addresses; the column indices are shared by both
// precisions.
struct Level {
  int n = 0;            // 3-component nodes
  int np = 0;           // pressure unknowns
  int64_t nnzb = 0;
  DBuf<int> rowptr, col, tags;
  DBuf<double> val;     // 9 * nnzb, plane-major
  DBuf<float> val32;     // FP32 copy of the kernel layout (k_val)
  DBuf<unsigned short> val16;   // BF16 bit patterns of the kernel layout (levels >= 1,
                                // AMG_FP32_BF16 only)
  DBuf<double> dinv;    // 12 * n: per node 3 padded rows (4 values) of the inverse
  DBuf<float> dinv32;
  int ncolours = 0;
  std::vector<int> colour_ptr;  // host: offsets into colour_rows, ncolours+1
  DBuf<int> colour, colour_rows;
  // Coloured levels keep a second copy of A whose block rows are stored in
  // colour order (stored row k is node colour_rows[k]; column ids unchanged), so
  // a colour sweep reads one contiguous range.  The cycle's row kernels use it.
  bool stored = false;
  DBuf<int> srowptr, scol;
  DBuf<double> sval;            // 9 planes, stored order
  const int* k_rowptr() const { return stored ? srowptr.p : rowptr.p; }
  const int* k_col() const { return stored ? scol.p : col.p; }
  const double* k_val() const { return stored ? sval.p : val.p; }
  const int* k_rows() const { return stored ? colour_rows.p : nullptr; }
  int max_row_blocks = 0;
  double avg_row_blocks = 0.0;
  int group = 0;        // lanes per block row in the row kernels (autotuned at setup)
  int group_gs = 0;     // the same for the colour-subset Gauss-Seidel kernel
  int gs_stream = 0;    // CTAs per SM of the grid-stride colour kernel (0: k_gs_pdl)
  int gs_tma = 0;       // 1: the FP32 colour kernel stages its rows' blocks by TMA (k_gs_tma)
  int gs_xnc = 0;       // k_gs_pdl gathers x through L1 (1) or L2 only (0), by timing
  int group64 = 0;      // the FP64 operator kernel when the cycle runs in FP32
  // level 0 of an FP32 SPD handle with outer_pair: the kernel-layout values as
  // 9 planes of (hi, lo) float pairs, hi = fl32(a), lo = fl32(a - hi)
  DBuf<float2> val2;
  int group_pair = 0;
  // the colour sweep as one launch of a gs_cl-CTA cluster with the iterate in
  // shared memory (0: one launch per colour), gs_cl_g lanes per block row
  int gs_cl = 0;
  int gs_cl_g = 0;
  int gs_cl_bytes = 0;  // sizeof the arithmetic type the cluster size was chosen for
  // the colour sweep as one cooperative launch in dataflow order (flow.cu):
  // flow = lanes per block row (0: off); the column indices with their
  // colour-order bits (stored order), [sweep number, finished CTAs], the tagged
  // exchange array of new node values (8 words a node), and the row chunks of
  // 32/flow rows that never cross a colour
  DBuf<unsigned> fcol, fstate;
  DBuf<unsigned long long> fxt;
  DBuf<int> fchunk;
  int flow = 0;
  int flow_nchunks = 0;
  int flow_grid32 = 0, flow_grid64 = 0;
  // learned weights of this level on the device: [0] relaxation multiplier,
  // [1] coarse-correction scale, [2] pressure-step multiplier (all 1: plain)
  double* wt = nullptr;

  // transfer to level+1 (absent on the coarsest level)
  DBuf<int> state, cid;
  int64_t p_nnz = 0;
  DBuf<int> p_rowptr, p_col;   // rows: fine nodes, cols: coarse nodes
  DBuf<double> p_val;
  DBuf<float> p_val32;
  DBuf<int> r_rowptr, r_col;   // R = P^T: rows coarse nodes, cols fine nodes (ascending)
  DBuf<double> r_val;
  DBuf<float> r_val32;

  // saddle parts
  int64_t b_nnz = 0, c_nnz = 0;
  DBuf<int> b_rowptr, b_col;   // rows: pressure; cols: velocity nodes
  DBuf<double> b_val;          // 3 planes of b_nnz
  DBuf<float> b_val32;
  DBuf<int> bt_rowptr, bt_col; // B^T: rows velocity nodes; cols pressure
  DBuf<double> bt_val;         // 3 planes
  DBuf<float> bt_val32;
  DBuf<int> c_rowptr, c_col;
  DBuf<double> c_val;
  DBuf<float> c_val32;
  DBuf<double> schur;          // sGS scaling S_D (np)
  DBuf<float> schur32;
  DBuf<int> pstate, pcid;
  // Braess-Sarazin smoother: 1 / (2 diag A) in the padded layout, and the S
  // hierarchy with the generalised inverse of its coarsest matrix
  DBuf<double> ahinv;
  DBuf<float> ahinv32;
  std::vector<std::unique_ptr<SLevel>> S;
  DBuf<double> s_coarse_inv;
  int s_coarse_m = 0;
  // Vanka smoother: patch k = pressure unknown k with the velocity nodes of row k
  // of B (m_k = 3 * row length unknowns); A_k^{-1} row-major at vk_off[k],
  // w_k = A_k^{-1} B_k^T at 3 * b_rowptr[k], s_k = B_k w_k + C_kk; the patches in
  // colour order (vk_rows[vk_colour_ptr[c] ..]) of the overlap-graph colouring
  DBuf<long long> vk_off;
  DBuf<double> vk_ainv, vk_w, vk_s;
  DBuf<float> vk_ainv32, vk_w32, vk_s32;
  DBuf<int> vk_colour, vk_rows;
  std::vector<int> vk_colour_ptr;
  DBuf<int> vk_cnodes;             // velocity nodes of the patches, colour by colour
  std::vector<int> vk_cnode_ptr;
  int vk_ncolours = 0;
  int vk_mmax = 0;
  int64_t h_nnz = 0;
  DBuf<int> h_rowptr, h_col, ht_rowptr, ht_col;
  DBuf<double> h_val, ht_val;
  DBuf<float> h_val32, ht_val32;

  // cycle work vectors, padded layout (4n + np)
  DBuf<double> x64, b64, r64, t64;
  DBuf<float> x32, b32, r32, t32;

  int dofs() const { return 3 * n + np; }    // unknowns (user layout)
  int dofs4() const { return 4 * n + np; }   // padded cycle layout
};

// multi-right-hand-side work vectors of one level ([node][kRhs][4])
constexpr int kRhs = 16;
struct BatchLevel {
  DBuf<double> x64, b64, r64, t64;
  DBuf<float> x32, b32, r32, t32;
  int tile = 0;     // block-row tile of the cycle's SpMM kernels (chosen by timing)
  int tile64 = 0;   // the same for the FP64 operator (level 0)
  int tile_pair = 0;   // the same for the FP32-pair operator (level 0)
  int tile_gs = 0;     // tile of the multi-right-hand-side colour kernel
};

}  // namespace amgp2

struct amg_handle {
  amg_options opt{};
  int kind = 0;
  bool saddle = false;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  std::vector<std::unique_ptr<amgp2::Level>> L;
  int coarse_m = 0;
  int coarse_rank = 0;
  amgp2::DBuf<double> coarse_inv;  // m x m row-major generalised inverse
  // Krylov state
  amgp2::DBuf<double> kb, kx, kr, kz, kp, kq, kw, kro;   // padded layout
  amgp2::DBuf<float> kpf;           // the CG direction in pair form (8 floats a node)
  amgp2::DBuf<double> ub, ux;                             // user layout staging
  amgp2::DBuf<double> gm_V, gm_Z;  // FGMRES bases (V holds FP32 pairs)
  amgp2::DBuf<double> gm_wp;       // the FGMRES Krylov vector as FP32 pairs
  amgp2::DBuf<double> red;         // reduction partials
  amgp2::DBuf<double> scal;        // device scalars
  amgp2::DBuf<double> pmass;       // Stokes pressure weights
  double pmass_sum = 0.0;
  double* host_scal = nullptr;     // pinned
  int* host_int = nullptr;         // pinned
  amgp2::DBuf<int> it_dev;         // device iteration counter of the graph loop
  cudaGraphExec_t cg_loop_pcg = nullptr, cg_loop_fcg = nullptr;   // whole-solve loops
  int64_t cg_loop_pcg_launches = 0, cg_loop_fcg_launches = 0;
  bool cg_loop_failed = false;
  bool iter_graph_failed = false;
  amgp2::DBuf<int> flag;           // device error word
  std::string last_error;
  int64_t launches = 0;
  double setup_ms = 0.0;
  cudaGraphExec_t cycle_graph = nullptr;  // one preconditioner application
  bool cycle_graph_valid = false;
  // coarse levels from `sub_from` down run as one cluster launch (0: off)
  int sub_from = 0;
  int sub_cluster = 0;                    // CTAs in the cluster (0: clusters unavailable)
  amgp2::DBuf<unsigned char> sub_ph32, sub_ph64;   // recorded phase lists
  int sub_n32 = 0, sub_n64 = 0;
  // or the whole cycle as one persistent cooperative launch
  bool use_full = false;
  bool use_pdl = true;      // colour kernels with programmatic dependent launch
  int grid_ctas = 0;
  amgp2::DBuf<unsigned char> full_ph32, full_ph64;
  int full_n32 = 0, full_n64 = 0;
  amgp2::DBuf<unsigned> grid_bar;
  // batched (multi-right-hand-side) solves
  std::vector<amgp2::BatchLevel> B;
  amgp2::DBuf<double> mb, mx, mr, mz, mp, mq, mro, bred, bscal;
  amgp2::DBuf<float> mpf;           // the directions in pair form (FP32-pair operator)
  amgp2::DBuf<int> bit;
  amgp2::DBuf<double> wts;          // 4 learned weights per level (see Level::wt)
  bool bf16_coarse = false;         // AMG_FP32_BF16: levels >= 1 keep BF16 values
  ~amg_handle();
};

namespace amgp2 {

// ------------------------------------------------------------------------ helpers

constexpr int kReduceBlocks = 608;   // 4 x 152 SMs
constexpr int kReduceThreads = 256;

inline int div_up(int64_t a, int64_t b) { return static_cast<int>((a + b - 1) / b); }

// exclusive scan of int counts; out[n] receives the total; returns the total
int64_t exclusive_scan(const int* in, int* out, int n, cudaStream_t s, amg_handle* h);

// setup (setup.cu)
void build_hierarchy(amg_handle* h, const amg_matrix* m, const int32_t* tags);

// cycle (cycle.cu)
template <typename T>
void level_apply(amg_handle* h, int l, const T* x, T* y);   // y = K_l x
template <typename T>
void level_residual(amg_handle* h, int l, const T* x, const T* b, T* r);
template <typename T>
void level_smooth(amg_handle* h, int l, T* x, const T* b, bool post, bool x_is_zero);
template <typename T>
void vcycle(amg_handle* h, int l, bool x_is_zero);
template <typename T>
void precondition_device(amg_handle* h, const double* r, double* z);
// y = K_0 x with the FP32-pair operator (level 0 values split into hi/lo float
// planes, x as 8 floats a node: hi x,y,z,0 then lo x,y,z,0); y padded FP64
void apply_pair(amg_handle* h, const float* xp, double* y);
void apply_K_pair(amg_handle* h, const double* x, float* xp, double* y);
// the 8-floats-a-node pair form of a padded FP64 vector of n4 = 4 n entries
void launch_split_pair(const double* x, float* xp, int64_t n4, cudaStream_t s, amg_handle* h);
// restriction (restrict = true) or prolongation between level and level+1 on
// the level work vectors, in FP32 or FP64
void level_transfer(amg_handle* h, int l, bool restrict_, bool f32);

// picks the lanes-per-row of each level by timing the operator kernel and the
// level from which the cycle runs as one cluster launch
void autotune_levels(amg_handle* h);
// records the cluster sub-cycle from level `from` (0 disables it)
void set_subcycle(amg_handle* h, int from);

// krylov (krylov.cu)
int solve_device(amg_handle* h, const double* b, double* x, double tol, amg_stats* st);

// noalloc.cu: the preconditioner application with static staging vectors
void apply_preconditioner_noalloc(amg_handle* h, const double* r, double* z);
// one-launch dataflow colour sweep (flow.cu): its per-level data (false if the
// level has no colours or the device has no cooperative launch), its chunks and
// grid for G lanes per row (sets lv.flow = G), and the launch
bool flow_prepare(amg_handle* h, Level& lv);
void flow_set_group(amg_handle* h, Level& lv, int G);
template <typename T>
void launch_gs_flow(amg_handle* h, Level& lv, T* x, const T* b, const T* val, const T* dinv,
                    bool reverse);
// After the handle's stream has been synchronised: reads the device error word
// that bounded waits (grid barrier, mbarrier) set when they give up, clears it
// and fails with AMG_ERR_TIMEOUT naming `what` if it was set.
void check_wait_flag(amg_handle* h, const char* what);

// learned.cu: statistics of the hierarchy, weights, selection with fallback
constexpr double kProbeTol = 1e-8;   // the probe solves run to the stopping tolerance of the workloads
void compute_features(amg_handle* h, double* out);
void compute_level_features(amg_handle* h, int l, double* out);
void set_weights(amg_handle* h, const double* w3);
void set_level_weights(amg_handle* h, const double* w, int n);
void get_weights(const amg_handle* h, double* out);
void learn_weights(amg_handle* h, const float* theta_host, amg_learned* out);

// mlp.cu: the network's kernels
int mlp_nparam();
void mlp_forward(const float* theta, const float* X, int n, float* y, cudaStream_t s);
void mlp_gradient(const float* theta, const float* X, const float* t, int n, float* grad,
                  float* loss, cudaStream_t s);
void mlp_adam(float* theta, const float* grad, float* m, float* v, int step, float lr,
              cudaStream_t s);
void mlp_backward(const float* theta, const float* X, const float* dy, int n, float* grad,
                  cudaStream_t s);

// batched.cu: all problems and right-hand sides in one graph launch
int solve_batched(amg_handle* const* hs, int np, int nrhs, const double* const* B,
                  double* const* X, double tol, amg_stats* stats, double* ms_out);

// small kernels shared across files
void launch_copy(const double* a, double* b, int64_t n, cudaStream_t s, amg_handle* h);
void launch_to_float(const double* a, float* b, int64_t n, cudaStream_t s, amg_handle* h);
void launch_to_double(const float* a, double* b, int64_t n, cudaStream_t s, amg_handle* h);
void launch_fill(double* a, double v, int64_t n, cudaStream_t s, amg_handle* h);
// user layout (3 per node, then pressure) <-> padded layout (4 per node, then pressure)
void launch_to_padded(const double* u, double* p, int n, int np, cudaStream_t s, amg_handle* h);
void launch_from_padded(const double* p, double* u, int n, int np, cudaStream_t s, amg_handle* h);

}  // namespace amgp2
