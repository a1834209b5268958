// C ABI of the amgp2 library (declarations and contracts in include/amgp2.h).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "amg_internal.cuh"

namespace amgp2 {

namespace {
thread_local std::string g_last_error;
}

[[noreturn]] void fail(int code, const std::string& msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  char buf[512];
  snprintf(buf, sizeof buf, "%s failed at %s:%d: %s", what, file, line, cudaGetErrorString(e));
  cudaGetLastError();  // clear a sticky-free error so the handle stays usable
  throw Error{e == cudaErrorMemoryAllocation ? AMG_ERR_NOMEM : AMG_ERR_CUDA, buf};
}

void max_dynamic_smem(const void* func, int bytes) {
  // the attribute belongs to the current device's context: set once per (device, kernel)
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  AMG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({dev, func})) return;
  AMG_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.insert({dev, func});
}

template <class F>
int guarded(amg_handle* h, F&& f) {
  try {
    return f();
  } catch (const Error& e) {
    g_last_error = e.msg;
    if (h) h->last_error = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    if (h) h->last_error = e.what();
    return AMG_ERR_INVALID;
  }
}

}  // namespace amgp2

using namespace amgp2;

amg_handle::~amg_handle() {
  if (host_scal) cudaFreeHost(host_scal);
  if (host_int) cudaFreeHost(host_int);
  if (cycle_graph) cudaGraphExecDestroy(cycle_graph);
  if (cg_loop_pcg) cudaGraphExecDestroy(cg_loop_pcg);
  if (cg_loop_fcg) cudaGraphExecDestroy(cg_loop_fcg);
  L.clear();
  coarse_inv.release();
  if (own_stream) cudaStreamDestroy(own_stream);
}

extern "C" {

void amg_default_options(amg_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->smoother = -1;          // resolved per kind in amg_setup
  o->m_pre = 1;
  o->m_post = 1;
  o->nu = 1;
  o->cycles = 1;
  o->precision = AMG_FP64;
  o->krylov = AMG_KRYLOV_AUTO;
  o->max_levels = 5;
  o->coarse_dofs = 300;
  o->gmres_restart = 50;
  o->separate = 1;
  o->max_iterations = 1000;
  o->use_graphs = 1;
  o->cluster_from = -1;
  o->cycle_kernel = 0;
  o->omega = 0.5;
  o->omega_p = 0.125;
  o->batch_tile = -1;
  o->gs_cluster = -1;
  o->outer_pair = 1;
  o->post_order = -1;     // resolved from the Krylov method in amg_setup
  o->gs_flow = -1;
  o->gs_stream = -1;
  o->gs_tma = -1;
}

int amg_setup(const amg_matrix* m, const int32_t* node_tags, int32_t kind, const amg_options* opt,
              void* stream, amg_handle** out) {
  if (out) *out = nullptr;
  amg_handle* h = nullptr;
  int rc = guarded(nullptr, [&]() -> int {
    if (!m || !node_tags || !out) fail(AMG_ERR_INVALID, "null argument");
    if (kind < AMG_VECTOR_LAPLACE || kind > AMG_STOKES) fail(AMG_ERR_INVALID, "unknown kind");
    if (m->n_nodes <= 0 || m->nnzb < m->n_nodes || !m->a_rowptr || !m->a_col || !m->a_val)
      fail(AMG_ERR_INVALID, "A must have n_nodes > 0 and a diagonal block per row");
    const bool saddle = kind == AMG_MIXED_ELASTICITY || kind == AMG_STOKES;
    if (saddle && (m->n_pres <= 0 || !m->b_rowptr || !m->b_col || !m->b_val || !m->c_rowptr ||
                   !m->c_col || !m->c_val || m->c_nnz < m->n_pres))
      fail(AMG_ERR_INVALID, "saddle kinds need B and C (C's pattern also for Stokes)");
    if (!saddle && m->n_pres != 0) fail(AMG_ERR_INVALID, "n_pres must be 0 for SPD kinds");
    int dev = 0;
    AMG_CUDA(cudaGetDevice(&dev));
    h = new amg_handle();
    if (opt) h->opt = *opt;
    else amg_default_options(&h->opt);
    if (h->opt.smoother < 0) h->opt.smoother = saddle ? AMG_SMOOTHER_SGS : AMG_SMOOTHER_GS;
    const bool saddle_smoother = h->opt.smoother == AMG_SMOOTHER_SGS ||
                                 h->opt.smoother == AMG_SMOOTHER_BS ||
                                 h->opt.smoother == AMG_SMOOTHER_VANKA;
    if (saddle && !saddle_smoother)
      fail(AMG_ERR_UNSUPPORTED,
           "saddle kinds use the segregated Gauss-Seidel, Braess-Sarazin or Vanka smoother");
    if (!saddle && saddle_smoother)
      fail(AMG_ERR_INVALID, "the sGS, Braess-Sarazin and Vanka smoothers need a saddle kind");
    if (h->opt.smoother == AMG_SMOOTHER_VANKA) {
      // the Vanka patch phase runs as its own launches only
      h->opt.cluster_from = 0;
      h->opt.cycle_kernel = 1;
    }
    if (h->opt.precision != AMG_FP64 && h->opt.precision != AMG_FP32 &&
        h->opt.precision != AMG_FP32_BF16)
      fail(AMG_ERR_INVALID, "unknown precision");
    if (h->opt.precision == AMG_FP32_BF16) {   // an FP32 cycle with BF16 coarse values
      h->bf16_coarse = true;
      h->opt.precision = AMG_FP32;
    }
    if (h->opt.gs_cluster < -1 || h->opt.gs_cluster > 16 ||
        (h->opt.gs_cluster > 0 && (h->opt.gs_cluster & (h->opt.gs_cluster - 1))))
      fail(AMG_ERR_INVALID, "gs_cluster must be -1, 0, 1, 2, 4, 8 or 16");
    if (h->opt.m_pre < 0 || h->opt.m_post < 0 || h->opt.nu < 1 || h->opt.nu > 2 ||
        h->opt.cycles < 1 || h->opt.max_levels < 1 || h->opt.gmres_restart < 1 ||
        h->opt.post_order < -1 || h->opt.post_order > 1 || h->opt.gs_flow < -1 ||
        h->opt.gs_flow > 1 || h->opt.gs_stream < -1 || h->opt.gs_stream > 8 ||
        h->opt.gs_tma < -1 || h->opt.gs_tma > 1)
      fail(AMG_ERR_INVALID, "option out of range");
    // post-smoothing colour order: the stand-alone iteration sweeps the colours in the
    // pre-smoothing order, a Krylov method gets the symmetric (reversed) order
    if (h->opt.post_order < 0) h->opt.post_order = h->opt.krylov == AMG_KRYLOV_NONE ? 1 : 0;
    h->kind = kind;
    h->saddle = saddle;
    if (stream) {
      h->stream = (cudaStream_t)stream;
    } else {
      // graph capture needs a non-legacy stream: the handle then owns one
      AMG_CUDA(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
      h->stream = h->own_stream;
    }
    h->flag.alloc(1);
    AMG_CUDA(cudaMallocHost(&h->host_scal, 8 * sizeof(double)));
    AMG_CUDA(cudaMallocHost(&h->host_int, 8 * sizeof(int)));
    auto t0 = std::chrono::steady_clock::now();
    nvtxRangePushA("amg_setup");
    struct Pop { ~Pop() { nvtxRangePop(); } } pop;
    build_hierarchy(h, m, node_tags);
    if (kind == AMG_STOKES) {
      const int np = m->n_pres;
      h->pmass.alloc(np);
      std::vector<double> w(np, 1.0);   // until amg_set_pressure_weights is called
      AMG_CUDA(cudaMemcpyAsync(h->pmass.p, w.data(), np * sizeof(double), cudaMemcpyHostToDevice,
                               h->stream));
      h->pmass_sum = (double)np;
    }
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    h->setup_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return AMG_OK;
  });
  if (rc != AMG_OK) {
    delete h;
    if (out) *out = nullptr;
  }
  return rc;
}

int amg_set_pressure_weights(amg_handle* h, const double* w, int32_t device_ptrs) {
  return guarded(h, [&]() -> int {
    if (!h || !w) fail(AMG_ERR_INVALID, "null argument");
    if (h->kind != AMG_STOKES) fail(AMG_ERR_INVALID, "pressure weights apply to Stokes only");
    const int np = h->L[0]->np;
    std::vector<double> hw(np);
    AMG_CUDA(cudaMemcpyAsync(hw.data(), w, np * sizeof(double),
                             device_ptrs ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost,
                             h->stream));
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    double s = 0.0;
    for (double v : hw) {
      if (!(v >= 0.0) || !std::isfinite(v)) fail(AMG_ERR_INVALID, "weights must be finite, >= 0");
      s += v;
    }
    if (!(s > 0.0)) fail(AMG_ERR_INVALID, "weights sum to zero");
    AMG_CUDA(cudaMemcpyAsync(h->pmass.p, hw.data(), np * sizeof(double), cudaMemcpyHostToDevice,
                             h->stream));
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    h->pmass_sum = s;
    return AMG_OK;
  });
}

static void fill_stats(amg_handle* h, amg_stats* st) {
  st->n_levels = (int)h->L.size();
  st->setup_ms = h->setup_ms;
  st->cluster_from = h->sub_from;
  st->cycle_kernel = h->use_full ? 2 : 1;
  for (int l = 0; l < AMG_MAX_LEVELS; ++l) {
    if (l < (int)h->L.size()) {
      st->level_nodes[l] = h->L[l]->n;
      st->level_pres[l] = h->L[l]->np;
      st->level_nnzb[l] = h->L[l]->nnzb;
      st->level_colours[l] = h->L[l]->ncolours;
      st->level_group[l] = h->L[l]->group;
      st->level_gs_cluster[l] = h->L[l]->gs_cl;
      // the dataflow sweep runs where neither the cluster sweep nor the
      // persistent cycle takes the level's sweeps
      st->level_gs_flow[l] = (h->use_full || h->L[l]->gs_cl > 0) ? 0 : h->L[l]->flow;
      // the grid-stride colour kernel runs where the colour chain does
      st->level_gs_stream[l] = (h->use_full || h->L[l]->gs_cl > 0 || st->level_gs_flow[l] > 0 ||
                                (int)l >= (h->sub_from > 0 ? h->sub_from : AMG_MAX_LEVELS))
                                   ? 0
                                   : h->L[l]->gs_stream;
      st->level_gs_tma[l] = st->level_gs_stream[l] > 0 ? 0
                            : (h->use_full || h->L[l]->gs_cl > 0 || st->level_gs_flow[l] > 0 ||
                               (int)l >= (h->sub_from > 0 ? h->sub_from : AMG_MAX_LEVELS))
                                  ? 0
                                  : h->L[l]->gs_tma;
    } else {
      st->level_gs_cluster[l] = 0;
      st->level_gs_flow[l] = 0;
      st->level_gs_stream[l] = 0;
      st->level_gs_tma[l] = 0;
      st->level_nodes[l] = st->level_pres[l] = st->level_colours[l] = 0;
      st->level_group[l] = 0;
      st->level_nnzb[l] = 0;
    }
  }
}

int amg_solve(amg_handle* h, const double* b, double* x, double rel_tol, int32_t device_ptrs,
              amg_stats* stats) {
  return guarded(h, [&]() -> int {
    if (!h || !b || !x) fail(AMG_ERR_INVALID, "null argument");
    if (b == x) fail(AMG_ERR_INVALID, "b and x must not alias");
    if (!(rel_tol > 0.0)) fail(AMG_ERR_INVALID, "rel_tol must be > 0");
    amg_stats local{};
    amg_stats* st = stats ? stats : &local;
    std::memset(st, 0, sizeof(*st));
    fill_stats(h, st);
    const int64_t n = h->L[0]->dofs();
    const int64_t l0 = h->launches;
    cudaEvent_t e0, e1;
    AMG_CUDA(cudaEventCreate(&e0));
    AMG_CUDA(cudaEventCreate(&e1));
    AMG_CUDA(cudaEventRecord(e0, h->stream));
    nvtxRangePushA(h->opt.precision == AMG_FP32 ? "amg_solve_fp32" : "amg_solve_fp64");
    struct Pop { ~Pop() { nvtxRangePop(); } } pop;
    int rc;
    if (device_ptrs) {
      rc = solve_device(h, b, x, rel_tol, st);
    } else {
      // staging vectors are kept in the handle so repeated solves allocate nothing
      if ((int64_t)h->ub.n < n) h->ub.alloc(n);
      if ((int64_t)h->ux.n < n) h->ux.alloc(n);
      AMG_CUDA(cudaMemcpyAsync(h->ub.p, b, n * sizeof(double), cudaMemcpyHostToDevice,
                               h->stream));
      rc = solve_device(h, h->ub, h->ux, rel_tol, st);
      AMG_CUDA(cudaMemcpyAsync(x, h->ux.p, n * sizeof(double), cudaMemcpyDeviceToHost,
                               h->stream));
    }
    AMG_CUDA(cudaEventRecord(e1, h->stream));
    AMG_CUDA(cudaEventSynchronize(e1));
    check_wait_flag(h, "the solve");
    float ms = 0.f;
    AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    st->solve_ms = ms;
    st->converged = rc == AMG_OK;
    st->kernel_launches = h->launches - l0;
    return rc;
  });
}

void amg_free(amg_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  delete h;
}

const char* amg_last_error(const amg_handle* h) {
  if (h) return h->last_error.c_str();
  return g_last_error.c_str();
}

int amg_level_info_get(const amg_handle* h, int32_t level, amg_level_info* info) {
  return guarded(const_cast<amg_handle*>(h), [&]() -> int {
    if (!h || !info) fail(AMG_ERR_INVALID, "null argument");
    if (level < 0 || level >= (int)h->L.size()) fail(AMG_ERR_INVALID, "no such level");
    const Level& lv = *h->L[level];
    info->n_nodes = lv.n;
    info->n_pres = lv.np;
    info->nnzb = lv.nnzb;
    info->p_nnz = lv.p_nnz;
    info->h_nnz = lv.h_nnz;
    info->b_nnz = lv.b_nnz;
    info->c_nnz = lv.c_nnz;
    info->n_colours = lv.ncolours;
    info->is_coarsest = level == (int)h->L.size() - 1;
    return AMG_OK;
  });
}

}  // extern "C"

namespace amgp2 {
namespace {

__global__ void k_planes_to_aos(const double* __restrict__ planes, int nv, int64_t nnz,
                                double* __restrict__ aos) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    for (int e = 0; e < nv; ++e) aos[nv * k + e] = planes[e * nnz + k];
}

}  // namespace

void check_wait_flag(amg_handle* h, const char* what) {
  int ferr = 0;
  AMG_CUDA(cudaMemcpy(&ferr, h->flag.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (!ferr) return;
  AMG_CUDA(cudaMemset(h->flag.p, 0, sizeof(int)));
  fail(AMG_ERR_TIMEOUT, std::string("a bounded device wait (grid barrier or mbarrier) gave up "
                                    "during ") + what + "; the result is not valid");
}

namespace {

void copy_out(amg_handle* h, const void* src, size_t bytes, void* dst, int64_t cap) {
  if ((int64_t)bytes > cap) fail(AMG_ERR_INVALID, "destination too small");
  if (bytes == 0) return;
  if (!src) fail(AMG_ERR_INVALID, "item not present on this level");
  AMG_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream));
  AMG_CUDA(cudaStreamSynchronize(h->stream));
}

void copy_planes(amg_handle* h, const double* planes, int nv, int64_t nnz, void* dst, int64_t cap) {
  if ((int64_t)(nnz * nv * sizeof(double)) > cap) fail(AMG_ERR_INVALID, "destination too small");
  if (nnz == 0) return;
  DBuf<double> tmp;
  tmp.alloc(nnz * nv);
  k_planes_to_aos<<<std::max(1, std::min(div_up(nnz, 256), 4096)), 256, 0, h->stream>>>(
      planes, nv, nnz, tmp);
  AMG_LAUNCH_CHECK();
  copy_out(h, tmp.p, nnz * nv * sizeof(double), dst, cap);
}

}  // namespace
}  // namespace amgp2

extern "C" {

int amg_level_copy(const amg_handle* hc, int32_t level, int32_t item, void* dst, int64_t cap) {
  amg_handle* h = const_cast<amg_handle*>(hc);
  return guarded(h, [&]() -> int {
    if (!h || !dst) fail(AMG_ERR_INVALID, "null argument");
    if (level < 0 || level >= (int)h->L.size()) fail(AMG_ERR_INVALID, "no such level");
    const Level& lv = *h->L[level];
    const bool last = level == (int)h->L.size() - 1;
    const size_t I = sizeof(int), D = sizeof(double);
    switch (item) {
      case AMG_Q_A_ROWPTR: copy_out(h, lv.rowptr, (lv.n + 1) * I, dst, cap); break;
      case AMG_Q_A_COL: copy_out(h, lv.col, lv.nnzb * I, dst, cap); break;
      case AMG_Q_A_VAL: copy_planes(h, lv.val, 9, lv.nnzb, dst, cap); break;
      case AMG_Q_TAGS: copy_out(h, lv.tags, lv.n * I, dst, cap); break;
      case AMG_Q_CF_STATE:
        if (last) fail(AMG_ERR_INVALID, "the coarsest level has no C/F split");
        copy_out(h, lv.state, lv.n * I, dst, cap); break;
      case AMG_Q_P_ROWPTR:
        if (last) fail(AMG_ERR_INVALID, "the coarsest level has no prolongation");
        copy_out(h, lv.p_rowptr, (lv.n + 1) * I, dst, cap); break;
      case AMG_Q_P_COL:
        if (last) fail(AMG_ERR_INVALID, "the coarsest level has no prolongation");
        copy_out(h, lv.p_col, lv.p_nnz * I, dst, cap); break;
      case AMG_Q_P_VAL:
        if (last) fail(AMG_ERR_INVALID, "the coarsest level has no prolongation");
        copy_out(h, lv.p_val, lv.p_nnz * D, dst, cap); break;
      case AMG_Q_COLOUR:
        if (last || h->saddle) fail(AMG_ERR_INVALID, "level has no colouring");
        copy_out(h, lv.colour, lv.n * I, dst, cap); break;
      case AMG_Q_DINV: {
        if ((int64_t)(9 * lv.n * D) > cap) fail(AMG_ERR_INVALID, "destination too small");
        std::vector<double> pad(12 * (size_t)lv.n);
        copy_out(h, lv.dinv, pad.size() * D, pad.data(), (int64_t)(pad.size() * D));
        double* o = static_cast<double*>(dst);
        for (int i = 0; i < lv.n; ++i)
          for (int r = 0; r < 3; ++r)
            for (int c2 = 0; c2 < 3; ++c2) o[9 * i + 3 * r + c2] = pad[12 * i + 4 * r + c2];
        break;
      }
      case AMG_Q_B_ROWPTR:
        if (!h->saddle) fail(AMG_ERR_INVALID, "no B");
        copy_out(h, lv.b_rowptr, (lv.np + 1) * I, dst, cap); break;
      case AMG_Q_B_COL:
        if (!h->saddle) fail(AMG_ERR_INVALID, "no B");
        copy_out(h, lv.b_col, lv.b_nnz * I, dst, cap); break;
      case AMG_Q_B_VAL:
        if (!h->saddle) fail(AMG_ERR_INVALID, "no B");
        copy_planes(h, lv.b_val, 3, lv.b_nnz, dst, cap); break;
      case AMG_Q_C_ROWPTR:
        if (!h->saddle) fail(AMG_ERR_INVALID, "no C");
        copy_out(h, lv.c_rowptr, (lv.np + 1) * I, dst, cap); break;
      case AMG_Q_C_COL:
        if (!h->saddle) fail(AMG_ERR_INVALID, "no C");
        copy_out(h, lv.c_col, lv.c_nnz * I, dst, cap); break;
      case AMG_Q_C_VAL:
        if (!h->saddle) fail(AMG_ERR_INVALID, "no C");
        copy_out(h, lv.c_val, lv.c_nnz * D, dst, cap); break;
      case AMG_Q_PCF_STATE:
        if (!h->saddle || last) fail(AMG_ERR_INVALID, "no pressure C/F split");
        copy_out(h, lv.pstate, lv.np * I, dst, cap); break;
      case AMG_Q_H_ROWPTR:
        if (!h->saddle || last) fail(AMG_ERR_INVALID, "no H");
        copy_out(h, lv.h_rowptr, (lv.np + 1) * I, dst, cap); break;
      case AMG_Q_H_COL:
        if (!h->saddle || last) fail(AMG_ERR_INVALID, "no H");
        copy_out(h, lv.h_col, lv.h_nnz * I, dst, cap); break;
      case AMG_Q_H_VAL:
        if (!h->saddle || last) fail(AMG_ERR_INVALID, "no H");
        copy_out(h, lv.h_val, lv.h_nnz * D, dst, cap); break;
      case AMG_Q_S_ROWPTR:
      case AMG_Q_S_COL:
      case AMG_Q_S_VAL: {
        if (lv.S.empty()) fail(AMG_ERR_INVALID, "level has no Braess-Sarazin S matrix");
        const SLevel& q = *lv.S[0];
        if (item == AMG_Q_S_ROWPTR) copy_out(h, q.rowptr, (q.n + 1) * I, dst, cap);
        else if (item == AMG_Q_S_COL) copy_out(h, q.col, q.nnz * I, dst, cap);
        else copy_out(h, q.val, q.nnz * D, dst, cap);
        break;
      }
      case AMG_Q_COARSE_INV:
        if (!last) fail(AMG_ERR_INVALID, "only the coarsest level has a factorisation");
        copy_out(h, h->coarse_inv, (size_t)h->coarse_m * h->coarse_m * D, dst, cap); break;
      default:
        fail(AMG_ERR_INVALID, "unknown item");
    }
    return AMG_OK;
  });
}

int amg_apply_preconditioner(amg_handle* h, const double* r, double* z) {
  return guarded(h, [&]() -> int {
    if (!h || !r || !z) fail(AMG_ERR_INVALID, "null argument");
    Level& lv = *h->L[0];
    const int64_t n4 = lv.dofs4();
    if ((int64_t)h->kr.n < n4) { h->kr.alloc(n4); h->kz.alloc(n4); }
    launch_to_padded(r, h->kr, lv.n, lv.np, h->stream, h);
    if (h->opt.precision == AMG_FP32) precondition_device<float>(h, h->kr, h->kz);
    else precondition_device<double>(h, h->kr, h->kz);
    launch_from_padded(h->kz, z, lv.n, lv.np, h->stream, h);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    check_wait_flag(h, "the preconditioner application");
    return AMG_OK;
  });
}

int amg_apply_preconditioner_noalloc(amg_handle* h, const double* r, double* z) {
  return guarded(h, [&]() -> int {
    if (!h || !r || !z) fail(AMG_ERR_INVALID, "null argument");
    apply_preconditioner_noalloc(h, r, z);
    return AMG_OK;
  });
}

int amg_level_apply(amg_handle* h, int32_t level, int32_t precision, const double* x, double* y) {
  return guarded(h, [&]() -> int {
    if (!h || !x || !y) fail(AMG_ERR_INVALID, "null argument");
    if (level < 0 || level >= (int)h->L.size()) fail(AMG_ERR_INVALID, "no such level");
    Level& lv = *h->L[level];
    launch_to_padded(x, lv.t64, lv.n, lv.np, h->stream, h);
    if (precision == AMG_FP64) {
      level_apply<double>(h, level, lv.t64.p, lv.r64.p);
    } else if (precision == AMG_FP32) {
      if (!lv.val32.p) fail(AMG_ERR_INVALID, "FP32 operators exist only with precision FP32");
      const int64_t n4 = lv.dofs4();
      launch_to_float(lv.t64, lv.t32, n4, h->stream, h);
      level_apply<float>(h, level, lv.t32.p, lv.r32.p);
      launch_to_double(lv.r32, lv.r64, n4, h->stream, h);
    } else if (precision == AMG_FP32_PAIR) {
      if (level != 0 || !lv.val2.p)
        fail(AMG_ERR_INVALID, "the FP32-pair operator exists on level 0 of FP32 handles "
                              "with outer_pair");
      DBuf<float> xp;
      xp.alloc(8 * (size_t)lv.n);
      apply_K_pair(h, lv.t64, xp, lv.r64);
      AMG_CUDA(cudaStreamSynchronize(h->stream));
    } else {
      fail(AMG_ERR_INVALID, "unknown precision");
    }
    launch_from_padded(lv.r64, y, lv.n, lv.np, h->stream, h);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    return AMG_OK;
  });
}

int amg_level_smooth(amg_handle* h, int32_t level, int32_t direction, double* x, const double* b) {
  return guarded(h, [&]() -> int {
    if (!h || !x || !b) fail(AMG_ERR_INVALID, "null argument");
    if (level < 0 || level >= (int)h->L.size() - 1)
      fail(AMG_ERR_INVALID, "no smoother on this level");
    Level& lv = *h->L[level];
    launch_to_padded(x, lv.x64, lv.n, lv.np, h->stream, h);
    launch_to_padded(b, lv.b64, lv.n, lv.np, h->stream, h);
    level_smooth<double>(h, level, lv.x64.p, lv.b64.p, direction != 0, false);
    launch_from_padded(lv.x64, x, lv.n, lv.np, h->stream, h);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    check_wait_flag(h, "the smoothing sweep");
    return AMG_OK;
  });
}

int amg_level_smooth_precision(amg_handle* h, int32_t level, int32_t direction,
                               int32_t precision, double* x, const double* b) {
  if (precision == AMG_FP64) return amg_level_smooth(h, level, direction, x, b);
  return guarded(h, [&]() -> int {
    if (!h || !x || !b) fail(AMG_ERR_INVALID, "null argument");
    if (precision != AMG_FP32) fail(AMG_ERR_INVALID, "precision must be AMG_FP64 or AMG_FP32");
    if (level < 0 || level >= (int)h->L.size() - 1)
      fail(AMG_ERR_INVALID, "no smoother on this level");
    Level& lv = *h->L[level];
    if (!lv.val32.p) fail(AMG_ERR_INVALID, "FP32 operators exist only with precision FP32");
    const int64_t n4 = lv.dofs4();
    launch_to_padded(x, lv.x64, lv.n, lv.np, h->stream, h);
    launch_to_padded(b, lv.b64, lv.n, lv.np, h->stream, h);
    launch_to_float(lv.x64, lv.x32, n4, h->stream, h);
    launch_to_float(lv.b64, lv.b32, n4, h->stream, h);
    level_smooth<float>(h, level, lv.x32.p, lv.b32.p, direction != 0, false);
    launch_to_double(lv.x32, lv.x64, n4, h->stream, h);
    launch_from_padded(lv.x64, x, lv.n, lv.np, h->stream, h);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    check_wait_flag(h, "the smoothing sweep");
    return AMG_OK;
  });
}

int amg_time_level_op(amg_handle* h, int32_t op, int32_t level, int32_t precision, int32_t reps,
                      int32_t warmup, double* ms_per_rep, int32_t* launches_per_rep) {
  return guarded(h, [&]() -> int {
    if (!h || !ms_per_rep || reps < 1 || warmup < 0) fail(AMG_ERR_INVALID, "bad argument");
    const int L = (int)h->L.size();
    if (op != AMG_OP_PRECOND && (level < 0 || level >= L)) fail(AMG_ERR_INVALID, "no such level");
    if ((op == AMG_OP_SMOOTH || op == AMG_OP_RESTRICT || op == AMG_OP_PROLONG) && level == L - 1)
      fail(AMG_ERR_INVALID, "the coarsest level has no smoother or transfer");
    const bool f32 = precision == AMG_FP32;
    const bool pair = precision == AMG_FP32_PAIR;
    if (f32 && !h->L[0]->val32.p) fail(AMG_ERR_INVALID, "FP32 operators exist only with FP32");
    if (pair && (op != AMG_OP_APPLY || level != 0 || !h->L[0]->val2.p))
      fail(AMG_ERR_INVALID, "the FP32-pair operator is AMG_OP_APPLY on level 0 of FP32 "
                            "handles with outer_pair");
    Level& lv = *h->L[op == AMG_OP_PRECOND ? 0 : level];
    DBuf<float> xp;
    if (pair) {
      xp.alloc(8 * (size_t)lv.n);
      AMG_CUDA(cudaMemsetAsync(xp.p, 0, xp.bytes(), h->stream));
    }
    if (op == AMG_OP_PRECOND && (int64_t)h->kr.n < lv.dofs4()) {
      h->kr.alloc(lv.dofs4());
      h->kz.alloc(lv.dofs4());
      AMG_CUDA(cudaMemsetAsync(h->kr.p, 0, h->kr.bytes(), h->stream));
    }
    auto once = [&]() {
      switch (op) {
        case AMG_OP_APPLY:
          if (pair) apply_pair(h, xp.p, lv.r64.p);
          else if (f32) level_apply<float>(h, level, lv.x32.p, lv.r32.p);
          else level_apply<double>(h, level, lv.x64.p, lv.r64.p);
          break;
        case AMG_OP_RESIDUAL:
          if (f32) level_residual<float>(h, level, lv.x32.p, lv.b32.p, lv.r32.p);
          else level_residual<double>(h, level, lv.x64.p, lv.b64.p, lv.r64.p);
          break;
        case AMG_OP_SMOOTH:
          if (f32) level_smooth<float>(h, level, lv.x32.p, lv.b32.p, false, false);
          else level_smooth<double>(h, level, lv.x64.p, lv.b64.p, false, false);
          break;
        case AMG_OP_RESTRICT:
        case AMG_OP_PROLONG:
          level_transfer(h, level, op == AMG_OP_RESTRICT, f32);
          break;
        case AMG_OP_PRECOND:
          if (h->opt.precision == AMG_FP32) precondition_device<float>(h, h->kr, h->kz);
          else precondition_device<double>(h, h->kr, h->kz);
          break;
        default:
          fail(AMG_ERR_INVALID, "unknown op");
      }
    };
    // vectors: zero x, b = 1 so that the data are finite
    launch_fill(lv.x64, 0.0, lv.dofs4(), h->stream, h);
    launch_fill(lv.b64, 1.0, lv.dofs4(), h->stream, h);
    if (f32) {
      launch_to_float(lv.x64, lv.x32, lv.dofs4(), h->stream, h);
      launch_to_float(lv.b64, lv.b32, lv.dofs4(), h->stream, h);
    }
    for (int i = 0; i < warmup; ++i) once();
    const int64_t l0 = h->launches;
    cudaEvent_t e0, e1;
    AMG_CUDA(cudaEventCreate(&e0));
    AMG_CUDA(cudaEventCreate(&e1));
    AMG_CUDA(cudaEventRecord(e0, h->stream));
    for (int i = 0; i < reps; ++i) once();
    AMG_CUDA(cudaEventRecord(e1, h->stream));
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_per_rep = ms / reps;
    if (launches_per_rep) *launches_per_rep = (int32_t)((h->launches - l0) / reps);
    return AMG_OK;
  });
}

int amg_solve_batched(amg_handle* const* handles, int32_t n_problems, int32_t n_rhs,
                      const double* const* B, double* const* X, double rel_tol,
                      amg_stats* stats) {
  amg_handle* h0 = (handles && n_problems > 0) ? handles[0] : nullptr;
  return guarded(h0, [&]() -> int {
    if (!handles || !B || !X || n_problems <= 0) fail(AMG_ERR_INVALID, "null argument");
    if (!(rel_tol > 0.0)) fail(AMG_ERR_INVALID, "rel_tol must be > 0");
    for (int p = 0; p < n_problems; ++p)
      if (!handles[p] || !B[p] || !X[p]) fail(AMG_ERR_INVALID, "null handle or vector");
    double ms = 0.0;
    return solve_batched(handles, n_problems, n_rhs, B, X, rel_tol, stats, &ms);
  });
}

int amg_features(amg_handle* h, double* features) {
  return guarded(h, [&]() -> int {
    if (!h || !features) fail(AMG_ERR_INVALID, "null argument");
    compute_features(h, features);
    return AMG_OK;
  });
}

int amg_set_weights(amg_handle* h, const double* w) {
  return guarded(h, [&]() -> int {
    if (!h || !w) fail(AMG_ERR_INVALID, "null argument");
    for (int e = 0; e < 3; ++e)
      if (!(std::isfinite(w[e]) && w[e] > 0.0)) fail(AMG_ERR_INVALID, "weights must be finite and > 0");
    set_weights(h, w);
    return AMG_OK;
  });
}

int amg_level_features(amg_handle* h, int32_t level, double* features) {
  return guarded(h, [&]() -> int {
    if (!h || !features) fail(AMG_ERR_INVALID, "null argument");
    compute_level_features(h, level, features);
    return AMG_OK;
  });
}

int amg_set_level_weights(amg_handle* h, const double* w, int32_t n_levels) {
  return guarded(h, [&]() -> int {
    if (!h || !w || n_levels < 0) fail(AMG_ERR_INVALID, "bad argument");
    for (int64_t e = 0; e < 3 * (int64_t)n_levels; ++e)
      if (!(std::isfinite(w[e]) && w[e] > 0.0))
        fail(AMG_ERR_INVALID, "weights must be finite and > 0");
    set_level_weights(h, w, n_levels);
    return AMG_OK;
  });
}

int amg_get_weights(const amg_handle* hc, double* w, int32_t capacity) {
  amg_handle* h = const_cast<amg_handle*>(hc);
  return guarded(h, [&]() -> int {
    if (!h || !w) fail(AMG_ERR_INVALID, "null argument");
    if (capacity < 4 * (int64_t)h->L.size()) fail(AMG_ERR_INVALID, "capacity < 4 * n_levels");
    get_weights(h, w);
    return AMG_OK;
  });
}

int amg_learn_weights(amg_handle* h, const float* theta, amg_learned* out) {
  return guarded(h, [&]() -> int {
    if (!h || !theta || !out) fail(AMG_ERR_INVALID, "null argument");
    for (int k = 0; k < AMG_MLP_NPARAM; ++k)
      if (!std::isfinite(theta[k])) fail(AMG_ERR_INVALID, "non-finite network parameter");
    learn_weights(h, theta, out);
    return AMG_OK;
  });
}

int amg_mlp_forward(const float* theta, const float* x, int32_t n, float* y, void* stream) {
  return guarded(nullptr, [&]() -> int {
    if (n < 0 || (n > 0 && (!theta || !x || !y))) fail(AMG_ERR_INVALID, "bad argument");
    mlp_forward(theta, x, n, y, (cudaStream_t)stream);
    return AMG_OK;
  });
}

int amg_mlp_gradient(const float* theta, const float* x, const float* t, int32_t n, float* grad,
                     float* loss, void* stream) {
  return guarded(nullptr, [&]() -> int {
    if (n < 0 || !grad || !loss || (n > 0 && (!theta || !x || !t)))
      fail(AMG_ERR_INVALID, "bad argument");
    mlp_gradient(theta, x, t, n, grad, loss, (cudaStream_t)stream);
    return AMG_OK;
  });
}

int amg_mlp_backward(const float* theta, const float* x, const float* dy, int32_t n,
                     float* grad, void* stream) {
  return guarded(nullptr, [&]() -> int {
    if (n < 0 || !grad || (n > 0 && (!theta || !x || !dy))) fail(AMG_ERR_INVALID, "bad argument");
    mlp_backward(theta, x, dy, n, grad, (cudaStream_t)stream);
    return AMG_OK;
  });
}

int amg_mlp_adam(float* theta, const float* grad, float* m, float* v, int32_t step, float lr,
                 void* stream) {
  return guarded(nullptr, [&]() -> int {
    if (!theta || !grad || !m || !v || step < 1 || !(lr > 0.f)) fail(AMG_ERR_INVALID, "bad argument");
    mlp_adam(theta, grad, m, v, step, lr, (cudaStream_t)stream);
    return AMG_OK;
  });
}

}  // extern "C"
