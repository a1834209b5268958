// Krylov accelerators of the AMG preconditioner (Sec. 3.1 and Sec. 4):
// preconditioned CG (SPD, FP64 cycle), flexible CG (SPD, FP32 cycle), right-
// preconditioned flexible GMRES(m) (saddle systems), and the stand-alone AMG
// iteration.  Residuals, inner products and orthogonalisation are FP64;
// scalars stay on the device and the host reads one residual norm per
// iteration for the stopping rule ||b - K x_k|| / ||b|| <= tol.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "amg_internal.cuh"

namespace amgp2 {

namespace {

enum Slot { S_RZ = 0, S_PQ, S_RR, S_RZN, S_ZRO, S_BB, S_BETA, S_T0, S_T1, S_TOL2, S_NSLOTS };
constexpr int kMaxDots = 320;  // multi-dot width (FGMRES restart + 2)

__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
  return t;   // valid in thread 0
}

// partial[blk*nd + d] = sum over this block's indices of a_d[k] * b_d[k], nd <= 2
__global__ void k_dots(int64_t n, int nd, const double* a0, const double* b0, const double* a1,
                       const double* b1, double* __restrict__ partial) {
  __shared__ double sh[32];
  for (int d = 0; d < nd; ++d) {
    const double* x = d == 0 ? a0 : a1;
    const double* y = d == 0 ? b0 : b1;
    double s = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
      s = fma(x[k], y[k], s);
    double t = block_sum(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x * nd + d] = t;
  }
}

// multi-dot against a basis, kMdotG basis vectors per block row (blockIdx.y): each
// thread keeps kMdotG sums, so w is read once per kMdotG vectors and the block
// reduction runs once per row instead of once per vector.
// partial[blockIdx.x * m + i] = sum over block column blockIdx.x's indices of V_i[k] w[k]
constexpr int kMdotG = 8;
__global__ void __launch_bounds__(256) k_mdot(int64_t n, int m, const double* __restrict__ V,
                                              int64_t ldv, const double* __restrict__ w,
                                              double* __restrict__ partial) {
  __shared__ double sh[kMdotG][32];
  const int i0 = blockIdx.y * kMdotG;
  const int gn = min(kMdotG, m - i0);
  double acc[kMdotG];
#pragma unroll
  for (int g = 0; g < kMdotG; ++g) acc[g] = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double wk = w[k];
#pragma unroll
    for (int g = 0; g < kMdotG; ++g)
      if (g < gn) acc[g] = fma(V[(int64_t)(i0 + g) * ldv + k], wk, acc[g]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < kMdotG; ++g) {
    double v = acc[g];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[g][wid] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x < gn) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[threadIdx.x][q];
    partial[blockIdx.x * (int64_t)m + i0 + threadIdx.x] = t;
  }
}

// out[i] = sum over b < nblk of partial[b * m + i] in block order, one warp per i
__global__ void k_mdot_final(const double* __restrict__ partial, int nblk, int m,
                             double* __restrict__ out) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += partial[(int64_t)b * m + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[i] = s;
}

// out[d] = sum_blk partial[blk*nd + d] in block order (deterministic)
__global__ void k_final(const double* __restrict__ partial, int nblk, int nd,
                        double* __restrict__ out) {
  __shared__ double sh[32];
  for (int d = 0; d < nd; ++d) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[b * nd + d];
    double t = block_sum(s, sh);
    if (threadIdx.x == 0) out[d] = t;
    __syncthreads();
  }
}

// CG step: alpha = rz / pq; x += alpha p; (ro = r); r -= alpha q; partial ||r||^2
__global__ void k_cg_update(int64_t n, double* __restrict__ x, double* __restrict__ r,
                            const double* __restrict__ p, const double* __restrict__ q,
                            double* __restrict__ ro, const double* __restrict__ s,
                            double* __restrict__ partial) {
  __shared__ double sh[32];
  const double alpha = s[S_RZ] / s[S_PQ];
  double acc = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    x[k] = fma(alpha, p[k], x[k]);
    const double rk = r[k];
    if (ro) ro[k] = rk;
    const double rn = fma(-alpha, q[k], rk);
    r[k] = rn;
    acc = fma(rn, rn, acc);
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// beta = (rz_new - <z, r_old>) / rz (flexible) or rz_new / rz; rz <- rz_new
__global__ void k_cg_beta(double* s, int flexible) {
  const double num = flexible ? s[S_RZN] - s[S_ZRO] : s[S_RZN];
  s[S_BETA] = num / s[S_RZ];
  s[S_RZ] = s[S_RZN];
}

// stopping rule on the device: continue while ||r||^2 > tol^2 ||b||^2, the
// iteration limit is not reached and the residual is finite
__global__ void k_cg_check(cudaGraphConditionalHandle cond, const double* __restrict__ s,
                           int* it, int maxit) {
  const int k = ++(*it);
  const double rr = s[S_RR];
  const bool go = !(rr <= s[S_TOL2] * s[S_BB]) && k < maxit && isfinite(rr);
  cudaGraphSetConditional(cond, go ? 1u : 0u);
}

__global__ void k_set_tol2(double* s, double tol) { s[S_TOL2] = tol * tol; }

__global__ void k_cg_dir(int64_t n, double* __restrict__ p, const double* __restrict__ z,
                         const double* __restrict__ s) {
  const double beta = s[S_BETA];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    p[k] = fma(beta, p[k], z[k]);
}

// the same, also writing p in the pair form of the FP32-pair operator (8 floats
// a node: hi of the 4 padded entries, then lo; lo = fl32(p - hi))
__global__ void k_cg_dir_pair(int64_t n, double* __restrict__ p, const double* __restrict__ z,
                              const double* __restrict__ s, float* __restrict__ pf) {
  const double beta = s[S_BETA];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double v = fma(beta, p[k], z[k]);
    p[k] = v;
    const float hi = (float)v;
    const int64_t o = 8 * (k >> 2) + (k & 3);
    pf[o] = hi;
    pf[o + 4] = (float)(v - (double)hi);
  }
}

// w -= sum_i c[i] V_i (c on the device, staged in shared memory; the basis loads
// of one index go out eight at a time, the sum keeps the order i = 0, 1, ...)
__global__ void __launch_bounds__(256) k_basis_sub(int64_t n, int m, const double* __restrict__ V,
                                                   int64_t ldv, const double* __restrict__ c,
                                                   double* __restrict__ w) {
  __shared__ double cs[kMaxDots];
  for (int i = threadIdx.x; i < m; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[k];
    int i = 0;
    for (; i + 8 <= m; i += 8) {
      double v[8];
#pragma unroll
      for (int g = 0; g < 8; ++g) v[g] = V[(int64_t)(i + g) * ldv + k];
#pragma unroll
      for (int g = 0; g < 8; ++g) acc = fma(-cs[i + g], v[g], acc);
    }
    for (; i < m; ++i) acc = fma(-cs[i], V[(int64_t)i * ldv + k], acc);
    w[k] = acc;
  }
}

// x += sum_i y[i] Z_i (the same access pattern)
__global__ void __launch_bounds__(256) k_basis_add(int64_t n, int m, const double* __restrict__ Z,
                                                   int64_t ldz, const double* __restrict__ y,
                                                   double* __restrict__ x) {
  __shared__ double ys[kMaxDots];
  for (int i = threadIdx.x; i < m; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    double acc = x[k];
    int i = 0;
    for (; i + 8 <= m; i += 8) {
      double v[8];
#pragma unroll
      for (int g = 0; g < 8; ++g) v[g] = Z[(int64_t)(i + g) * ldz + k];
#pragma unroll
      for (int g = 0; g < 8; ++g) acc = fma(ys[i + g], v[g], acc);
    }
    for (; i < m; ++i) acc = fma(ys[i], Z[(int64_t)i * ldz + k], acc);
    x[k] = acc;
  }
}

__global__ void k_scale(int64_t n, const double* __restrict__ a, double alpha,
                        double* __restrict__ b) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = alpha * a[k];
}

__global__ void k_axpy(int64_t n, double alpha, const double* __restrict__ a, double* __restrict__ b) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = fma(alpha, a[k], b[k]);
}

// c = a - b; c may be b (element-wise, in place)
__global__ void k_sub(int64_t n, const double* __restrict__ a, const double* b, double* c) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    c[k] = a[k] - b[k];
}

// p -= (w . p) / sum(w): pressure mean zero in the P1 mass weighting
__global__ void k_shift(int64_t n, double* __restrict__ p, const double* __restrict__ s,
                        double wsum) {
  const double c = s[0] / wsum;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    p[k] -= c;
}

inline int gridr(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, kReduceBlocks));
}

struct Ctx {
  amg_handle* h;
  cudaStream_t s;
  int64_t n;

  // scal[slot] = a0 . b0 (and scal[slot+1] = a1 . b1), over `len` entries
  void dots(const double* a0, const double* b0, int slot, const double* a1 = nullptr,
            const double* b1 = nullptr, int64_t len = -1) {
    const int nd = a1 ? 2 : 1;
    k_dots<<<kReduceBlocks, kReduceThreads, 0, s>>>(len < 0 ? n : len, nd, a0, b0, a1, b1,
                                                    h->red);
    k_final<<<1, 256, 0, s>>>(h->red, kReduceBlocks, nd, h->scal.p + slot);
    h->launches += 2;
  }
};

void apply_K(amg_handle* h, const double* x, double* y) { level_apply<double>(h, 0, x, y); }

void precond(amg_handle* h, const double* r, double* z) {
  if (h->opt.precision == AMG_FP32) precondition_device<float>(h, r, z);
  else precondition_device<double>(h, r, z);
}

void project_pressure(amg_handle* h, Ctx& c, double* v) {
  if (h->kind != AMG_STOKES || !h->pmass.p) return;
  const Level& lv = *h->L[0];
  double* p = v + 4 * lv.n;
  const int64_t np = lv.np;
  c.dots(h->pmass.p, p, S_T0, nullptr, nullptr, np);
  k_shift<<<gridr(np), 256, 0, c.s>>>(np, p, h->scal.p + S_T0, h->pmass_sum);
  h->launches++;
}

double read_scalar(amg_handle* h, int slot) {
  AMG_CUDA(cudaMemcpyAsync(h->host_scal, h->scal.p + slot, sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
  AMG_CUDA(cudaStreamSynchronize(h->stream));
  return *h->host_scal;
}

double true_residual(amg_handle* h, Ctx& c, const double* b, const double* x) {
  apply_K(h, x, h->kw);
  k_sub<<<gridr(c.n), 256, 0, c.s>>>(c.n, b, h->kw, h->kw);
  h->launches++;
  c.dots(h->kw.p, h->kw.p, S_T1);
  return std::sqrt(std::max(0.0, read_scalar(h, S_T1)));
}

// ---------------------------------------------------------------- CG / flexible CG

int solve_cg(amg_handle* h, Ctx& c, const double* b, double* x, double tol, bool flexible,
             amg_stats* st) {
  cudaStream_t s = c.s;
  const int64_t n = c.n;
  double* r = h->kr;
  double* z = h->kz;
  double* p = h->kp;
  double* q = h->kq;
  double* ro = flexible ? h->kro.p : nullptr;
  AMG_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  launch_copy(b, r, n, s, h);
  c.dots(b, b, S_BB);
  const double bb = read_scalar(h, S_BB);
  const double bnorm = std::sqrt(bb);
  int it = 0;
  double rel = 0.0;
  if (bnorm == 0.0) {
    st->iterations = 0;
    st->rel_residual = 0.0;
    return AMG_OK;
  }
  precond(h, r, z);
  c.dots(r, z, S_RZ);
  launch_copy(z, p, n, s, h);
  // FP32 cycle: the operator products in FP32-pair arithmetic (outer_pair)
  float* pf = (h->opt.precision == AMG_FP32 && h->L[0]->val2.p) ? h->kpf.p : nullptr;

  // the body of one iteration after the first: z = M r, beta, p, q = A p, alpha, x, r
  auto body = [&](bool first) {
    if (!first) {
      precond(h, r, z);
      if (flexible) c.dots(r, z, S_RZN, z, ro);
      else c.dots(r, z, S_RZN);
      k_cg_beta<<<1, 1, 0, s>>>(h->scal.p, flexible ? 1 : 0);
      if (pf) k_cg_dir_pair<<<gridr(n), 256, 0, s>>>(n, p, z, h->scal.p, pf);
      else k_cg_dir<<<gridr(n), 256, 0, s>>>(n, p, z, h->scal.p);
      h->launches += 2;
    } else if (pf) {
      launch_split_pair(p, pf, n, s, h);
    }
    if (pf) apply_pair(h, pf, q);
    else apply_K(h, p, q);
    c.dots(p, q, S_PQ);
    k_cg_update<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, x, r, p, q, ro, h->scal.p, h->red);
    k_final<<<1, 256, 0, s>>>(h->red, kReduceBlocks, 1, h->scal.p + S_RR);
    h->launches += 2;
  };

  body(true);
  ++it;
  rel = std::sqrt(std::max(0.0, read_scalar(h, S_RR))) / bnorm;
  // All further iterations in one graph launch: a conditional WHILE node whose
  // body is one iteration followed by the stopping test (k_cg_check).
  if (h->opt.use_graphs && !(rel <= tol) && it < h->opt.max_iterations && std::isfinite(rel)) {
    cudaGraphExec_t& wexec = flexible ? h->cg_loop_fcg : h->cg_loop_pcg;
    int64_t& per_iter = flexible ? h->cg_loop_fcg_launches : h->cg_loop_pcg_launches;
    if (!wexec && !h->cg_loop_failed) {
      const int64_t l0 = h->launches;
      cudaGraph_t g = nullptr;
      bool capturing = false;
      try {
        AMG_CUDA(cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle cond;
        AMG_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        AMG_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
        cudaGraph_t bodyg = np.conditional.phGraph_out[0];
        AMG_CUDA(cudaStreamBeginCaptureToGraph(s, bodyg, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
        capturing = true;
        body(false);
        k_cg_check<<<1, 1, 0, s>>>(cond, h->scal.p, h->it_dev.p, h->opt.max_iterations);
        AMG_LAUNCH_CHECK();
        capturing = false;
        AMG_CUDA(cudaStreamEndCapture(s, &bodyg));
        AMG_CUDA(cudaGraphInstantiate(&wexec, g, 0));
        per_iter = h->launches - l0 + 1;
      } catch (const Error&) {
        if (capturing) {
          cudaGraph_t junk = nullptr;
          cudaStreamEndCapture(s, &junk);
          if (junk) cudaGraphDestroy(junk);
        }
        cudaGetLastError();
        if (wexec) cudaGraphExecDestroy(wexec);
        wexec = nullptr;
        h->cg_loop_failed = true;   // fall back to one graph launch per iteration
      }
      if (g) cudaGraphDestroy(g);
      h->launches = l0;
    }
    if (wexec) {
      k_set_tol2<<<1, 1, 0, s>>>(h->scal.p, tol);
      *h->host_int = it;
      AMG_CUDA(cudaMemcpyAsync(h->it_dev.p, h->host_int, sizeof(int), cudaMemcpyHostToDevice, s));
      AMG_CUDA(cudaGraphLaunch(wexec, s));
      AMG_CUDA(cudaMemcpyAsync(h->host_int, h->it_dev.p, sizeof(int), cudaMemcpyDeviceToHost, s));
      rel = std::sqrt(std::max(0.0, read_scalar(h, S_RR))) / bnorm;   // synchronises
      h->launches += (int64_t)(*h->host_int - it) * per_iter + 1;
      it = *h->host_int;
    }
  }
  cudaGraphExec_t exec = nullptr;
  int64_t per_iter = 0;
  const bool use_graph = h->opt.use_graphs != 0;
  while (!(rel <= tol) && it < h->opt.max_iterations) {
    if (!std::isfinite(rel)) fail(AMG_ERR_BREAKDOWN, "non-finite residual in CG");
    if (use_graph && !exec && !h->iter_graph_failed) {
      const int64_t l0 = h->launches;
      cudaGraph_t g = nullptr;
      bool capturing = false;
      try {
        AMG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        capturing = true;
        body(false);
        capturing = false;
        AMG_CUDA(cudaStreamEndCapture(s, &g));
        AMG_CUDA(cudaGraphInstantiate(&exec, g, 0));
        per_iter = h->launches - l0;
      } catch (const Error&) {
        if (capturing) {
          cudaGraph_t junk = nullptr;
          cudaStreamEndCapture(s, &junk);
          if (junk) cudaGraphDestroy(junk);
        }
        cudaGetLastError();
        exec = nullptr;
        h->iter_graph_failed = true;   // run the iterations as plain launches
      }
      if (g) cudaGraphDestroy(g);
      h->launches = l0;
    }
    if (exec) {
      AMG_CUDA(cudaGraphLaunch(exec, s));
      h->launches += per_iter;
    } else {
      body(false);
    }
    ++it;
    rel = std::sqrt(std::max(0.0, read_scalar(h, S_RR))) / bnorm;
  }
  if (exec) cudaGraphExecDestroy(exec);
  st->iterations = it;
  st->rel_residual = rel;
  st->true_rel_residual = true_residual(h, c, b, x) / bnorm;
  return (rel <= tol) ? AMG_OK : AMG_NOT_CONVERGED;
}

// ---------------------------------------------------------------- stand-alone AMG

int solve_amg(amg_handle* h, Ctx& c, const double* b, double* x, double tol, amg_stats* st) {
  cudaStream_t s = c.s;
  const int64_t n = c.n;
  AMG_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  c.dots(b, b, S_BB);
  const double bnorm = std::sqrt(read_scalar(h, S_BB));
  if (bnorm == 0.0) { st->iterations = 0; return AMG_OK; }
  int it = 0;
  double rel = 1.0;
  while (it < h->opt.max_iterations) {
    // one application of Algorithm 1 to the current iterate: x += M (b - K x)
    level_residual<double>(h, 0, x, b, h->kr);
    precond(h, h->kr, h->kz);
    k_axpy<<<gridr(n), 256, 0, s>>>(n, 1.0, h->kz, x);
    h->launches++;
    ++it;
    rel = true_residual(h, c, b, x) / bnorm;
    if (!std::isfinite(rel)) fail(AMG_ERR_BREAKDOWN, "non-finite residual in AMG iteration");
    if (rel <= tol) break;
  }
  st->iterations = it;
  st->rel_residual = rel;
  st->true_rel_residual = rel;
  return rel <= tol ? AMG_OK : AMG_NOT_CONVERGED;
}

// ---------------------------------------------------------------- FGMRES

int solve_fgmres(amg_handle* h, Ctx& c, const double* b, double* x, double tol, amg_stats* st) {
  cudaStream_t s = c.s;
  const int64_t n = c.n;
  const int m = std::max(1, std::min(h->opt.gmres_restart, kMaxDots - 2));
  double* V = h->gm_V;
  double* Z = h->gm_Z;
  // basis vectors start on 64-byte boundaries: node loads are 32-byte vector accesses
  const int64_t ld = (n + 7) / 8 * 8;
  double* w = h->kw;
  AMG_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  c.dots(b, b, S_BB);
  const double bnorm = std::sqrt(read_scalar(h, S_BB));
  if (bnorm == 0.0) { st->iterations = 0; return AMG_OK; }
  DBuf<double> hcol, ydev;
  hcol.alloc(2 * kMaxDots);   // the two Gram-Schmidt passes' coefficients
  ydev.alloc(kMaxDots);
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), hc(2 * kMaxDots);
  int it = 0;
  double rel = 1.0;
  bool conv = false;
  auto mdot = [&](int cnt, const double* vec, double* out) {
    const int rows = (cnt + kMdotG - 1) / kMdotG;
    const int cols = (int)std::max<int64_t>(
        1, std::min<int64_t>(kReduceBlocks / rows, (n + 255) / 256));
    k_mdot<<<dim3(cols, rows), 256, 0, s>>>(n, cnt, V, ld, vec, h->red);
    k_mdot_final<<<(cnt + 7) / 8, 256, 0, s>>>(h->red, cols, cnt, out);
    h->launches += 2;
  };
  while (it < h->opt.max_iterations && !conv) {
    // r = b - K x, v_0 = r / ||r||
    apply_K(h, x, w);
    k_sub<<<gridr(n), 256, 0, s>>>(n, b, w, w);
    h->launches++;
    c.dots(w, w, S_T0);
    const double beta = std::sqrt(read_scalar(h, S_T0));
    if (beta == 0.0) { conv = true; rel = 0.0; break; }
    k_scale<<<gridr(n), 256, 0, s>>>(n, w, 1.0 / beta, V);
    h->launches++;
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jused = 0;
    for (int j = 0; j < m; ++j) {
      double* zj = Z + (int64_t)j * ld;
      precond(h, V + (int64_t)j * ld, zj);
      project_pressure(h, c, zj);
      apply_K(h, zj, w);
      // classical Gram-Schmidt, applied twice (CGS2)
      for (int pass = 0; pass < 2; ++pass) {
        double* coef = hcol.p + pass * kMaxDots;
        mdot(j + 1, w, coef);
        k_basis_sub<<<gridr(n), 256, 0, s>>>(n, j + 1, V, ld, coef, w);
        h->launches++;
      }
      c.dots(w, w, S_T0);
      // both passes' coefficients come back with the norm: one synchronisation
      AMG_CUDA(cudaMemcpyAsync(hc.data(), hcol.p, (kMaxDots + j + 1) * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
      const double hn = std::sqrt(read_scalar(h, S_T0));
      for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i <= j; ++i) H[i * m + j] += hc[pass * kMaxDots + i];
      H[(j + 1) * m + j] = hn;
      if (hn != 0.0) {
        k_scale<<<gridr(n), 256, 0, s>>>(n, w, 1.0 / hn, V + (int64_t)(j + 1) * ld);
        h->launches++;
      }
      for (int i = 0; i < j; ++i) {
        double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
      }
      double den = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
      cs[j] = H[j * m + j] / den;
      sn[j] = H[(j + 1) * m + j] / den;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      jused = j + 1;
      rel = std::fabs(g[j + 1]) / bnorm;
      if (!std::isfinite(rel)) fail(AMG_ERR_BREAKDOWN, "non-finite residual in FGMRES");
      if (rel <= tol || it >= h->opt.max_iterations || hn == 0.0) {
        conv = rel <= tol;
        break;
      }
    }
    // y = H^{-1} g (upper triangular), x += Z y
    std::vector<double> y(jused);
    for (int i = jused - 1; i >= 0; --i) {
      double t = g[i];
      for (int k = i + 1; k < jused; ++k) t -= H[i * m + k] * y[k];
      y[i] = t / H[i * m + i];
    }
    AMG_CUDA(cudaMemcpyAsync(ydev.p, y.data(), jused * sizeof(double), cudaMemcpyHostToDevice, s));
    k_basis_add<<<gridr(n), 256, 0, s>>>(n, jused, Z, ld, ydev.p, x);
    h->launches++;
    AMG_CUDA(cudaStreamSynchronize(s));
  }
  project_pressure(h, c, x);
  st->iterations = it;
  st->rel_residual = rel;
  st->true_rel_residual = true_residual(h, c, b, x) / bnorm;
  return (rel <= tol) ? AMG_OK : AMG_NOT_CONVERGED;
}

}  // namespace

int solve_device(amg_handle* h, const double* b_user, double* x_user, double tol,
                 amg_stats* st) {
  const Level& lv = *h->L[0];
  const int64_t n = lv.dofs4();
  Ctx c{h, h->stream, n};
  auto ensure = [&](DBuf<double>& v, int64_t cnt) {
    if ((int64_t)v.n < cnt) {
      v.alloc(cnt);
      AMG_CUDA(cudaMemsetAsync(v.p, 0, v.bytes(), h->stream));
    }
  };
  ensure(h->kb, n); ensure(h->kx, n);
  ensure(h->kr, n); ensure(h->kz, n); ensure(h->kp, n); ensure(h->kq, n); ensure(h->kw, n);
  if (lv.val2.p && (int64_t)h->kpf.n < 2 * n) {
    h->kpf.alloc(2 * n);
    AMG_CUDA(cudaMemsetAsync(h->kpf.p, 0, h->kpf.bytes(), h->stream));
  }
  ensure(h->red, (int64_t)kReduceBlocks * kMaxDots);
  ensure(h->scal, 64);
  if (!h->it_dev.p) h->it_dev.alloc(1);
  int krylov = h->opt.krylov;
  if (krylov == AMG_KRYLOV_AUTO)
    krylov = h->saddle ? AMG_KRYLOV_FGMRES
                       : (h->opt.precision == AMG_FP32 ? AMG_KRYLOV_FCG : AMG_KRYLOV_PCG);
  if (h->saddle && (krylov == AMG_KRYLOV_PCG || krylov == AMG_KRYLOV_FCG))
    fail(AMG_ERR_UNSUPPORTED, "CG needs an SPD system; use FGMRES for saddle kinds");
  launch_to_padded(b_user, h->kb, lv.n, lv.np, h->stream, h);
  const double* b = h->kb;
  double* x = h->kx;
  int rc;
  switch (krylov) {
    case AMG_KRYLOV_PCG:
      rc = solve_cg(h, c, b, x, tol, false, st);
      break;
    case AMG_KRYLOV_FCG:
      ensure(h->kro, n);
      rc = solve_cg(h, c, b, x, tol, true, st);
      break;
    case AMG_KRYLOV_NONE:
      rc = solve_amg(h, c, b, x, tol, st);
      break;
    case AMG_KRYLOV_FGMRES: {
      const int m = std::max(1, std::min(h->opt.gmres_restart, kMaxDots - 2));
      const int64_t ld = (n + 7) / 8 * 8;
      ensure(h->gm_V, (int64_t)(m + 1) * ld);
      ensure(h->gm_Z, (int64_t)m * ld);
      rc = solve_fgmres(h, c, b, x, tol, st);
      break;
    }
    default:
      fail(AMG_ERR_INVALID, "unknown Krylov method");
  }
  launch_from_padded(x, x_user, lv.n, lv.np, h->stream, h);
  return rc;
}

}  // namespace amgp2
