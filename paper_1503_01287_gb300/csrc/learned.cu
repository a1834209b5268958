// Learned smoother and correction weights, per level: block-diagonal statistics
// of every level (the network's inputs), the weights array of the cycle kernels
// (4 doubles a level), and the selection of each level's multipliers by the
// trained network with a measured fallback to the plain method (all weights 1).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "amg_internal.cuh"

namespace amgp2 {

namespace {

constexpr int kAcc = 8;   // accumulators of one level's statistics

__device__ __forceinline__ double frob(const double* v, int64_t nnzb, int64_t k) {
  double s = 0.0;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const double a = v[e * nnzb + k];
    s = fma(a, a, s);
  }
  return sqrt(s);
}

// Per non-Dirichlet node i of a level (D_i its diagonal block, A_ij the blocks
// of its row, Frobenius norms):
//   acc[0] += log10(|D_i| |D_i^-1|)     acc[1] += log10 |D_i|
//   acc[2] += (log10 |D_i|)^2          acc[3] += sum_{j != i} |A_ij| / |D_i|
//   acc[4] += 1
// and per non-Dirichlet F node with an interpolation row (state 2):
//   acc[5] += sum_{j C-node in P row i} |A_ij| / sum_{j != i} |A_ij|
//   acc[6] += number of entries of P row i        acc[7] += 1
__global__ void k_level_stats(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                              const double* __restrict__ val, int64_t nnzb,
                              const double* __restrict__ dinv, const int* __restrict__ tags,
                              const int* __restrict__ state, const int* __restrict__ cid,
                              const int* __restrict__ prow, const int* __restrict__ pcol,
                              double* __restrict__ acc) {
  double a[kAcc] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (tags[i] & AMG_NODE_DIRICHLET) continue;
    double dn = 0.0, off = 0.0, offc = 0.0;
    const bool fnode = state && state[i] == 2 && prow[i + 1] > prow[i];
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int j = col[k];
      const double f = frob(val, nnzb, k);
      if (j == i) {
        dn = f;
        continue;
      }
      off += f;
      if (fnode && state[j] == 1) {
        const int c = cid[j];
        for (int q = prow[i]; q < prow[i + 1]; ++q)
          if (pcol[q] == c) {
            offc += f;
            break;
          }
      }
    }
    const double* d = dinv + 12 * (int64_t)i;
    double di = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) di = fma(d[4 * r + c], d[4 * r + c], di);
    di = sqrt(di);
    const double ld = log10(dn);
    a[0] += log10(dn * di);
    a[1] += ld;
    a[2] += ld * ld;
    a[3] += off / dn;
    a[4] += 1.0;
    if (fnode) {
      a[5] += off > 0.0 ? offc / off : 0.0;
      a[6] += (double)(prow[i + 1] - prow[i]);
      a[7] += 1.0;
    }
  }
  __shared__ double red[kAcc][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int e = 0; e < kAcc; ++e) {
    double v = a[e];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[e][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < kAcc) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    atomicAdd(&acc[threadIdx.x], v);
  }
}

// acc[0] += C_kk / S_D[k], acc[1] += 1 over the pressure rows (S_D > 0)
__global__ void k_pres_stats(int np, const int* __restrict__ crow, const int* __restrict__ ccol,
                             const double* __restrict__ cval, const double* __restrict__ schur,
                             double* __restrict__ acc) {
  double s = 0.0, c = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
    double ckk = 0.0;
    for (int q = crow[k]; q < crow[k + 1]; ++q)
      if (ccol[q] == k) ckk = cval[q];
    if (schur[k] > 0.0) {
      s += ckk / schur[k];
      c += 1.0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], s);
    atomicAdd(&acc[1], c);
  }
}

// Counter-based uniform values in [-1, 1) (splitmix64 of seed + index), zero on
// Dirichlet nodes; user layout.
__global__ void k_probe_vector(int n, int np, const int* __restrict__ tags, uint64_t seed,
                               double* __restrict__ y) {
  const int64_t m = 3 * (int64_t)n + np;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    double v = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    if (i < 3 * (int64_t)n && (tags[i / 3] & AMG_NODE_DIRICHLET)) v = 0.0;
    y[i] = v;
  }
}

int grid_of(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 1216); }

}  // namespace

void compute_features(amg_handle* h, double* out) {
  cudaStream_t s = h->stream;
  const int nl = (int)h->L.size();
  DBuf<double> acc;
  acc.alloc(2 * kAcc + 2);
  AMG_CUDA(cudaMemsetAsync(acc.p, 0, acc.bytes(), s));
  for (int l = 0; l < std::min(nl, 2); ++l) {
    const Level& lv = *h->L[l];
    const bool has_p = l + 1 < nl;
    k_level_stats<<<grid_of(lv.n), 256, 0, s>>>(
        lv.n, lv.rowptr, lv.col, lv.val, lv.nnzb, lv.dinv, lv.tags, has_p ? lv.state.p : nullptr,
        has_p ? lv.cid.p : nullptr, has_p ? lv.p_rowptr.p : nullptr,
        has_p ? lv.p_col.p : nullptr, acc.p + kAcc * l);
    AMG_LAUNCH_CHECK();
    h->launches++;
  }
  const Level& l0 = *h->L[0];
  if (h->saddle && l0.np > 0 && l0.schur.p) {
    k_pres_stats<<<grid_of(l0.np), 256, 0, s>>>(l0.np, l0.c_rowptr, l0.c_col, l0.c_val, l0.schur,
                                                 acc.p + 2 * kAcc);
    AMG_LAUNCH_CHECK();
    h->launches++;
  }
  double a[2 * kAcc + 2];
  AMG_CUDA(cudaMemcpyAsync(a, acc.p, sizeof a, cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  out[0] = std::log10((double)l0.dofs()) / 7.0;
  for (int l = 0; l < 2; ++l) {
    const double* q = a + kAcc * l;
    double* f = out + 1 + 5 * l;
    const double cnt = q[4], fc = q[7];
    if (l >= nl || cnt <= 0.0) {
      for (int e = 0; e < 5; ++e) f[e] = 0.0;
      continue;
    }
    const double mean = q[1] / cnt;
    f[0] = q[0] / cnt;
    f[1] = std::sqrt(std::max(0.0, q[2] / cnt - mean * mean));
    f[2] = q[3] / cnt;
    f[3] = fc > 0.0 ? q[5] / fc : 0.0;
    f[4] = fc > 0.0 ? q[6] / fc / 8.0 : 0.0;
  }
  out[11] = a[2 * kAcc + 1] > 0.0 ? a[2 * kAcc] / a[2 * kAcc + 1] : 0.0;
  out[12] = h->saddle ? 1.0 : 0.0;
}

// The statistics accumulators of every level (kAcc each) and the pressure
// accumulators (2 each) of every saddle level with an sGS scaling.
static void level_stats_all(amg_handle* h, std::vector<double>& acc) {
  cudaStream_t s = h->stream;
  const int nl = (int)h->L.size();
  const int per = kAcc + 2;
  DBuf<double> dacc;
  dacc.alloc((size_t)per * nl);
  AMG_CUDA(cudaMemsetAsync(dacc.p, 0, dacc.bytes(), s));
  for (int l = 0; l < nl; ++l) {
    const Level& lv = *h->L[l];
    const bool has_p = l + 1 < nl;
    k_level_stats<<<grid_of(lv.n), 256, 0, s>>>(
        lv.n, lv.rowptr, lv.col, lv.val, lv.nnzb, lv.dinv, lv.tags, has_p ? lv.state.p : nullptr,
        has_p ? lv.cid.p : nullptr, has_p ? lv.p_rowptr.p : nullptr,
        has_p ? lv.p_col.p : nullptr, dacc.p + per * l);
    AMG_LAUNCH_CHECK();
    h->launches++;
    if (h->saddle && lv.np > 0 && lv.schur.p) {
      k_pres_stats<<<grid_of(lv.np), 256, 0, s>>>(lv.np, lv.c_rowptr, lv.c_col, lv.c_val,
                                                   lv.schur, dacc.p + per * l + kAcc);
      AMG_LAUNCH_CHECK();
      h->launches++;
    }
  }
  acc.assign((size_t)per * nl, 0.0);
  AMG_CUDA(cudaMemcpyAsync(acc.data(), dacc.p, acc.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
}

// the five statistics of a level from its accumulators (zeros without nodes)
static void stats5(const double* q, double* f) {
  const double cnt = q[4], fc = q[7];
  if (cnt <= 0.0) {
    for (int e = 0; e < 5; ++e) f[e] = 0.0;
    return;
  }
  const double mean = q[1] / cnt;
  f[0] = q[0] / cnt;
  f[1] = std::sqrt(std::max(0.0, q[2] / cnt - mean * mean));
  f[2] = q[3] / cnt;
  f[3] = fc > 0.0 ? q[5] / fc : 0.0;
  f[4] = fc > 0.0 ? q[6] / fc / 8.0 : 0.0;
}

static void level_features_from(const amg_handle* h, const std::vector<double>& acc, int l,
                                 double* out) {
  const int per = kAcc + 2;
  const Level& lv = *h->L[l];
  out[0] = std::log10((double)std::max(lv.dofs(), 1)) / 7.0;
  stats5(acc.data() + per * l, out + 1);
  double nx[5];
  stats5(acc.data() + per * (l + 1), nx);
  for (int e = 0; e < 4; ++e) out[6 + e] = nx[e];
  out[10] = l / 4.0;
  const double* pq = acc.data() + per * l + kAcc;
  out[11] = (h->saddle && pq[1] > 0.0) ? pq[0] / pq[1] : 0.0;
  out[12] = h->saddle ? 1.0 : 0.0;
}

void compute_level_features(amg_handle* h, int l, double* out) {
  if (l < 0 || l + 1 >= (int)h->L.size())
    fail(AMG_ERR_INVALID, "level features exist for the non-coarsest levels");
  std::vector<double> acc;
  level_stats_all(h, acc);
  level_features_from(h, acc, l, out);
}

void set_level_weights(amg_handle* h, const double* w, int n) {
  const int nl = (int)h->L.size();
  std::vector<double> v(4 * (size_t)nl, 1.0);
  for (int l = 0; l < nl && l < n; ++l)
    for (int e = 0; e < 3; ++e) v[4 * l + e] = w[3 * l + e];
  AMG_CUDA(cudaMemcpyAsync(h->wts.p, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice,
                           h->stream));
  AMG_CUDA(cudaStreamSynchronize(h->stream));
}

void set_weights(amg_handle* h, const double* w3) {
  const int nl = (int)h->L.size();
  std::vector<double> w(4 * (size_t)nl);
  for (int l = 0; l < nl; ++l) {
    w[4 * l + 0] = w3[0];
    w[4 * l + 1] = w3[1];
    w[4 * l + 2] = w3[2];
    w[4 * l + 3] = 1.0;
  }
  AMG_CUDA(cudaMemcpyAsync(h->wts.p, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice,
                           h->stream));
  AMG_CUDA(cudaStreamSynchronize(h->stream));
}

void get_weights(const amg_handle* h, double* out) {
  AMG_CUDA(cudaMemcpyAsync(out, h->wts.p, 4 * h->L.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream));
  AMG_CUDA(cudaStreamSynchronize(h->stream));
}

// Convergence factor of a short solve: rel_residual^(1/iterations) of the
// handle's Krylov method on b = K y (y a fixed pseudo-random vector) to 1e-8.
double probe_rate(amg_handle* h, DBuf<double>& b, DBuf<double>& x, int* iters) {
  amg_stats st{};
  AMG_CUDA(cudaMemsetAsync(x.p, 0, x.bytes(), h->stream));
  solve_device(h, b, x, kProbeTol, &st);
  AMG_CUDA(cudaStreamSynchronize(h->stream));
  *iters = st.iterations;
  if (st.iterations <= 0) return 0.0;
  const double r = std::max(st.rel_residual, 1e-300);
  return std::pow(r, 1.0 / st.iterations);
}

// Per-level selection: for every non-coarsest level the network predicts, for
// each candidate (ws, wc, wp) of the grid, the log10 ratio of the convergence
// factor with that level's multipliers changed (the others plain) to the plain
// factor; each level takes its grid argmin (the grid holds the plain point).
// Measured fallback: the combined choice is kept only if a probe solve to 1e-8
// converges faster per iteration than with the plain weights; otherwise the
// level with the largest predicted gain alone is probed, and otherwise the
// plain weights stay.
void learn_weights(amg_handle* h, const float* theta_host, amg_learned* out) {
  cudaStream_t s = h->stream;
  const int nl = (int)h->L.size();
  const int ns = std::max(nl - 1, 0);     // levels with multipliers that act
  std::vector<double> acc;
  level_stats_all(h, acc);
  // candidate grid: ws x wc (x log2 wp for saddle kinds)
  std::vector<double> W;
  const int nwp = h->saddle ? AMG_GRID_NWP : 1;
  for (int a = 0; a < AMG_GRID_NWS; ++a)
    for (int b = 0; b < AMG_GRID_NWC; ++b)
      for (int c = 0; c < nwp; ++c) {
        W.push_back(AMG_WS_MIN + (AMG_WS_MAX - AMG_WS_MIN) * a / (AMG_GRID_NWS - 1));
        W.push_back(AMG_WC_MIN + (AMG_WC_MAX - AMG_WC_MIN) * b / (AMG_GRID_NWC - 1));
        W.push_back(h->saddle ? AMG_WP_LOG2_MIN + (AMG_WP_LOG2_MAX - AMG_WP_LOG2_MIN) * c /
                                                      (AMG_GRID_NWP - 1)
                              : 0.0);
      }
  const int nc = (int)W.size() / 3;
  std::vector<float> X;
  X.reserve((size_t)ns * nc * AMG_MLP_INPUTS);
  for (int l = 0; l < ns; ++l) {
    double f[AMG_N_FEATURES];
    level_features_from(h, acc, l, f);
    for (int k = 0; k < nc; ++k) {
      for (int e = 0; e < AMG_N_FEATURES; ++e) X.push_back((float)f[e]);
      for (int e = 0; e < 3; ++e) X.push_back((float)W[3 * k + e]);
    }
  }
  std::memset(out, 0, sizeof(*out));
  out->n_candidates = nc;
  out->n_levels = nl;
  std::vector<double> plain(3 * (size_t)nl, 1.0), chosen(plain);
  std::vector<float> y((size_t)ns * nc, 0.f);
  if (ns > 0) {
    DBuf<float> dth, dx, dy;
    dth.alloc(mlp_nparam());
    dx.alloc(X.size());
    dy.alloc(y.size());
    AMG_CUDA(cudaMemcpyAsync(dth.p, theta_host, mlp_nparam() * sizeof(float),
                             cudaMemcpyHostToDevice, s));
    AMG_CUDA(cudaMemcpyAsync(dx.p, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice,
                             s));
    mlp_forward(dth, dx, (int)y.size(), dy, s);
    h->launches++;
    AMG_CUDA(cudaMemcpyAsync(y.data(), dy.p, y.size() * sizeof(float), cudaMemcpyDeviceToHost,
                             s));
    AMG_CUDA(cudaStreamSynchronize(s));
  }
  int l_best = -1;
  float gain_best = 0.f;
  for (int l = 0; l < ns; ++l) {
    const float* yl = y.data() + (size_t)l * nc;
    int best = 0;
    for (int k = 1; k < nc; ++k)
      if (yl[k] < yl[best]) best = k;
    chosen[3 * l + 0] = W[3 * best];
    chosen[3 * l + 1] = W[3 * best + 1];
    chosen[3 * l + 2] = std::exp2(W[3 * best + 2]);
    out->level_predicted[l] = yl[best];
    out->predicted += yl[best];
    if (yl[best] < gain_best) {
      gain_best = yl[best];
      l_best = l;
    }
  }
  // measured fallback on one probe system, b = K y with y fixed pseudo-random
  const Level& l0 = *h->L[0];
  const int64_t m = l0.dofs();
  DBuf<double> yv, b, x, ypad, bpad;
  yv.alloc(m);
  b.alloc(m);
  x.alloc(m);
  ypad.alloc(l0.dofs4());
  bpad.alloc(l0.dofs4());
  k_probe_vector<<<grid_of(m), 256, 0, s>>>(l0.n, l0.np, l0.tags, 0x5eedull, yv);
  AMG_LAUNCH_CHECK();
  launch_to_padded(yv, ypad, l0.n, l0.np, s, h);
  level_apply<double>(h, 0, ypad.p, bpad.p);
  launch_from_padded(bpad, b, l0.n, l0.np, s, h);
  int itp = 0, itl = 0;
  set_level_weights(h, plain.data(), nl);
  out->rho_plain = probe_rate(h, b, x, &itp);
  out->probe_iterations_plain = itp;
  const std::vector<double>* keep = &plain;
  std::vector<double> single(plain);
  if (chosen != plain) {
    set_level_weights(h, chosen.data(), nl);
    out->rho_learned = probe_rate(h, b, x, &itl);
    out->probe_iterations_learned = itl;
    if (out->rho_learned < out->rho_plain) keep = &chosen;
  }
  if (keep == &plain && l_best >= 0) {
    for (int e = 0; e < 3; ++e) single[3 * l_best + e] = chosen[3 * l_best + e];
    if (single != plain && single != chosen) {
      set_level_weights(h, single.data(), nl);
      int its = 0;
      const double rs = probe_rate(h, b, x, &its);
      if (rs < out->rho_plain) {
        keep = &single;
        out->rho_learned = rs;
        out->probe_iterations_learned = its;
      }
    }
  }
  out->fell_back = keep == &plain ? 1 : 0;
  if (out->fell_back) out->rho_learned = out->rho_learned > 0 ? out->rho_learned : out->rho_plain;
  set_level_weights(h, keep->data(), nl);
  for (int l = 0; l < nl && l < AMG_MAX_LEVELS; ++l)
    for (int e = 0; e < 3; ++e) out->level_weights[3 * l + e] = (*keep)[3 * l + e];
  for (int e = 0; e < 3; ++e) out->weights[e] = (*keep)[e];
}

}  // namespace amgp2
