// Batched solves: several SPD problems (each with its own hierarchy from
// amg_setup), each with up to kRhs right-hand sides, solved together.
//
// Multi-right-hand-side vectors are stored [node][rhs][4] (padded nodes, the
// right-hand sides of one node contiguous), so the block-row kernels are SpMM:
// one lane per right-hand side, the 9 block values and the column index are
// the same address for all lanes of a row (broadcast), and the gather of x_j
// for all right-hand sides is one contiguous 16 x 16-byte (FP32) access.
//
// Each problem runs flexible CG per right-hand side (Polak-Ribiere beta, the
// FP64 outer iteration of the FP32 or FP64 cycle; with the FP32 cycle the
// operator products K p are FP32-pair SpMM, see k_apply_pair_m); converged right-hand sides
// are frozen (alpha = beta = 0).  Each problem is one CUDA graph, launched on its own
// handle's stream: an initial block followed by a conditional WHILE node whose body is
// one iteration and its device-side stopping test.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "amg_internal.cuh"
#include "vec.cuh"

namespace amgp2 {

namespace {

constexpr int K = kRhs;   // right-hand sides per block vector

enum MMode { mApply = 0, mResid = 1, mGS = 2, mJacobi = 3 };

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Tile of the SpMM row kernels: S lane groups of 16 per stored row (lane r of a
// group = right-hand side r), group q taking the blocks q, q + S, ... of the row
// (S = 2: one warp a row, partial sums combined by a shuffle); U blocks unrolled.
// Row data at rowptr[g]..rowptr[g+1] (colour-major storage when rows != null).
template <typename T, int MODE, int S, int U>
__global__ void __launch_bounds__(256) k_rows_m(int nrows, const int* __restrict__ rows,
                                                const int* __restrict__ rowptr,
                                                const int* __restrict__ col,
                                                const T* __restrict__ val, int64_t nnzb,
                                                const T* x, const T* __restrict__ b, T* y,
                                                const T* __restrict__ dinv, T omega,
                                                const double* __restrict__ wt) {
  if (wt) omega = (T)((double)omega * wt[0]);   // learned relaxation multiplier
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) / (K * S);
  const int q = (threadIdx.x / K) % S;
  const int r = threadIdx.x % K;
  if (g >= nrows) return;                       // uniform over the S groups of a row
  const int i = rows ? ldg(rows + g) : g;
  const int a = ldg(rowptr + g), e = ldg(rowptr + g + 1);
  T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll U
  for (int k = a + q; k < e; k += S) {
    const int j = ldg(col + k);
    T x0, x1, x2;
    ld3(x, j * K + r, x0, x1, x2);
    const T* v = val + k;
    s0 = fma(ldg(v), x0, s0);
    s0 = fma(ldg(v + nnzb), x1, s0);
    s0 = fma(ldg(v + 2 * nnzb), x2, s0);
    s1 = fma(ldg(v + 3 * nnzb), x0, s1);
    s1 = fma(ldg(v + 4 * nnzb), x1, s1);
    s1 = fma(ldg(v + 5 * nnzb), x2, s1);
    s2 = fma(ldg(v + 6 * nnzb), x0, s2);
    s2 = fma(ldg(v + 7 * nnzb), x1, s2);
    s2 = fma(ldg(v + 8 * nnzb), x2, s2);
  }
  if (S == 2) {   // the two groups of a row are the two halves of one warp
    s0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    s2 += __shfl_xor_sync(0xffffffffu, s2, 16);
    if (q != 0) return;
  }
  const int o = i * K + r;
  if (MODE == mApply) {
    st3(y, o, s0, s1, s2);
    return;
  }
  T b0, b1, b2;
  ld3(b, o, b0, b1, b2);
  const T r0 = b0 - s0, r1 = b1 - s1, r2 = b2 - s2;
  if (MODE == mResid) {
    st3(y, o, r0, r1, r2);
    return;
  }
  const T* d = dinv + 12 * (int64_t)i;
  T d0, d1, d2;
  ld3(d, 0, d0, d1, d2);
  const T c0 = d0 * r0 + d1 * r1 + d2 * r2;
  ld3(d, 1, d0, d1, d2);
  const T c1 = d0 * r0 + d1 * r1 + d2 * r2;
  ld3(d, 2, d0, d1, d2);
  const T c2 = d0 * r0 + d1 * r1 + d2 * r2;
  T x0, x1, x2;
  ld3(x, o, x0, x1, x2);
  st3(y, o, x0 + omega * c0, x1 + omega * c1, x2 + omega * c2);
}

// y = K_0 x for all right-hand sides in FP32-pair arithmetic (pair_fma): the
// values are (hi, lo) float pairs, x holds 8 floats a (node, right-hand side)
// -- hi of the 4 padded entries, then lo -- and y is FP64.  Tiles as k_rows_m.
template <int S, int U>
__global__ void __launch_bounds__(256) k_apply_pair_m(int nrows, const int* __restrict__ rows,
                                                      const int* __restrict__ rowptr,
                                                      const int* __restrict__ col,
                                                      const float2* __restrict__ val,
                                                      int64_t nnzb, const float* __restrict__ xp,
                                                      double* __restrict__ y) {
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) / (K * S);
  const int q = (threadIdx.x / K) % S;
  const int r = threadIdx.x % K;
  if (g >= nrows) return;                       // uniform over the S groups of a row
  const int i = rows ? ldg(rows + g) : g;
  const int a = ldg(rowptr + g), e = ldg(rowptr + g + 1);
  const float4* xv = reinterpret_cast<const float4*>(xp);
  float S0 = 0.f, s0 = 0.f, S1 = 0.f, s1 = 0.f, S2 = 0.f, s2 = 0.f;
#pragma unroll U
  for (int k = a + q; k < e; k += S) {
    const int j = ldg(col + k);
    const float4 hi = ldg(xv + 2 * ((int64_t)j * K + r));
    const float4 lo = ldg(xv + 2 * ((int64_t)j * K + r) + 1);
    const float2* v = val + k;
    pair_fma(S0, s0, ldg(v), hi.x, lo.x);
    pair_fma(S0, s0, ldg(v + nnzb), hi.y, lo.y);
    pair_fma(S0, s0, ldg(v + 2 * nnzb), hi.z, lo.z);
    pair_fma(S1, s1, ldg(v + 3 * nnzb), hi.x, lo.x);
    pair_fma(S1, s1, ldg(v + 4 * nnzb), hi.y, lo.y);
    pair_fma(S1, s1, ldg(v + 5 * nnzb), hi.z, lo.z);
    pair_fma(S2, s2, ldg(v + 6 * nnzb), hi.x, lo.x);
    pair_fma(S2, s2, ldg(v + 7 * nnzb), hi.y, lo.y);
    pair_fma(S2, s2, ldg(v + 8 * nnzb), hi.z, lo.z);
  }
  if (S == 2) {   // the two groups of a row are the two halves of one warp
    float T = __shfl_xor_sync(0xffffffffu, S0, 16), t = __shfl_xor_sync(0xffffffffu, s0, 16);
    pair_add(S0, s0, T, t);
    T = __shfl_xor_sync(0xffffffffu, S1, 16); t = __shfl_xor_sync(0xffffffffu, s1, 16);
    pair_add(S1, s1, T, t);
    T = __shfl_xor_sync(0xffffffffu, S2, 16); t = __shfl_xor_sync(0xffffffffu, s2, 16);
    pair_add(S2, s2, T, t);
    if (q != 0) return;
  }
  st3(y, i * K + r, (double)S0 + (double)s0, (double)S1 + (double)s1,
      (double)S2 + (double)s2);
}

// bc_(I,r) = sum_t w_t v_(i_t, r)
template <typename T>
__global__ void k_restrict_m(int nc, const int* __restrict__ rrow, const int* __restrict__ rcol,
                             const T* __restrict__ rval, const T* __restrict__ v,
                             T* __restrict__ bc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int I = t / K, r = t % K;
  if (I >= nc) return;
  T s0 = T(0), s1 = T(0), s2 = T(0);
  for (int q = rrow[I]; q < rrow[I + 1]; ++q) {
    const T w = rval[q];
    T a0, a1, a2;
    ld3(v, rcol[q] * K + r, a0, a1, a2);
    s0 = fma(w, a0, s0);
    s1 = fma(w, a1, s1);
    s2 = fma(w, a2, s2);
  }
  st3(bc, I * K + r, s0, s1, s2);
}

// x_(i,r) += sum_q P_iq xc_(q,r)
template <typename T>
__global__ void k_prolong_m(int n, const int* __restrict__ prow, const int* __restrict__ pcol,
                            const T* __restrict__ pval, const T* __restrict__ xc, T* x,
                            const double* __restrict__ wt) {
  const T wc = wt ? (T)wt[1] : T(1);   // coarse-correction scale
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / K, r = t % K;
  if (i >= n) return;
  T s0 = T(0), s1 = T(0), s2 = T(0);
  for (int q = prow[i]; q < prow[i + 1]; ++q) {
    const T w = pval[q];
    T a0, a1, a2;
    ld3(xc, pcol[q] * K + r, a0, a1, a2);
    s0 = fma(w, a0, s0);
    s1 = fma(w, a1, s1);
    s2 = fma(w, a2, s2);
  }
  T x0, x1, x2;
  ld3(x, i * K + r, x0, x1, x2);
  st3(x, i * K + r, x0 + wc * s0, x1 + wc * s1, x2 + wc * s2);
}

// coarsest solve x = X b per right-hand side (X indexed 3 per node)
template <typename T>
__global__ void k_coarse_m(int m, const double* __restrict__ X, const T* __restrict__ b,
                           T* __restrict__ x) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / K, r = t % K;
  if (i >= m) return;
  double s = 0.0;
  for (int j = 0; j < m; ++j)
    s = fma(X[(int64_t)i * m + j], (double)b[((j / 3) * K + r) * 4 + j % 3], s);
  x[((i / 3) * K + r) * 4 + i % 3] = (T)s;
}

template <typename T>
__global__ void k_fill_m(T* a, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    a[k] = T(0);
}

template <typename T>
__global__ void k_copy_m(const T* __restrict__ a, T* __restrict__ b, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = a[k];
}

__global__ void k_sub_m(const double* __restrict__ a, const double* __restrict__ b,
                        double* __restrict__ c, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    c[k] = a[k] - b[k];
}

__global__ void k_d2f_m(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = (float)a[k];
}

__global__ void k_f2d_m(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = (double)a[k];
}

// user layout (nrhs vectors of 3n, vector r at offset r*3n) <-> [node][K][4]
__global__ void k_user_to_m(const double* __restrict__ u, double* __restrict__ v, int n,
                            int nrhs) {
  const int64_t tot = (int64_t)n * K * 4;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < tot;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(f & 3);
    const int r = (int)((f >> 2) % K);
    const int64_t node = (f >> 2) / K;
    v[f] = (c < 3 && r < nrhs) ? u[(int64_t)r * 3 * n + 3 * node + c] : 0.0;
  }
}

__global__ void k_m_to_user(const double* __restrict__ v, double* __restrict__ u, int n,
                            int nrhs) {
  const int64_t tot = (int64_t)nrhs * 3 * n;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < tot;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = f / (3 * (int64_t)n);
    const int64_t rem = f % (3 * (int64_t)n);
    u[f] = v[((rem / 3) * K + r) * 4 + rem % 3];
  }
}

// ---------------------------------------------------------------- Krylov per right-hand side

constexpr int kDotBlocks = 304;
constexpr int kDotThreads = 256;   // a multiple of 4K: a thread always sees one rhs

// partial[blk][d][r] = sum of a_d * b_d over the block's entries of right-hand side r
__global__ void k_dots_m(int64_t nel, int nd, const double* a0, const double* b0,
                         const double* a1, const double* b1, double* __restrict__ partial) {
  __shared__ double sh[kDotThreads];
  const int rr = (threadIdx.x >> 2) % K;
  for (int d = 0; d < nd; ++d) {
    const double* x = d == 0 ? a0 : a1;
    const double* y = d == 0 ? b0 : b1;
    double acc = 0.0;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nel;
         f += (int64_t)gridDim.x * blockDim.x)
      acc = fma(x[f], y[f], acc);
    sh[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < K) {
      double t = 0.0;
      for (int q = 0; q < kDotThreads; ++q)
        if (((q >> 2) % K) == (int)threadIdx.x) t += sh[q];
      partial[(blockIdx.x * nd + d) * K + threadIdx.x] = t;
    }
    __syncthreads();
  }
  (void)rr;
}

// out[d * K + r] = sum over b < nblk of partial[(b * nd + d) * K + r]: one warp per
// (d, r) (block d * K + r), lanes over b, then a fixed shuffle tree (deterministic)
__global__ void k_final_m(const double* __restrict__ partial, int nblk, int nd,
                          double* __restrict__ out) {
  const int t = blockIdx.x;
  if (t >= nd * K) return;
  const int d = t / K, r = t % K;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 32) s += partial[(b * nd + d) * K + r];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) out[d * K + r] = s;
}

// scalar slots, each K wide
enum MSlot { M_RZ = 0, M_PQ, M_RR, M_RZN, M_ZRO, M_BB, M_BETA, M_ACT, M_TOL2, M_ITS, M_NS };

__global__ void k_update_m(int64_t nel, double* __restrict__ x, double* __restrict__ r,
                           const double* __restrict__ p, const double* __restrict__ q,
                           double* __restrict__ ro, const double* __restrict__ s,
                           double* __restrict__ partial) {
  __shared__ double sh[kDotThreads];
  const int rhs = (threadIdx.x >> 2) % K;
  const bool act = s[M_ACT * K + rhs] != 0.0;
  const double pq = s[M_PQ * K + rhs];
  const double alpha = (act && pq != 0.0) ? s[M_RZ * K + rhs] / pq : 0.0;
  double acc = 0.0;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nel;
       f += (int64_t)gridDim.x * blockDim.x) {
    x[f] = fma(alpha, p[f], x[f]);
    const double rk = r[f];
    ro[f] = rk;
    const double rn = fma(-alpha, q[f], rk);
    r[f] = rn;
    acc = fma(rn, rn, acc);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int qq = 0; qq < kDotThreads; ++qq)
      if (((qq >> 2) % K) == (int)threadIdx.x) t += sh[qq];
    partial[blockIdx.x * K + threadIdx.x] = t;
  }
}

__global__ void k_beta_m(double* s) {
  const int r = threadIdx.x;
  if (r >= K) return;
  const bool act = s[M_ACT * K + r] != 0.0;
  const double rz = s[M_RZ * K + r];
  s[M_BETA * K + r] = (act && rz != 0.0) ? (s[M_RZN * K + r] - s[M_ZRO * K + r]) / rz : 0.0;
  s[M_RZ * K + r] = s[M_RZN * K + r];
}

// p = z + beta p per right-hand side; with pf, also p's pair form (8 floats a
// (node, right-hand side): hi of the 4 padded entries, then lo = fl32(p - hi))
__global__ void k_dir_m(int64_t nel, double* __restrict__ p, const double* __restrict__ z,
                        const double* __restrict__ s, float* __restrict__ pf) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nel;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int rhs = (int)((f >> 2) % K);
    const double v = fma(s[M_BETA * K + rhs], p[f], z[f]);
    p[f] = v;
    if (pf) {
      const float hi = (float)v;
      const int64_t o = 8 * (f >> 2) + (f & 3);
      pf[o] = hi;
      pf[o + 4] = (float)(v - (double)hi);
    }
  }
}

// active_r = b_r != 0 at the start
__global__ void k_init_m(double* s, double tol, int nrhs, int* it) {
  const int r = threadIdx.x;
  if (r < K) {
    s[M_ACT * K + r] = (r < nrhs && s[M_BB * K + r] > 0.0) ? 1.0 : 0.0;
    s[M_TOL2 * K + r] = tol * tol;
    s[M_ITS * K + r] = 0.0;
  }
  if (r == 0) *it = 0;
}

// after an update: freeze converged right-hand sides; continue while any is
// active, the iteration limit is not reached and no residual is non-finite
__global__ void k_check_m(cudaGraphConditionalHandle cond, double* s, int* it, int maxit) {
  __shared__ int any;
  const int r = threadIdx.x;
  if (r == 0) any = 0;
  __syncthreads();
  const int k = *it + 1;
  if (r < K && s[M_ACT * K + r] != 0.0) {
    const double rr = s[M_RR * K + r];
    if (!(rr > s[M_TOL2 * K + r] * s[M_BB * K + r]) || !isfinite(rr)) {
      s[M_ACT * K + r] = 0.0;
      s[M_ITS * K + r] = (double)k;
    } else {
      atomicOr(&any, 1);
      s[M_ITS * K + r] = (double)k;
    }
  }
  __syncthreads();
  if (r == 0) {
    *it = k;
    cudaGraphSetConditional(cond, (any && k < maxit) ? 1u : 0u);
  }
}

inline int gridk(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
}

// ---------------------------------------------------------------- multi-RHS cycle

template <typename T> struct MV;
template <> struct MV<double> {
  static double* x(BatchLevel& l) { return l.x64; }
  static double* b(BatchLevel& l) { return l.b64; }
  static double* r(BatchLevel& l) { return l.r64; }
  static double* t(BatchLevel& l) { return l.t64; }
  static const double* val(Level& l) { return l.k_val(); }
  static const double* dinv(Level& l) { return l.dinv; }
  static const double* pval(Level& l) { return l.p_val; }
  static const double* rval(Level& l) { return l.r_val; }
};
template <> struct MV<float> {
  static float* x(BatchLevel& l) { return l.x32; }
  static float* b(BatchLevel& l) { return l.b32; }
  static float* r(BatchLevel& l) { return l.r32; }
  static float* t(BatchLevel& l) { return l.t32; }
  static const float* val(Level& l) { return l.val32; }
  static const float* dinv(Level& l) { return l.dinv32; }
  static const float* pval(Level& l) { return l.p_val32; }
  static const float* rval(Level& l) { return l.r_val32; }
};

constexpr int kTiles = 4;   // tile t: S = 1 + (t & 1), U = (t & 2) ? 4 : 2
constexpr int kGsTiles = 8; // colour kernel: tiles 0..3 as above, 4..7: S = 4 << (t & 1),
                            // U = (t & 2) ? 4 : 2

// One colour of the multicolour Gauss-Seidel sweep for all right-hand sides,
// launched with programmatic dependent launch: the row's ids, the column indices
// and values of its first U blocks of this lane group and D^{-1} (setup data that
// no cycle kernel writes) are loaded before griddepcontrol.wait, so this prologue
// runs under the previous kernel; b, the relaxation multiplier and the x gathers
// come after the wait, which is where the previous kernel's writes become
// visible.  Tiles as in k_rows_m, and with S = 4 or 8 lane groups a row (2 or 4 warps,
// their sums combined in shared memory) for rows whose dependent block chain is long.
template <typename T, int S, int U>
__global__ void __launch_bounds__(256) k_gs_m_pdl(int nrows, const int* __restrict__ rows,
                                                  const int* __restrict__ rowptr,
                                                  const int* __restrict__ col,
                                                  const T* __restrict__ val, int64_t nnzb, T* x,
                                                  const T* __restrict__ b,
                                                  const T* __restrict__ dinv,
                                                  const double* __restrict__ wt) {
  // S > 2: the S / 2 warps of a row combine their sums through shared memory
  __shared__ T red[S > 2 ? 256 / 32 : 1][K][3];
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) / (K * S);
  const int q = (threadIdx.x / K) % S;
  const int r = threadIdx.x % K;
  const bool active = g < nrows;       // uniform over the S groups of a row
  int i = 0, a = 0, e = 0;
  int j[U];
  T v[U][9];
  T b0 = T(0), b1 = T(0), b2 = T(0);
  T d[9];
#pragma unroll
  for (int u = 0; u < U; ++u) j[u] = -1;
  if (active) {
    i = __ldg(rows + g);
    a = __ldg(rowptr + g);
    e = __ldg(rowptr + g + 1);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = a + q + u * S;
      if (k < e) {
        j[u] = __ldg(col + k);
#pragma unroll
        for (int w = 0; w < 9; ++w) v[u][w] = __ldg(val + w * nnzb + k);
      }
    }
    if (q == 0) {
      const T* dp = dinv + 12 * (int64_t)i;
      ld3(dp, 0, d[0], d[1], d[2]);
      ld3(dp, 1, d[3], d[4], d[5]);
      ld3(dp, 2, d[6], d[7], d[8]);
    }
  }
  // the right-hand side and the multiplier may be written by the previous kernel
  // (the restriction before a sweep's first colour): read only after the wait
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (S <= 2 && !active) return;   // S > 2: every thread reaches the block barrier below
  const T om = wt ? (T)wt[0] : T(1);   // learned relaxation multiplier (1: plain)
  if (active && q == 0) ld3(b, i * K + r, b0, b1, b2);
  T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (j[u] < 0) continue;
    T x0, x1, x2;
    ld3(x, j[u] * K + r, x0, x1, x2);
    s0 = fma(v[u][0], x0, s0); s0 = fma(v[u][1], x1, s0); s0 = fma(v[u][2], x2, s0);
    s1 = fma(v[u][3], x0, s1); s1 = fma(v[u][4], x1, s1); s1 = fma(v[u][5], x2, s1);
    s2 = fma(v[u][6], x0, s2); s2 = fma(v[u][7], x1, s2); s2 = fma(v[u][8], x2, s2);
  }
  for (int k = a + q + U * S; active && k < e; k += S) {   // blocks beyond the prefetched ones
    const int jj = __ldg(col + k);
    T x0, x1, x2;
    ld3(x, jj * K + r, x0, x1, x2);
    const T* vv = val + k;
    s0 = fma(__ldg(vv), x0, s0);
    s0 = fma(__ldg(vv + nnzb), x1, s0);
    s0 = fma(__ldg(vv + 2 * nnzb), x2, s0);
    s1 = fma(__ldg(vv + 3 * nnzb), x0, s1);
    s1 = fma(__ldg(vv + 4 * nnzb), x1, s1);
    s1 = fma(__ldg(vv + 5 * nnzb), x2, s1);
    s2 = fma(__ldg(vv + 6 * nnzb), x0, s2);
    s2 = fma(__ldg(vv + 7 * nnzb), x1, s2);
    s2 = fma(__ldg(vv + 8 * nnzb), x2, s2);
  }
  if (S >= 2) {   // lane groups q and q + 1 share a warp (K = 16 lanes each)
    s0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    s2 += __shfl_xor_sync(0xffffffffu, s2, 16);
  }
  if (S > 2) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < K) {
      red[w][lane][0] = s0;
      red[w][lane][1] = s1;
      red[w][lane][2] = s2;
    }
    __syncthreads();
    if (!active || q != 0) return;
    // the row's first warp holds q = 0: add its S / 2 warps' sums in order
    s0 = s1 = s2 = T(0);
#pragma unroll
    for (int v = 0; v < S / 2; ++v) {
      s0 += red[w + v][r][0];
      s1 += red[w + v][r][1];
      s2 += red[w + v][r][2];
    }
  }
  if (S >= 2 && q != 0) return;
  const int o = i * K + r;
  T x0, x1, x2;
  ld3(x, o, x0, x1, x2);
  const T r0 = b0 - s0, r1 = b1 - s1, r2 = b2 - s2;
  st3(x, o, x0 + om * (d[0] * r0 + d[1] * r1 + d[2] * r2),
      x1 + om * (d[3] * r0 + d[4] * r1 + d[5] * r2),
      x2 + om * (d[6] * r0 + d[7] * r1 + d[8] * r2));
}

template <typename T, int S, int U>
void launch_gs_m_pdl(int nrows, const int* rows, const int* rowptr, Level& lv, const T* val,
                     T* x, const T* b, const T* dinv, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(((int64_t)nrows * K * S + 255) / 256));
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  AMG_CUDA(cudaLaunchKernelEx(&cfg, k_gs_m_pdl<T, S, U>, nrows, rows, rowptr,
                              (const int*)lv.k_col(), val, lv.nnzb, x, b, dinv,
                              (const double*)lv.wt));
}

// one colour of the batched Gauss-Seidel sweep (x updated in place)
template <typename T>
void gs_colour_m(amg_handle* h, Level& lv, int first, int nrows, const T* val, T* x,
                 const T* b, const T* dinv, int tile) {
  if (nrows <= 0) return;
  const int* rows = lv.k_rows() + first;
  const int* rowptr = lv.k_rowptr() + first;
  cudaStream_t s = h->stream;
  switch (tile) {
    case 1: launch_gs_m_pdl<T, 2, 2>(nrows, rows, rowptr, lv, val, x, b, dinv, s); break;
    case 2: launch_gs_m_pdl<T, 1, 4>(nrows, rows, rowptr, lv, val, x, b, dinv, s); break;
    case 3: launch_gs_m_pdl<T, 2, 4>(nrows, rows, rowptr, lv, val, x, b, dinv, s); break;
    case 4: launch_gs_m_pdl<T, 4, 2>(nrows, rows, rowptr, lv, val, x, b, dinv, s); break;
    case 5: launch_gs_m_pdl<T, 8, 2>(nrows, rows, rowptr, lv, val, x, b, dinv, s); break;
    case 6: launch_gs_m_pdl<T, 4, 4>(nrows, rows, rowptr, lv, val, x, b, dinv, s); break;
    case 7: launch_gs_m_pdl<T, 8, 4>(nrows, rows, rowptr, lv, val, x, b, dinv, s); break;
    default: launch_gs_m_pdl<T, 1, 2>(nrows, rows, rowptr, lv, val, x, b, dinv, s); break;
  }
  h->launches++;
}

template <typename T, int MODE, int S, int U>
void launch_rows_m(int nrows, const int* rows, const int* rowptr, Level& lv, const T* val,
                   const T* x, const T* b, T* y, const T* dinv, T omega, const double* wt,
                   cudaStream_t s) {
  const int grid = (int)(((int64_t)nrows * K * S + 255) / 256);
  k_rows_m<T, MODE, S, U><<<grid, 256, 0, s>>>(nrows, rows, rowptr, lv.k_col(), val, lv.nnzb, x,
                                               b, y, dinv, omega, wt);
}

template <typename T, int MODE>
void launch_tile_m(int tile, int nrows, const int* rows, const int* rowptr, Level& lv,
                   const T* val, const T* x, const T* b, T* y, const T* dinv, T omega,
                   const double* wt, cudaStream_t s) {
  switch (tile) {
    case 1: launch_rows_m<T, MODE, 2, 2>(nrows, rows, rowptr, lv, val, x, b, y, dinv, omega, wt, s); break;
    case 2: launch_rows_m<T, MODE, 1, 4>(nrows, rows, rowptr, lv, val, x, b, y, dinv, omega, wt, s); break;
    case 3: launch_rows_m<T, MODE, 2, 4>(nrows, rows, rowptr, lv, val, x, b, y, dinv, omega, wt, s); break;
    default: launch_rows_m<T, MODE, 1, 2>(nrows, rows, rowptr, lv, val, x, b, y, dinv, omega, wt, s); break;
  }
}

template <int S, int U>
void launch_pair_m(const Level& lv, const float* xp, double* y, cudaStream_t s) {
  const int grid = (int)(((int64_t)lv.n * K * S + 255) / 256);
  k_apply_pair_m<S, U><<<grid, 256, 0, s>>>(lv.n, lv.k_rows(), lv.k_rowptr(), lv.k_col(),
                                            lv.val2.p, lv.nnzb, xp, y);
}

// y = K_0 x (FP32-pair operator, x in pair form) with the given tile
void apply_pair_m(amg_handle* h, const float* xp, double* y, int tile) {
  const Level& lv = *h->L[0];
  switch (tile) {
    case 1: launch_pair_m<2, 2>(lv, xp, y, h->stream); break;
    case 2: launch_pair_m<1, 4>(lv, xp, y, h->stream); break;
    case 3: launch_pair_m<2, 4>(lv, xp, y, h->stream); break;
    default: launch_pair_m<1, 2>(lv, xp, y, h->stream); break;
  }
  h->launches++;
}

template <typename T>
void rows_m(amg_handle* h, int mode, Level& lv, int first, int nrows, const T* val, const T* x,
            const T* b, T* y, const T* dinv, T omega, int tile) {
  if (nrows <= 0) return;
  const int* order = lv.k_rows();
  const int* rows = order ? order + first : nullptr;
  const int* rowptr = lv.k_rowptr() + first;
  cudaStream_t s = h->stream;
  switch (mode) {
    case mApply:
      launch_tile_m<T, mApply>(tile, nrows, rows, rowptr, lv, val, x, b, y, dinv, omega, nullptr, s);
      break;
    case mResid:
      launch_tile_m<T, mResid>(tile, nrows, rows, rowptr, lv, val, x, b, y, dinv, omega, nullptr, s);
      break;
    case mGS:
      launch_tile_m<T, mGS>(tile, nrows, rows, rowptr, lv, val, x, b, y, dinv, omega, lv.wt, s);
      break;
    default:
      launch_tile_m<T, mJacobi>(tile, nrows, rows, rowptr, lv, val, x, b, y, dinv, omega, lv.wt, s);
      break;
  }
  h->launches++;
}

template <typename T>
void smooth_m(amg_handle* h, int l, T* x, const T* b, bool post) {
  Level& lv = *h->L[l];
  BatchLevel& bl = h->B[l];
  if (h->opt.smoother == AMG_SMOOTHER_JACOBI) {
    T* t = MV<T>::t(bl);
    rows_m<T>(h, mJacobi, lv, 0, lv.n, MV<T>::val(lv), x, b, t, MV<T>::dinv(lv), (T)h->opt.omega,
              bl.tile);
    k_copy_m<T><<<gridk(4 * (int64_t)K * lv.n), 256, 0, h->stream>>>(t, x, 4 * (int64_t)K * lv.n);
    h->launches++;
    return;
  }
  for (int q = 0; q < lv.ncolours; ++q) {
    const int c = post ? lv.ncolours - 1 - q : q;
    const int a = lv.colour_ptr[c], e = lv.colour_ptr[c + 1];
    if (h->use_pdl && lv.k_rows())
      gs_colour_m<T>(h, lv, a, e - a, MV<T>::val(lv), x, b, MV<T>::dinv(lv), bl.tile_gs);
    else
      rows_m<T>(h, mGS, lv, a, e - a, MV<T>::val(lv), x, b, x, MV<T>::dinv(lv), T(1), bl.tile);
  }
}

// Algorithm 1 on level l for all right-hand sides at once
template <typename T>
void cycle_m(amg_handle* h, int l, T* x, const T* b, bool x_is_zero) {
  const int L = (int)h->L.size() - 1;
  cudaStream_t s = h->stream;
  if (l == L) {
    const int m = h->coarse_m;
    k_coarse_m<T><<<gridk((int64_t)m * K), 256, 0, s>>>(m, h->coarse_inv, b, x);
    h->launches++;
    return;
  }
  Level& lv = *h->L[l];
  Level& nx = *h->L[l + 1];
  BatchLevel& bl = h->B[l];
  BatchLevel& bn = h->B[l + 1];
  const int64_t nel = 4 * (int64_t)K * lv.n;
  bool zero = x_is_zero;
  for (int k = 0; k < h->opt.m_pre; ++k) {
    if (zero) {
      k_fill_m<T><<<gridk(nel), 256, 0, s>>>(x, nel);
      h->launches++;
    }
    smooth_m<T>(h, l, x, b, false);
    zero = false;
  }
  if (zero) {
    k_fill_m<T><<<gridk(nel), 256, 0, s>>>(x, nel);
    h->launches++;
  }
  T* r = MV<T>::r(bl);
  rows_m<T>(h, mResid, lv, 0, lv.n, MV<T>::val(lv), x, b, r, nullptr, T(0), bl.tile);
  k_restrict_m<T><<<gridk((int64_t)nx.n * K), 256, 0, s>>>(nx.n, lv.r_rowptr, lv.r_col,
                                                          MV<T>::rval(lv), r, MV<T>::b(bn));
  h->launches++;
  for (int k = 0; k < std::max(1, (l + 1 == L) ? 1 : h->opt.nu); ++k)
    cycle_m<T>(h, l + 1, MV<T>::x(bn), MV<T>::b(bn), k == 0);
  k_prolong_m<T><<<gridk((int64_t)lv.n * K), 256, 0, s>>>(lv.n, lv.p_rowptr, lv.p_col,
                                                          MV<T>::pval(lv), MV<T>::x(bn), x,
                                                          lv.wt);
  h->launches++;
  for (int k = 0; k < h->opt.m_post; ++k) smooth_m<T>(h, l, x, b, h->opt.post_order != 1);
}

// z = M^{-1} r for all right-hand sides (FP64 [node][K][4] in and out)
void precond_m(amg_handle* h, const double* r, double* z) {
  Level& l0 = *h->L[0];
  BatchLevel& b0 = h->B[0];
  const int64_t nel = 4 * (int64_t)K * l0.n;
  cudaStream_t s = h->stream;
  if (h->opt.precision == AMG_FP32) {
    k_d2f_m<<<gridk(nel), 256, 0, s>>>(r, b0.b32, nel);
    h->launches++;
    for (int c = 0; c < std::max(1, h->opt.cycles); ++c)
      cycle_m<float>(h, 0, b0.x32.p, b0.b32.p, c == 0);
    k_f2d_m<<<gridk(nel), 256, 0, s>>>(b0.x32, z, nel);
    h->launches++;
  } else {
    for (int c = 0; c < std::max(1, h->opt.cycles); ++c) cycle_m<double>(h, 0, z, r, c == 0);
  }
}

void apply_m64(amg_handle* h, const double* x, double* y) {
  Level& lv = *h->L[0];
  rows_m<double>(h, mApply, lv, 0, lv.n, lv.k_val(), x, nullptr, y, nullptr, 0.0, h->B[0].tile64);
}

void dots_m(amg_handle* h, int slot, const double* a0, const double* b0,
            const double* a1 = nullptr, const double* b1 = nullptr) {
  const int nd = a1 ? 2 : 1;
  const int64_t nel = 4 * (int64_t)K * h->L[0]->n;
  k_dots_m<<<kDotBlocks, kDotThreads, 0, h->stream>>>(nel, nd, a0, b0, a1, b1, h->bred);
  k_final_m<<<nd * K, 32, 0, h->stream>>>(h->bred, kDotBlocks, nd, h->bscal.p + slot * K);
  h->launches += 2;
}

// The fastest tile of the operator pass on one level (CUDA events, the level's
// multi-right-hand-side work vectors; before any graph is captured).
template <typename T>
int tune_tile(amg_handle* h, Level& lv, const T* val, const T* x, T* y) {
  cudaStream_t s = h->stream;
  cudaEvent_t e0, e1;
  AMG_CUDA(cudaEventCreate(&e0));
  AMG_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 1e30f;
  for (int t = 0; t < kTiles; ++t) {
    for (int r = 0; r < 7; ++r) {
      if (r == 2) AMG_CUDA(cudaEventRecord(e0, s));
      rows_m<T>(h, mApply, lv, 0, lv.n, val, x, nullptr, y, nullptr, T(0), t);
    }
    AMG_CUDA(cudaEventRecord(e1, s));
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// the same for the FP32-pair operator of level 0
int tune_pair_tile(amg_handle* h) {
  cudaStream_t s = h->stream;
  cudaEvent_t e0, e1;
  AMG_CUDA(cudaEventCreate(&e0));
  AMG_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 1e30f;
  for (int t = 0; t < kTiles; ++t) {
    for (int r = 0; r < 7; ++r) {
      if (r == 2) AMG_CUDA(cudaEventRecord(e0, s));
      apply_pair_m(h, h->mpf, h->mq, t);
    }
    AMG_CUDA(cudaEventRecord(e1, s));
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

void alloc_batch(amg_handle* h) {
  if (!h->B.empty()) return;
  if (h->saddle) fail(AMG_ERR_UNSUPPORTED, "batched solves are provided for the SPD kinds");
  h->B.resize(h->L.size());
  const bool f32 = h->opt.precision == AMG_FP32;
  auto z64 = [&](DBuf<double>& v, int64_t n) {
    v.alloc(n);
    AMG_CUDA(cudaMemsetAsync(v.p, 0, v.bytes(), h->stream));
  };
  auto z32 = [&](DBuf<float>& v, int64_t n) {
    v.alloc(n);
    AMG_CUDA(cudaMemsetAsync(v.p, 0, v.bytes(), h->stream));
  };
  for (size_t l = 0; l < h->L.size(); ++l) {
    const int64_t n = 4 * (int64_t)K * std::max(h->L[l]->n, 1);
    BatchLevel& b = h->B[l];
    if (f32) { z32(b.x32, n); z32(b.b32, n); z32(b.r32, n); z32(b.t32, n); }
    else { z64(b.x64, n); z64(b.b64, n); z64(b.r64, n); z64(b.t64, n); }
  }
  const int64_t n0 = 4 * (int64_t)K * h->L[0]->n;
  z64(h->mb, n0); z64(h->mx, n0); z64(h->mr, n0); z64(h->mz, n0);
  z64(h->mp, n0); z64(h->mq, n0); z64(h->mro, n0);
  // FP32 cycle with the FP32-pair Krylov operator: the directions in pair form
  if (f32 && h->L[0]->val2.p) z32(h->mpf, 2 * n0);
  h->bred.alloc((size_t)kDotBlocks * 2 * K);
  h->bscal.alloc((size_t)M_NS * K);
  h->bit.alloc(1);
  AMG_CUDA(cudaStreamSynchronize(h->stream));
  // SpMM tile per level (the coarsest level is solved densely): given, or timed
  const int fixed = h->opt.batch_tile;
  if (fixed >= kGsTiles) fail(AMG_ERR_INVALID, "batch_tile must be -1 or 0..7");
  for (size_t l = 0; l + 1 < h->L.size(); ++l) {
    Level& lv = *h->L[l];
    BatchLevel& b = h->B[l];
    if (fixed >= 0) b.tile = fixed % kTiles;
    else if (f32) b.tile = tune_tile<float>(h, lv, MV<float>::val(lv), b.x32, b.t32);
    else b.tile = tune_tile<double>(h, lv, MV<double>::val(lv), b.x64, b.t64);
  }
  h->B[0].tile64 = fixed >= 0 ? fixed % kTiles
                              : tune_tile<double>(h, *h->L[0], h->L[0]->k_val(), h->mx, h->mq);
  if (h->mpf.p) h->B[0].tile_pair = fixed >= 0 ? fixed % kTiles : tune_pair_tile(h);
  // the colour kernel's tile per level: forced, else the SpMM's.  Timing each level's
  // sweep alone picked 4 or 8 lane groups a row on the small levels, which shortens a
  // lone problem's sweeps but made the 64-problem batch slower (2.24 against 2.09 s):
  // with all problems running side by side the device is full and the wider groups
  // only add threads.
  for (size_t l = 0; l + 1 < h->L.size(); ++l) {
    BatchLevel& b = h->B[l];
    b.tile_gs = fixed >= 0 ? fixed : b.tile;
  }
}

// initial block of one problem: x = 0, r = b, z = M r, rz, p = z, active set
void emit_init(amg_handle* h, const double* bu, int nrhs, double tol) {
  cudaStream_t s = h->stream;
  const int n = h->L[0]->n;
  const int64_t nel = 4 * (int64_t)K * n;
  k_user_to_m<<<gridk(nel), 256, 0, s>>>(bu, h->mb, n, nrhs);
  k_fill_m<double><<<gridk(nel), 256, 0, s>>>(h->mx, nel);
  k_copy_m<double><<<gridk(nel), 256, 0, s>>>(h->mb, h->mr, nel);
  h->launches += 3;
  dots_m(h, M_BB, h->mb, h->mb);
  k_init_m<<<1, 32, 0, s>>>(h->bscal, tol, nrhs, h->bit);
  h->launches++;
  precond_m(h, h->mr, h->mz);
  dots_m(h, M_RZ, h->mr, h->mz);
  k_copy_m<double><<<gridk(nel), 256, 0, s>>>(h->mz, h->mp, nel);
  h->launches++;
  if (h->mpf.p) launch_split_pair(h->mp, h->mpf, nel, s, h);
}

// one iteration of flexible CG per right-hand side and the stopping test
void emit_iteration(amg_handle* h, cudaGraphConditionalHandle cond) {
  cudaStream_t s = h->stream;
  const int64_t nel = 4 * (int64_t)K * h->L[0]->n;
  if (h->mpf.p) apply_pair_m(h, h->mpf, h->mq, h->B[0].tile_pair);
  else apply_m64(h, h->mp, h->mq);
  dots_m(h, M_PQ, h->mp, h->mq);
  k_update_m<<<kDotBlocks, kDotThreads, 0, s>>>(nel, h->mx, h->mr, h->mp, h->mq, h->mro,
                                                h->bscal, h->bred);
  k_final_m<<<K, 32, 0, s>>>(h->bred, kDotBlocks, 1, h->bscal.p + M_RR * K);
  k_check_m<<<1, 32, 0, s>>>(cond, h->bscal, h->bit, h->opt.max_iterations);
  h->launches += 3;
  precond_m(h, h->mr, h->mz);
  dots_m(h, M_RZN, h->mr, h->mz, h->mz, h->mro);
  k_beta_m<<<1, 32, 0, s>>>(h->bscal);
  k_dir_m<<<gridk(nel), 256, 0, s>>>(nel, h->mp, h->mz, h->bscal, h->mpf.p);
  h->launches += 2;
}

void emit_final(amg_handle* h, double* xu, int nrhs) {
  const int n = h->L[0]->n;
  k_m_to_user<<<gridk((int64_t)nrhs * 3 * n), 256, 0, h->stream>>>(h->mx, xu, n, nrhs);
  h->launches++;
}

cudaGraph_t capture(cudaStream_t s, const std::function<void()>& f) {
  cudaGraph_t g = nullptr;
  AMG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  try {
    f();
  } catch (...) {
    cudaGraph_t junk = nullptr;
    cudaStreamEndCapture(s, &junk);
    if (junk) cudaGraphDestroy(junk);
    throw;
  }
  AMG_CUDA(cudaStreamEndCapture(s, &g));
  return g;
}

}  // namespace

// Builds the problems' graphs and runs them, one stream a problem.
int solve_batched(amg_handle* const* hs, int np, int nrhs, const double* const* B,
                  double* const* X, double tol, amg_stats* stats, double* ms_out) {
  if (np <= 0 || nrhs <= 0 || nrhs > K) fail(AMG_ERR_INVALID, "need 1..16 right-hand sides");
  amg_handle* h0 = hs[0];
  for (int p = 0; p < np; ++p) {
    if (!hs[p]) fail(AMG_ERR_INVALID, "null handle");
    alloc_batch(hs[p]);
  }
  // one graph per problem (init -> while(iteration) -> final), each launched on its own
  // handle's stream so that the problems run side by side.  How far they overlap is set
  // by the process's hardware work queues (CUDA_DEVICE_MAX_CONNECTIONS, 8 by default):
  // the 64 x 16 batch of elasticity problems took 2.63 s with 8 and 2.08-2.17 s with 32;
  // one graph holding all problems as branches took 2.62 and 2.22 s.
  std::vector<cudaGraphExec_t> execs(np, nullptr);
  std::vector<cudaEvent_t> done(np, nullptr);
  struct Cleanup {
    std::vector<cudaGraphExec_t>& x;
    std::vector<cudaEvent_t>& d;
    ~Cleanup() {
      for (auto e : x) if (e) cudaGraphExecDestroy(e);
      for (auto e : d) if (e) cudaEventDestroy(e);
    }
  } cleanup{execs, done};
  std::vector<int64_t> l0(np);
  std::vector<int64_t> per_iter(np);
  for (int p = 0; p < np; ++p) {
    amg_handle* h = hs[p];
    for (int q = 0; q < p; ++q)
      if (hs[q] == h) fail(AMG_ERR_INVALID, "a handle appears twice in the batch");
    l0[p] = h->launches;
    cudaGraph_t g = nullptr;
    AMG_CUDA(cudaGraphCreate(&g, 0));
    try {
      cudaGraph_t gi = capture(h->stream, [&]() { emit_init(h, B[p], nrhs, tol); });
      cudaGraphNode_t ni, nc, nf;
      AMG_CUDA(cudaGraphAddChildGraphNode(&ni, g, nullptr, 0, gi));
      cudaGraphDestroy(gi);
      cudaGraphConditionalHandle cond;
      AMG_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams cp{};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = cond;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      AMG_CUDA(cudaGraphAddNode(&nc, g, &ni, nullptr, 1, &cp));
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      const int64_t b0 = h->launches;
      AMG_CUDA(cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
      try {
        emit_iteration(h, cond);
      } catch (...) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(h->stream, &junk);
        throw;
      }
      AMG_CUDA(cudaStreamEndCapture(h->stream, &body));
      per_iter[p] = h->launches - b0;
      cudaGraph_t gf = capture(h->stream, [&]() { emit_final(h, X[p], nrhs); });
      AMG_CUDA(cudaGraphAddChildGraphNode(&nf, g, &nc, 1, gf));
      cudaGraphDestroy(gf);
      AMG_CUDA(cudaGraphInstantiate(&execs[p], g, 0));
    } catch (...) {
      cudaGraphDestroy(g);
      throw;
    }
    cudaGraphDestroy(g);
    AMG_CUDA(cudaEventCreateWithFlags(&done[p], cudaEventDisableTiming));
  }
  cudaEvent_t e0, e1;
  AMG_CUDA(cudaEventCreate(&e0));
  AMG_CUDA(cudaEventCreate(&e1));
  // the NVTX range holds the graph launches only (not the tuning and capture of a
  // first call), so a profiler filtered on it sees the solve alone
  nvtxRangePushA("amg_solve_batched");
  AMG_CUDA(cudaEventRecord(e0, h0->stream));
  for (int p = 0; p < np; ++p) {
    cudaStream_t sp = hs[p]->stream;
    if (sp != h0->stream) AMG_CUDA(cudaStreamWaitEvent(sp, e0, 0));
    AMG_CUDA(cudaGraphLaunch(execs[p], sp));
    AMG_CUDA(cudaEventRecord(done[p], sp));
  }
  for (int p = 0; p < np; ++p)
    if (hs[p]->stream != h0->stream) AMG_CUDA(cudaStreamWaitEvent(h0->stream, done[p], 0));
  AMG_CUDA(cudaEventRecord(e1, h0->stream));
  nvtxRangePop();
  AMG_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ms_out) *ms_out = ms;
  // statistics: iterations and true residuals per problem (max over right-hand sides)
  int rc = AMG_OK;
  for (int p = 0; p < np; ++p) {
    amg_handle* h = hs[p];
    int it = 0;
    AMG_CUDA(cudaMemcpy(&it, h->bit.p, sizeof(int), cudaMemcpyDeviceToHost));
    // true residuals r = b - A x per right-hand side (slots reused after the solve)
    const int64_t nel = 4 * (int64_t)K * h->L[0]->n;
    apply_m64(h, h->mx, h->mq);
    k_sub_m<<<gridk(nel), 256, 0, h->stream>>>(h->mb, h->mq, h->mr, nel);
    AMG_LAUNCH_CHECK();
    dots_m(h, M_RZN, h->mr, h->mr, h->mb, h->mb);
    std::vector<double> sc((size_t)M_NS * K);
    AMG_CUDA(cudaMemcpyAsync(sc.data(), h->bscal.p, sc.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream));
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    std::vector<double> rr(K), bb(K);
    for (int r = 0; r < K; ++r) {
      rr[r] = sc[M_RZN * K + r];
      bb[r] = sc[M_ZRO * K + r];
    }
    double worst = 0.0;
    bool conv = true;
    for (int r = 0; r < nrhs; ++r) {
      const double rel = bb[r] > 0 ? std::sqrt(rr[r] / bb[r]) : 0.0;
      worst = std::max(worst, rel);
      if (sc[M_ACT * K + r] != 0.0) conv = false;
    }
    if (!conv) rc = AMG_NOT_CONVERGED;
    h->launches = l0[p] + per_iter[p] * it;
    if (stats) {
      amg_stats& st = stats[p];
      std::memset(&st, 0, sizeof(st));
      st.iterations = it;
      st.converged = conv;
      st.n_levels = (int)h->L.size();
      st.true_rel_residual = worst;
      st.rel_residual = worst;
      st.solve_ms = ms;
      st.setup_ms = h->setup_ms;
      st.kernel_launches = per_iter[p] * it;
      for (int l = 0; l < AMG_MAX_LEVELS && l < (int)h->L.size(); ++l) {
        st.level_nodes[l] = h->L[l]->n;
        st.level_nnzb[l] = h->L[l]->nnzb;
        st.level_colours[l] = h->L[l]->ncolours;
      }
    }
  }
  return rc;
}

}  // namespace amgp2
