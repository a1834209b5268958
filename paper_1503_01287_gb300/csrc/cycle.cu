// The AMG cycle of Algorithm 1 on the GPU: 3x3-block row kernels (operator
// application, residual, multicolour block Gauss-Seidel, damped block Jacobi),
// transfers P / R = P^T, the dense coarsest solve, and the saddle-point
// segregated Gauss-Seidel sweep of Eq. (uzsm).
//
// Every operation has one __device__ body.  The cycle is written once against
// an emitter that either launches one kernel per operation or records it as a
// phase.  The recorded phases of the small coarse levels run in one launch of a
// thread-block cluster, separated by cluster barriers, so both paths perform the
// same operations in the same order.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <cstring>
#include <vector>

#include "amg_internal.cuh"
#include "vec.cuh"

namespace cg = cooperative_groups;

namespace amgp2 {

namespace {

enum RowMode { kApply = 0, kResid = 1, kGS = 2, kJacobi = 3 };

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Operator values stored as V (T itself, or BF16 for the coarse levels of
// AMG_FP32_BF16), returned in the arithmetic type T.
template <typename T, typename V>
__device__ __forceinline__ T ldcs_v(const V* p) {
  if constexpr (std::is_same<T, V>::value) return __ldcs(p);
  else return __bfloat162float(__ldcs(p));
}
template <typename T, typename V>
__device__ __forceinline__ T ldg_v(const V* p) {
  if constexpr (std::is_same<T, V>::value) return __ldg(p);
  else return __bfloat162float(__ldg(p));
}

// Vector loads.  COH = false: read-only path (vectors written by earlier
// kernels).  COH = true: through L2 only, for vectors written earlier in the
// same cluster launch by other CTAs.
template <bool COH>
struct VL;
template <>
struct VL<false> {
  template <typename T>
  __device__ static void node(const T* p, int j, T& a, T& b, T& c) { ld3(p, j, a, b, c); }
  template <typename T>
  __device__ static T one(const T* p) { return __ldg(p); }
};
template <>
struct VL<true> {
  __device__ static void node(const float* p, int j, float& a, float& b, float& c) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(p) + j);
    a = v.x; b = v.y; c = v.z;
  }
  __device__ static void node(const double* p, int j, double& a, double& b, double& c) {
    double w;
    asm volatile("ld.global.cg.v4.f64 {%0, %1, %2, %3}, [%4];"
                 : "=d"(a), "=d"(b), "=d"(c), "=d"(w)
                 : "l"(p + 4 * (size_t)j)
                 : "memory");
  }
  template <typename T>
  __device__ static T one(const T* p) { return __ldcg(p); }
};

// ------------------------------------------------------------------- bodies

// One group of G lanes per block row, 32/G rows per warp, warp-uniform loop.
// Each lane walks the row's blocks with stride G; block values come from the 9
// planes (consecutive lanes read consecutive addresses of each plane), x_j is
// one vector load of the padded node; the three partial sums are reduced with
// shuffles inside the group.
//   kApply : y_i = (A x)_i
//   kResid : y_i = b_i - (A x)_i
//   kGS    : x_i += D_i^{-1} (b_i - (A x)_i)
//   kJacobi: y_i = x_i + omega D_i^{-1} (b_i - (A x)_i)
// Stored row g holds the blocks rowptr[g]..rowptr[g+1] of node i = rows[g]
// (i = g when rows is null).  D^{-1} is stored as 3 padded rows per node.
template <typename T, int G, int MODE, bool COH, typename V = T>
__device__ __forceinline__ void rows_body(int nrows, const int* __restrict__ rows,
                                          const int* __restrict__ rowptr,
                                          const int* __restrict__ col,
                                          const V* __restrict__ val, int64_t nnzb, const T* x,
                                          const T* b, T* y, const T* __restrict__ dinv,
                                          T omega, const double* __restrict__ wt, int warp,
                                          int nwarps) {
  constexpr int RPW = 32 / G;
  // relaxation: omega (Jacobi damping, 1 for Gauss-Seidel) times the level's
  // learned multiplier (1 for the plain method)
  if (MODE == kGS || MODE == kJacobi) omega = wt ? (T)((double)omega * wt[0]) : omega;
  const int lane = threadIdx.x & 31;
  const int sub = lane / G, gl = lane & (G - 1);
  for (int base = warp * RPW; base < nrows; base += nwarps * RPW) {
    const int g = base + sub;
    const bool active = g < nrows;
    int i = 0;
    T s0 = T(0), s1 = T(0), s2 = T(0);
    // operands of the row update that depend only on the row: loaded before the
    // row's blocks so that they are not on the critical path
    T b0 = T(0), b1 = T(0), b2 = T(0), xi0 = T(0), xi1 = T(0), xi2 = T(0);
    if (active) {
      i = rows ? ldg(rows + g) : g;
      if (MODE != kApply && gl == 0) {
        VL<COH>::node(b, i, b0, b1, b2);
        if (MODE != kResid) VL<COH>::node(x, i, xi0, xi1, xi2);
      }
      const int a = ldg(rowptr + g), e = ldg(rowptr + g + 1);
      // U blocks per lane per step: all column indices of the step are loaded
      // before the gathers that depend on them
      // FP64 keeps fewer blocks in flight per lane (register budget)
      // (one block per step inside the cluster and persistent kernels, whose one
      // body holds every row variant within the 128 registers of a 512-thread CTA)
      constexpr int U = COH ? 1
                            : (sizeof(T) == 8 ? (G >= 16 ? 1 : 2)
                                              : (G >= 32 ? 3 : (G >= 16 ? 2 : 4)));
      for (int k0 = a + gl; k0 < e; k0 += U * G) {
        // the matrix is streamed once per pass: evict-first loads keep the
        // gathered vector resident in L2; values do not wait for the columns
        int j[U];
        T v[U][9];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int k = k0 + u * G;
          if (k < e) {
            j[u] = __ldcs(col + k);
#pragma unroll
            for (int q = 0; q < 9; ++q) v[u][q] = ldcs_v<T>(val + q * nnzb + k);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (k0 + u * G >= e) continue;
          T x0, x1, x2;
          VL<COH>::node(x, j[u], x0, x1, x2);
          s0 = fma(v[u][0], x0, s0);
          s0 = fma(v[u][1], x1, s0);
          s0 = fma(v[u][2], x2, s0);
          s1 = fma(v[u][3], x0, s1);
          s1 = fma(v[u][4], x1, s1);
          s1 = fma(v[u][5], x2, s1);
          s2 = fma(v[u][6], x0, s2);
          s2 = fma(v[u][7], x1, s2);
          s2 = fma(v[u][8], x2, s2);
        }
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (!active || gl != 0) continue;
    if (MODE == kApply) {
      st3(y, i, s0, s1, s2);
      continue;
    }
    const T r0 = b0 - s0, r1 = b1 - s1, r2 = b2 - s2;
    if (MODE == kResid) {
      st3(y, i, r0, r1, r2);
      continue;
    }
    const T* d = dinv + 12 * (int64_t)i;
    T d0, d1, d2;
    ld3(d, 0, d0, d1, d2);
    const T c0 = d0 * r0 + d1 * r1 + d2 * r2;
    ld3(d, 1, d0, d1, d2);
    const T c1 = d0 * r0 + d1 * r1 + d2 * r2;
    ld3(d, 2, d0, d1, d2);
    const T c2 = d0 * r0 + d1 * r1 + d2 * r2;
    st3(y, i, xi0 + omega * c0, xi1 + omega * c1, xi2 + omega * c2);
  }
}

// R = P^T gather: bc_I = sum_t w_t r_{i_t} (3 components, same weight)
template <typename T, bool COH>
__device__ __forceinline__ void restrict_body(int nc, const int* __restrict__ rrow,
                                              const int* __restrict__ rcol,
                                              const T* __restrict__ rval, const T* r, T* bc,
                                              int tid, int nthr) {
  for (int I = tid; I < nc; I += nthr) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int t = rrow[I]; t < rrow[I + 1]; ++t) {
      const int i = rcol[t];
      const T w = rval[t];
      T r0, r1, r2;
      VL<COH>::node(r, i, r0, r1, r2);
      s0 = fma(w, r0, s0);
      s1 = fma(w, r1, s1);
      s2 = fma(w, r2, s2);
    }
    st3(bc, I, s0, s1, s2);
  }
}

// x_i += sum_q P_iq xc_q
template <typename T, bool COH>
__device__ __forceinline__ void prolong_body(int n, const int* __restrict__ prow,
                                             const int* __restrict__ pcol,
                                             const T* __restrict__ pval, const T* xc, T* x,
                                             const double* __restrict__ wt, int tid, int nthr) {
  // coarse-grid correction x += w_c P x_c (w_c = 1 for the plain method)
  const T wc = wt ? (T)wt[1] : T(1);
  for (int i = tid; i < n; i += nthr) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int q = prow[i]; q < prow[i + 1]; ++q) {
      const int J = pcol[q];
      const T w = pval[q];
      T c0, c1, c2;
      VL<COH>::node(xc, J, c0, c1, c2);
      s0 = fma(w, c0, s0);
      s1 = fma(w, c1, s1);
      s2 = fma(w, c2, s2);
    }
    T x0, x1, x2;
    VL<COH>::node(x, i, x0, x1, x2);
    st3(x, i, x0 + wc * s0, x1 + wc * s1, x2 + wc * s2);
  }
}

// scalar versions for the pressure (H^T restriction, H prolongation)
template <typename T, bool COH>
__device__ __forceinline__ void restrict1_body(int nc, const int* __restrict__ rrow,
                                               const int* __restrict__ rcol,
                                               const T* __restrict__ rval, const T* r, T* bc,
                                               int tid, int nthr) {
  for (int I = tid; I < nc; I += nthr) {
    T s = T(0);
    for (int t = rrow[I]; t < rrow[I + 1]; ++t) s = fma(rval[t], VL<COH>::one(r + rcol[t]), s);
    bc[I] = s;
  }
}

template <typename T, bool COH>
__device__ __forceinline__ void prolong1_body(int n, const int* __restrict__ prow,
                                              const int* __restrict__ pcol,
                                              const T* __restrict__ pval, const T* xc, T* x,
                                              const double* __restrict__ wt, int tid, int nthr) {
  const T wc = wt ? (T)wt[1] : T(1);
  for (int i = tid; i < n; i += nthr) {
    T s = T(0);
    for (int q = prow[i]; q < prow[i + 1]; ++q) s = fma(pval[q], VL<COH>::one(xc + pcol[q]), s);
    x[i] = VL<COH>::one(x + i) + wc * s;
  }
}

// x = X b with the FP64 generalised inverse of the coarsest matrix (warp per
// row).  X is indexed in the unpadded order (3 per node, then pressure).
__device__ __forceinline__ int pad_index(int j, int n3) {
  return j < n3 ? 4 * (j / 3) + j % 3 : j + n3 / 3;
}

template <typename T, bool COH>
__device__ __forceinline__ void coarse_body(int m, int n3, const double* __restrict__ X,
                                            const T* b, T* x, int warp, int nwarps) {
  const int lane = threadIdx.x & 31;
  for (int i = warp; i < m; i += nwarps) {
    double s = 0.0;
    for (int j = lane; j < m; j += 32)
      s = fma(X[(int64_t)i * m + j], (double)VL<COH>::one(b + pad_index(j, n3)), s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[pad_index(i, n3)] = (T)s;
  }
}

template <typename T, bool COH>
__device__ __forceinline__ void copy_body(const T* a, T* b, int64_t n, int tid, int nthr) {
  for (int64_t k = tid; k < n; k += nthr) b[k] = VL<COH>::one(a + k);
}

template <typename T>
__device__ __forceinline__ void zero_body(T* a, int64_t n, int tid, int nthr) {
  for (int64_t k = tid; k < n; k += nthr) a[k] = T(0);
}

// y_i += sign * sum_k B_ki^T p_k (rows of B^T are velocity nodes)
template <typename T, bool COH>
__device__ __forceinline__ void bt_add_body(int n, const int* __restrict__ row,
                                            const int* __restrict__ col,
                                            const T* __restrict__ val, int64_t nnz, const T* p,
                                            T sign, T* y, int tid, int nthr) {
  for (int i = tid; i < n; i += nthr) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int q = row[i]; q < row[i + 1]; ++q) {
      const T pk = VL<COH>::one(p + col[q]);
      s0 = fma(val[q], pk, s0);
      s1 = fma(val[nnz + q], pk, s1);
      s2 = fma(val[2 * nnz + q], pk, s2);
    }
    T y0, y1, y2;
    VL<COH>::node(y, i, y0, y1, y2);
    st3(y, i, y0 + sign * s0, y1 + sign * s1, y2 + sign * s2);
  }
}

// MODE 0: yp = B u - C p;  MODE 1: yp = g - B u + C p (residual);
// MODE 2: yp = p + omega (B u - C p - g) / S_D (sGS pressure step);
// MODE 3: yp = B u - g (Braess-Sarazin: g holds the pressure residual)
// The pressure rows: kProwLanes consecutive lanes share a row (its B entries and then
// its C entries taken in strides of kProwLanes, the lane sums combined by shuffles),
// so a row's dependent gather chain is about 1/kProwLanes of its length.
constexpr int kProwLanes = 8;
template <typename T, int MODE, bool COH>
__device__ __forceinline__ void prows_body(int np, const int* __restrict__ brow,
                                           const int* __restrict__ bcol,
                                           const T* __restrict__ bval, int64_t bnnz,
                                           const int* __restrict__ crow,
                                           const int* __restrict__ ccol,
                                           const T* __restrict__ cval, const T* u, const T* p,
                                           const T* g, T* yp, const T* __restrict__ sd, T omega,
                                           const double* __restrict__ wt, int tid, int nthr) {
  if (MODE == 2 && wt) omega = (T)((double)omega * wt[2]);
  constexpr int L = kProwLanes;
  const int gl = tid & (L - 1);
  const unsigned gmask = ((1u << L) - 1u) << (threadIdx.x & 31 & ~(L - 1));
  for (int k = tid / L; k < np; k += nthr / L) {
    T s = T(0);
    for (int q = brow[k] + gl; q < brow[k + 1]; q += L) {
      const int j = bcol[q];
      T u0, u1, u2;
      VL<COH>::node(u, j, u0, u1, u2);
      s = fma(bval[q], u0, s);
      s = fma(bval[bnnz + q], u1, s);
      s = fma(bval[2 * bnnz + q], u2, s);
    }
    T cp = T(0);
    if (MODE != 3)
      for (int q = crow[k] + gl; q < crow[k + 1]; q += L)
        cp = fma(cval[q], VL<COH>::one(p + ccol[q]), cp);
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
      s += __shfl_xor_sync(gmask, s, o);
      cp += __shfl_xor_sync(gmask, cp, o);
    }
    if (gl != 0) continue;
    if (MODE == 3) {               // Braess-Sarazin right-hand side B w - r_p
      yp[k] = s - VL<COH>::one(g + k);
    } else if (MODE == 0) {
      yp[k] = s - cp;
    } else if (MODE == 1) {
      yp[k] = VL<COH>::one(g + k) - s + cp;
    } else {
      const T d = sd[k];
      const T r = s - cp - VL<COH>::one(g + k);
      yp[k] = VL<COH>::one(p + k) + (d != T(0) ? omega * r / d : T(0));
    }
  }
}

// Scalar CSR rows of an S-hierarchy matrix (Braess-Sarazin smoother):
// MODE 0: y = b - S x;  MODE 1: y = x + omega d (b - S x) (damped Jacobi, d = 1/S_kk)
template <typename T, int MODE, bool COH>
__device__ __forceinline__ void srows_body(int n, const int* __restrict__ rowptr,
                                           const int* __restrict__ col,
                                           const T* __restrict__ val, const T* x, const T* b,
                                           const T* __restrict__ d, T omega, T* y, int tid,
                                           int nthr) {
  for (int k = tid; k < n; k += nthr) {
    T acc = T(0);
    for (int q = rowptr[k]; q < rowptr[k + 1]; ++q)
      acc = fma(val[q], VL<COH>::one(x + col[q]), acc);
    const T r = VL<COH>::one(b + k) - acc;
    y[k] = MODE == 0 ? r : VL<COH>::one(x + k) + omega * d[k] * r;
  }
}

// Element-wise: MODE 0: y = omega d x;  MODE 1: y += x;  MODE 2: y += x - d b
template <typename T, int MODE, bool COH>
__device__ __forceinline__ void vec_body(int64_t n, const T* __restrict__ d, const T* x,
                                         const T* b, T omega, T* y, int tid, int nthr) {
  for (int64_t k = tid; k < n; k += nthr) {
    const T xv = VL<COH>::one(x + k);
    if (MODE == 0) y[k] = omega * d[k] * xv;
    else if (MODE == 1) y[k] = VL<COH>::one(y + k) + xv;
    else y[k] = VL<COH>::one(y + k) + xv - d[k] * VL<COH>::one(b + k);
  }
}

// Vanka patch corrections of one colour (Eq. (locpatchsm)), one CTA of 256 threads
// per patch k: every warp holds r_k in registers (unknown j = lane + 32 q of the
// patch), the 8 warps share the rows of y = A_k^{-1} r_u (two rows in flight per
// warp, warp-reduced, into shared memory), then dp = (B_k y - r_p) / s_k (0 when
// s_k = 0), du = y - w_k dp, x_patch += omega du, p_k += omega dp.  Patches of one
// colour share no unknown.
constexpr int kVankaRegs = 16;   // 16 x 32 = 512 unknowns a patch

template <typename T>
__global__ void __launch_bounds__(256) k_vanka(int npatch, const int* __restrict__ patches,
                                               const int* __restrict__ brow,
                                               const int* __restrict__ bcol,
                                               const T* __restrict__ bval, int64_t bnnz,
                                               const long long* __restrict__ off,
                                               const T* __restrict__ ainv,
                                               const T* __restrict__ w,
                                               const T* __restrict__ sk, const T* r, T* x,
                                               int n4, T omega) {
  __shared__ T ysh[32 * kVankaRegs];
  __shared__ T red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < npatch; t += gridDim.x) {
    const int k = patches[t];
    const int q0 = brow[k], m = 3 * (brow[k + 1] - q0);
    T rj[kVankaRegs];
#pragma unroll
    for (int q = 0; q < kVankaRegs; ++q) {
      const int j = lane + 32 * q;
      rj[q] = j < m ? r[4 * bcol[q0 + j / 3] + j % 3] : T(0);
    }
    const T* Ai = ainv + off[k];
    for (int i0 = 2 * warp; i0 < m; i0 += 16) {
      const int i1 = i0 + 1;
      const T* row0 = Ai + (int64_t)i0 * m;
      const T* row1 = Ai + (int64_t)min(i1, m - 1) * m;
      T p0 = T(0), p1 = T(0);
#pragma unroll
      for (int q = 0; q < kVankaRegs; ++q) {
        const int j = lane + 32 * q;
        if (j < m) {
          p0 = fma(row0[j], rj[q], p0);
          p1 = fma(row1[j], rj[q], p1);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        p0 += __shfl_xor_sync(0xffffffffu, p0, o);
        p1 += __shfl_xor_sync(0xffffffffu, p1, o);
      }
      if (lane == 0) {
        ysh[i0] = p0;
        if (i1 < m) ysh[i1] = p1;
      }
    }
    __syncthreads();
    T bd = T(0);
    for (int j = threadIdx.x; j < m; j += blockDim.x)
      bd = fma(bval[(j % 3) * bnnz + q0 + j / 3], ysh[j], bd);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bd += __shfl_xor_sync(0xffffffffu, bd, o);
    if (lane == 0) red[warp] = bd;
    __syncthreads();
    T tot = T(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) tot += red[q];
    const T s = sk[k];
    const T dp = s != T(0) ? (tot - r[n4 + k]) / s : T(0);
    const T* wk = w + 3 * (int64_t)q0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const int dof = 4 * bcol[q0 + j / 3] + j % 3;
      x[dof] += omega * (ysh[j] - wk[j] * dp);
    }
    if (threadIdx.x == 0) x[n4 + k] += omega * dp;
    __syncthreads();
  }
}

// ------------------------------------------------------------------- phases

enum PhaseType : int {
  PH_ZERO = 0, PH_COPY, PH_ROWS, PH_RESTRICT, PH_PROLONG, PH_RESTRICT1, PH_PROLONG1,
  PH_COARSE, PH_BT_ADD, PH_PROWS, PH_SROWS, PH_VEC, PH_VANKA
};

// One operation of the cycle with its operands (a plain record, copied to the
// device for the cluster launch or passed by value to a single launch).
struct Phase {
  int type, mode, G, n;   // n: rows / nodes / entries
  const int* rows;
  const int* rowptr;
  const int* col;
  const void* val;
  int64_t nnz;
  const void* dinv;
  const void* x;
  const void* b;
  void* y;
  const int* crow;
  const int* ccol;
  const void* cval;
  const void* sd;
  const void* p;          // pressure iterate (PH_PROWS)
  const double* X;
  int m, n3;
  double omega;
  const double* wt;       // the level's learned weights (null: plain method)
  int vbf;                // PH_ROWS: values stored as BF16 (FP32 arithmetic)
  int sctas;              // PH_ROWS, Gauss-Seidel: CTAs per SM of the streaming colour
                          // kernel (0: one group of lanes per row, k_gs_pdl)
  int xnc;                // PH_ROWS, Gauss-Seidel (k_gs_pdl): x through the L1 path
  int tma;                // PH_ROWS, Gauss-Seidel, FP32: the TMA-staged colour kernel
  int* err;               // the handle's error word (bounded waits that gave up)
  const long long* off;   // PH_VANKA: offsets of the patch inverses
};

template <typename T, bool COH, typename V = T>
__device__ void dispatch_rows_v(const Phase& P, int warp, int nwarps) {
  const V* val = (const V*)P.val;
  const T* x = (const T*)P.x;
  const T* b = (const T*)P.b;
  T* y = (T*)P.y;
  const T* d = (const T*)P.dinv;
  const T om = (T)P.omega;
#define AMG_ROWS_MODE(GG, MM)                                                                   \
  rows_body<T, GG, MM, COH, V>(P.n, P.rows, P.rowptr, P.col, val, P.nnz, x, b, y, d, om, P.wt, \
                               warp, nwarps)
#define AMG_ROWS_G(GG)                              \
  switch (P.mode) {                                 \
    case kApply: AMG_ROWS_MODE(GG, kApply); break;  \
    case kResid: AMG_ROWS_MODE(GG, kResid); break;  \
    case kGS: AMG_ROWS_MODE(GG, kGS); break;        \
    default: AMG_ROWS_MODE(GG, kJacobi); break;     \
  }
  switch (P.G) {
    case 4: AMG_ROWS_G(4) break;
    case 8: AMG_ROWS_G(8) break;
    case 16: AMG_ROWS_G(16) break;
    default: AMG_ROWS_G(32) break;
  }
#undef AMG_ROWS_G
#undef AMG_ROWS_MODE
}

template <typename T, bool COH>
__device__ void dispatch_rows(const Phase& P, int warp, int nwarps) {
  if constexpr (std::is_same<T, float>::value) {
    if (P.vbf) {
      dispatch_rows_v<float, COH, __nv_bfloat16>(P, warp, nwarps);
      return;
    }
  }
  dispatch_rows_v<T, COH, T>(P, warp, nwarps);
}

template <typename T, bool COH>
__device__ __forceinline__ void exec_phase(const Phase& P, int tid, int nthr) {
  const int warp = tid >> 5, nwarps = nthr >> 5;
  switch (P.type) {
    case PH_ZERO: zero_body<T>((T*)P.y, P.n, tid, nthr); break;
    case PH_COPY: copy_body<T, COH>((const T*)P.x, (T*)P.y, P.n, tid, nthr); break;
    case PH_ROWS: dispatch_rows<T, COH>(P, warp, nwarps); break;
    case PH_RESTRICT:
      restrict_body<T, COH>(P.n, P.rowptr, P.col, (const T*)P.val, (const T*)P.x, (T*)P.y, tid,
                            nthr);
      break;
    case PH_PROLONG:
      prolong_body<T, COH>(P.n, P.rowptr, P.col, (const T*)P.val, (const T*)P.x, (T*)P.y, P.wt,
                           tid, nthr);
      break;
    case PH_RESTRICT1:
      restrict1_body<T, COH>(P.n, P.rowptr, P.col, (const T*)P.val, (const T*)P.x, (T*)P.y, tid,
                             nthr);
      break;
    case PH_PROLONG1:
      prolong1_body<T, COH>(P.n, P.rowptr, P.col, (const T*)P.val, (const T*)P.x, (T*)P.y, P.wt,
                            tid, nthr);
      break;
    case PH_COARSE:
      coarse_body<T, COH>(P.m, P.n3, P.X, (const T*)P.b, (T*)P.y, warp, nwarps);
      break;
    case PH_BT_ADD:
      bt_add_body<T, COH>(P.n, P.rowptr, P.col, (const T*)P.val, P.nnz, (const T*)P.x,
                          (T)P.omega, (T*)P.y, tid, nthr);
      break;
    case PH_PROWS: {
      const T* u = (const T*)P.x;
      const T* p = (const T*)P.p;
      const T om = (T)P.omega;
#define AMG_PROWS(MM)                                                                        \
  prows_body<T, MM, COH>(P.n, P.rowptr, P.col, (const T*)P.val, P.nnz, P.crow, P.ccol,      \
                         (const T*)P.cval, u, p, (const T*)P.b, (T*)P.y, (const T*)P.sd, om, \
                         P.wt, tid, nthr)
      if (P.mode == 0) AMG_PROWS(0);
      else if (P.mode == 1) AMG_PROWS(1);
      else if (P.mode == 2) AMG_PROWS(2);
      else AMG_PROWS(3);
#undef AMG_PROWS
      break;
    }
    case PH_SROWS:
      if (P.mode == 0)
        srows_body<T, 0, COH>(P.n, P.rowptr, P.col, (const T*)P.val, (const T*)P.x,
                              (const T*)P.b, (const T*)P.dinv, (T)P.omega, (T*)P.y, tid, nthr);
      else
        srows_body<T, 1, COH>(P.n, P.rowptr, P.col, (const T*)P.val, (const T*)P.x,
                              (const T*)P.b, (const T*)P.dinv, (T)P.omega, (T*)P.y, tid, nthr);
      break;
    case PH_VEC:
      if (P.mode == 0)
        vec_body<T, 0, COH>(P.n, (const T*)P.dinv, (const T*)P.x, (const T*)P.b, (T)P.omega,
                            (T*)P.y, tid, nthr);
      else if (P.mode == 1)
        vec_body<T, 1, COH>(P.n, (const T*)P.dinv, (const T*)P.x, (const T*)P.b, (T)P.omega,
                            (T*)P.y, tid, nthr);
      else
        vec_body<T, 2, COH>(P.n, (const T*)P.dinv, (const T*)P.x, (const T*)P.b, (T)P.omega,
                            (T*)P.y, tid, nthr);
      break;
    default:
      break;
  }
}

// Multicolour Gauss-Seidel for one colour, launched with programmatic dependent
// launch: the operands that setup wrote and no cycle kernel writes (row ids,
// block columns and values, D_i^{-1}) are loaded before griddepcontrol.wait, so
// this prologue overlaps the previous kernel; b_i, the relaxation multiplier and
// the x gathers come after the wait, since only then are the previous kernel's
// writes guaranteed visible (the first colour of a sweep follows the
// restriction that writes b).
// One group of G lanes per stored row; each lane prefetches up to U blocks.
// XNC: x is gathered through the read-only (L1-cached) path instead of L2 only.
// Within one colour launch nothing that is gathered is written (rows of one
// colour are not neighbours; a row reads its own x_i before writing it), and the
// previous kernels' writes are visible after griddepcontrol.wait.
template <typename T, int G, int U, typename V = T, bool XNC = false>
__global__ void __launch_bounds__(256) k_gs_pdl(int nrows, const int* __restrict__ rows,
                                                const int* __restrict__ rowptr,
                                                const int* __restrict__ col,
                                                const V* __restrict__ val, int64_t nnzb, T* x,
                                                const T* __restrict__ b,
                                                const T* __restrict__ dinv,
                                                const double* __restrict__ wt) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int gl = threadIdx.x & (G - 1);
  const bool active = g < nrows;
  int i = 0, a = 0, e = 0;
  int j[U];
  T v[U][9];
  T b0 = T(0), b1 = T(0), b2 = T(0);
  T d[9];
#pragma unroll
  for (int u = 0; u < U; ++u) j[u] = -1;
  if (active) {
    i = ldg(rows + g);
    a = ldg(rowptr + g);
    e = ldg(rowptr + g + 1);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = a + gl + u * G;
      if (k < e) {
        j[u] = __ldcs(col + k);
#pragma unroll
        for (int q = 0; q < 9; ++q) v[u][q] = ldcs_v<T>(val + q * nnzb + k);
      }
    }
    if (gl == 0) {
      const T* dp = dinv + 12 * (int64_t)i;
      ld3(dp, 0, d[0], d[1], d[2]);
      ld3(dp, 1, d[3], d[4], d[5]);
      ld3(dp, 2, d[6], d[7], d[8]);
    }
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const T om = wt ? (T)wt[0] : T(1);   // learned relaxation multiplier (1: plain)
  T s0 = T(0), s1 = T(0), s2 = T(0);
  T xi0 = T(0), xi1 = T(0), xi2 = T(0);
  if (active) {
    if (gl == 0) {
      ld3(b, i, b0, b1, b2);
      VL<!XNC>::node(x, i, xi0, xi1, xi2);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j[u] < 0) continue;
      T x0, x1, x2;
      VL<!XNC>::node(x, j[u], x0, x1, x2);
      s0 = fma(v[u][0], x0, s0); s0 = fma(v[u][1], x1, s0); s0 = fma(v[u][2], x2, s0);
      s1 = fma(v[u][3], x0, s1); s1 = fma(v[u][4], x1, s1); s1 = fma(v[u][5], x2, s1);
      s2 = fma(v[u][6], x0, s2); s2 = fma(v[u][7], x1, s2); s2 = fma(v[u][8], x2, s2);
    }
    // blocks beyond the prefetched U per lane
    for (int k = a + gl + U * G; k < e; k += G) {
      const int jj = ldg(col + k);
      T x0, x1, x2;
      VL<!XNC>::node(x, jj, x0, x1, x2);
      const V* vv = val + k;
      s0 = fma(ldg_v<T>(vv), x0, s0);
      s0 = fma(ldg_v<T>(vv + nnzb), x1, s0);
      s0 = fma(ldg_v<T>(vv + 2 * nnzb), x2, s0);
      s1 = fma(ldg_v<T>(vv + 3 * nnzb), x0, s1);
      s1 = fma(ldg_v<T>(vv + 4 * nnzb), x1, s1);
      s1 = fma(ldg_v<T>(vv + 5 * nnzb), x2, s1);
      s2 = fma(ldg_v<T>(vv + 6 * nnzb), x0, s2);
      s2 = fma(ldg_v<T>(vv + 7 * nnzb), x1, s2);
      s2 = fma(ldg_v<T>(vv + 8 * nnzb), x2, s2);
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (!active || gl != 0) return;
  const T r0 = b0 - s0, r1 = b1 - s1, r2 = b2 - s2;
  st3(x, i, xi0 + om * (d[0] * r0 + d[1] * r1 + d[2] * r2),
      xi1 + om * (d[3] * r0 + d[4] * r1 + d[5] * r2), xi2 + om * (d[6] * r0 + d[7] * r1 + d[8] * r2));
}

template <typename T, int G, typename V, bool XNC>
void launch_gs_pdl_x(const Phase& P, cudaStream_t s) {
  constexpr int U = (sizeof(T) == 8) ? (G >= 16 ? 2 : 3) : (G >= 16 ? 3 : 4);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(((int64_t)P.n * G + 255) / 256));
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  AMG_CUDA(cudaLaunchKernelEx(&cfg, k_gs_pdl<T, G, U, V, XNC>, P.n, P.rows, P.rowptr, P.col,
                              (const V*)P.val, P.nnz, (T*)P.y, (const T*)P.b,
                              (const T*)P.dinv, P.wt));
}

template <typename T, int G, typename V = T>
void launch_gs_pdl(const Phase& P, cudaStream_t s) {
  if (P.xnc) launch_gs_pdl_x<T, G, V, true>(P, s);
  else launch_gs_pdl_x<T, G, V, false>(P, s);
}

// Multicolour Gauss-Seidel sweep of one small level as ONE launch: a single CTA,
// or a thread-block cluster.  Every CTA keeps in shared memory the level's whole
// iterate x and right-hand side b (4 values a node) and the row ids and block
// offsets of the colour-ordered rows, so a row update reads global memory only
// for its block columns and values and D_i^{-1}, at addresses known from shared
// memory; each group of G lanes loads its next row's operands before it waits
// for the colour it must follow.  The colours run in sweep order.
//   single CTA: the new value of a row goes to shared memory; __syncthreads
//   between the colours.
//   cluster: the new value of a row goes to the x copy of every CTA of the
//   cluster by st.async (distributed shared memory), which counts its bytes on
//   the receiving CTA's mbarrier of that step of the sweep (one mbarrier a
//   colour, each completing one phase); a warp starts a colour once every row
//   of the previous colour has arrived.  That also orders the reads: a row's
//   value is sent after its owner has read every x_j of the row, so a value of
//   colour q + 1 can reach a CTA only after all reads of colour q have been
//   done.  No cluster barrier or memory fence is needed between the colours.
// Rows of one colour share no block, so the updates of a colour never read a
// value written in the same colour (the row's own x_i is read before its own
// update).  Every mbarrier wait is bounded: after kMbarSpins polls the CTA sets
// *err and stops waiting.
constexpr int kGsClThreads = 512;
constexpr int kGsClMaxColours = 127;
constexpr int kGsClSmemBytes = 200 * 1024;
constexpr unsigned kMbarSpins = 1u << 18;

struct GsColours {
  int ptr[kGsClMaxColours + 1];   // stored rows of colour c: ptr[c] .. ptr[c+1]
};

// shared memory of the one-launch sweep: an mbarrier a colour (1 KB), x and b
// (4 n values each), the row id and the first block of every stored row
constexpr int kGsClBarBytes = 8 * (kGsClMaxColours + 1);
template <typename T>
constexpr int64_t gs_cl_smem(int64_t n) {
  return kGsClBarBytes + 8 * n * (int64_t)sizeof(T) + 4 * n + 4 * (n + 1);
}

__device__ __forceinline__ void lds3(const float* p, int j, float& a, float& b, float& c) {
  const float4 v = reinterpret_cast<const float4*>(p)[j];
  a = v.x; b = v.y; c = v.z;
}
__device__ __forceinline__ void lds3(const double* p, int j, double& a, double& b, double& c) {
  const double2 v = reinterpret_cast<const double2*>(p)[2 * j];
  a = v.x; b = v.y;
  c = p[4 * j + 2];
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// waits for the completion of the mbarrier phase of parity `par`; false after
// kMbarSpins polls
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t par) {
  for (unsigned spins = 0; spins < kMbarSpins; ++spins) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(par)
        : "memory");
    if (done) return true;
  }
  return false;
}
// a node's new value (x, y, z, 0) into the shared memory of a cluster CTA,
// counted on that CTA's mbarrier
__device__ __forceinline__ void st_async_node(uint32_t dst, uint32_t bar, float a, float b,
                                              float c) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, "
      "[%5];" ::"r"(dst),
      "f"(a), "f"(b), "f"(c), "f"(0.f), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void st_async_node(uint32_t dst, uint32_t bar, double a, double b,
                                              double c) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(
          dst),
      "d"(a), "d"(b), "r"(bar)
      : "memory");
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(
          dst + 16),
      "d"(c), "d"(0.0), "r"(bar)
      : "memory");
}

// blocks carried per lane in each of the two operand sets (register budget of
// a 512-thread CTA: 128 a thread)
template <typename T, int G, typename V>
constexpr int gs_cl_unroll() {
  return sizeof(T) == 8 ? 1 : 2;
}

template <typename T, int G, int U, typename V, bool ONE>
__global__ void __launch_bounds__(kGsClThreads, 1)
    k_gs_cluster(int n, int ncolours, const GsColours cp, int post, int x_zero,
                 const int* __restrict__ rows, const int* __restrict__ rowptr,
                 const int* __restrict__ col, const V* __restrict__ val, int64_t nnzb, T* x,
                 const T* __restrict__ b, const T* __restrict__ dinv,
                 const double* __restrict__ wt, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char gs_smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(gs_smem);
  T* xs = reinterpret_cast<T*>(gs_smem + kGsClBarBytes);
  T* bs = xs + 4 * (int64_t)n;
  int* rows_s = reinterpret_cast<int*>(bs + 4 * (int64_t)n);
  int* rp_s = rows_s + n;
  const int cs = ONE ? 1 : (int)cg::this_cluster().num_blocks();
  const int rank = ONE ? 0 : (int)cg::this_cluster().block_rank();
  constexpr int RPW = 32 / G;
  constexpr uint32_t kNodeBytes = 4 * sizeof(T);
  const int lane = threadIdx.x & 31, sub = lane / G, gl = lane & (G - 1);
  const int warp = (rank * (int)blockDim.x + (int)threadIdx.x) >> 5;
  const int nwarps = (cs * (int)blockDim.x) >> 5;
  const int stride = nwarps * RPW;
  const T om = wt ? (T)wt[0] : T(1);   // learned relaxation multiplier (1: plain)
  auto colour_of = [&](int q) { return post ? ncolours - 1 - q : q; };
  auto colour_bytes = [&](int q) {
    const int c = colour_of(q);
    return (uint32_t)(cp.ptr[c + 1] - cp.ptr[c]) * kNodeBytes;
  };
  const uint32_t bar0 = smem_addr(bars), xs0 = smem_addr(xs);

  {
    // x and b as 16-byte words (a node is one or two), several loads in flight
    const int nw = n * 4 * (int)sizeof(T) / 16;
    uint4* xw = reinterpret_cast<uint4*>(xs);
    uint4* bw = reinterpret_cast<uint4*>(bs);
    const uint4* xg = reinterpret_cast<const uint4*>(x);
    const uint4* bg = reinterpret_cast<const uint4*>(b);
#pragma unroll 4
    for (int k = threadIdx.x; k < nw; k += blockDim.x) {
      xw[k] = x_zero ? make_uint4(0u, 0u, 0u, 0u) : xg[k];
      bw[k] = __ldg(bg + k);
    }
#pragma unroll 4
    for (int k = threadIdx.x; k < n; k += blockDim.x) rows_s[k] = __ldg(rows + k);
#pragma unroll 4
    for (int k = threadIdx.x; k <= n; k += blockDim.x) rp_s[k] = __ldg(rowptr + k);
  }
  if constexpr (ONE) {
    __syncthreads();
  } else {
    // mbarrier q counts step q of the sweep: one arrival (its expect_tx) and the
    // bytes of every row of the colour
    if (threadIdx.x == 0) {
      for (int q = 0; q < ncolours; ++q) mbar_init(bar0 + 8 * q);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      for (int q = 0; q < ncolours; ++q) mbar_expect(bar0 + 8 * q, colour_bytes(q));
    }
    // every copy and mbarrier is ready before any CTA stores into another
    cg::this_cluster().sync();
  }

  // operands of a row: node, block range, the first U blocks' columns and
  // values, D_i^{-1}.  Two sets: the first rows of the next two colours are
  // loaded while the current one runs.
  struct RowOps {
    int i, a, e;
    int j[U];
    T v[U][9];
    T d[9];
  };
  auto load_row = [&](RowOps& o, int g, int end) {
    o.a = o.e = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) o.j[u] = -1;
    if (g >= end) return;
    o.i = rows_s[g];
    o.a = rp_s[g];
    o.e = rp_s[g + 1];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = o.a + gl + u * G;
      if (k < o.e) {
        o.j[u] = __ldg(col + k);
#pragma unroll
        for (int q = 0; q < 9; ++q) o.v[u][q] = ldg_v<T>(val + q * nnzb + k);
      }
    }
    if (gl == 0) {
      const T* dp = dinv + 12 * (int64_t)o.i;
      ld3(dp, 0, o.d[0], o.d[1], o.d[2]);
      ld3(dp, 1, o.d[3], o.d[4], o.d[5]);
      ld3(dp, 2, o.d[6], o.d[7], o.d[8]);
    }
  };
  auto first_row = [&](RowOps& o, int q) {
    if (q >= ncolours) return;
    const int c = colour_of(q);
    load_row(o, cp.ptr[c] + warp * RPW + sub, cp.ptr[c + 1]);
  };

  bool ok = true;
  // step q of the sweep from the operands in `o` (its first row); `o` then
  // takes the first row of step q + 2
  auto step = [&](int q, RowOps& o) {
    const int c = colour_of(q);
    const int a = cp.ptr[c], e = cp.ptr[c + 1];
    const uint32_t bar = bar0 + 8 * q;
    for (int base = a + warp * RPW; base < e; base += stride) {
      const bool active = base + sub < e;
      const int i = o.i, ka = o.a, ke = o.e;
      T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (o.j[u] < 0) continue;
        T x0, x1, x2;
        lds3(xs, o.j[u], x0, x1, x2);
        s0 = fma(o.v[u][0], x0, s0); s0 = fma(o.v[u][1], x1, s0); s0 = fma(o.v[u][2], x2, s0);
        s1 = fma(o.v[u][3], x0, s1); s1 = fma(o.v[u][4], x1, s1); s1 = fma(o.v[u][5], x2, s1);
        s2 = fma(o.v[u][6], x0, s2); s2 = fma(o.v[u][7], x1, s2); s2 = fma(o.v[u][8], x2, s2);
      }
      // blocks beyond the U carried ones
      for (int k = ka + gl + U * G; k < ke; k += G) {
        const int jj = __ldg(col + k);
        T x0, x1, x2;
        lds3(xs, jj, x0, x1, x2);
        const V* vv = val + k;
        s0 = fma(ldg_v<T>(vv), x0, s0);
        s0 = fma(ldg_v<T>(vv + nnzb), x1, s0);
        s0 = fma(ldg_v<T>(vv + 2 * nnzb), x2, s0);
        s1 = fma(ldg_v<T>(vv + 3 * nnzb), x0, s1);
        s1 = fma(ldg_v<T>(vv + 4 * nnzb), x1, s1);
        s1 = fma(ldg_v<T>(vv + 5 * nnzb), x2, s1);
        s2 = fma(ldg_v<T>(vv + 6 * nnzb), x0, s2);
        s2 = fma(ldg_v<T>(vv + 7 * nnzb), x1, s2);
        s2 = fma(ldg_v<T>(vv + 8 * nnzb), x2, s2);
      }
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      }
      T n0 = T(0), n1 = T(0), n2 = T(0);
      if (active && gl == 0) {
        T xi0, xi1, xi2, b0, b1, b2;
        lds3(xs, i, xi0, xi1, xi2);
        lds3(bs, i, b0, b1, b2);
        const T r0 = b0 - s0, r1 = b1 - s1, r2 = b2 - s2;
        n0 = xi0 + om * (o.d[0] * r0 + o.d[1] * r1 + o.d[2] * r2);
        n1 = xi1 + om * (o.d[3] * r0 + o.d[4] * r1 + o.d[5] * r2);
        n2 = xi2 + om * (o.d[6] * r0 + o.d[7] * r1 + o.d[8] * r2);
      }
      // the group's first lane holds the new value: every lane of the group
      // takes it (a cluster sends it to ranks gl, gl + G, ...)
      n0 = __shfl_sync(0xffffffffu, n0, sub * G);
      n1 = __shfl_sync(0xffffffffu, n1, sub * G);
      n2 = __shfl_sync(0xffffffffu, n2, sub * G);
      // the next row's operands in this colour
      if (base + stride < e) load_row(o, base + stride + sub, e);
      if (active) {
        if constexpr (ONE) {
          if (gl == 0) {
            xs[4 * (int64_t)i] = n0;
            xs[4 * (int64_t)i + 1] = n1;
            xs[4 * (int64_t)i + 2] = n2;
          }
        } else {
          for (int r = gl; r < cs; r += G)
            st_async_node(cluster_addr(xs0 + 4 * (uint32_t)i * (uint32_t)sizeof(T), r),
                          cluster_addr(bar, r), n0, n1, n2);
        }
      }
    }
    // the first row of step q + 2, before waiting for this colour
    first_row(o, q + 2);
    if constexpr (ONE) {
      __syncthreads();
    } else {
      // all of colour q has arrived (the one phase of mbarrier q)
      if (ok && !mbar_wait(bar, 0u)) {
        atomicOr(err, 1);
        ok = false;
      }
    }
  };
  RowOps A, B;
  first_row(A, 0);
  first_row(B, 1);
  for (int q = 0; q < ncolours; q += 2) {
    step(q, A);
    if (q + 1 < ncolours) step(q + 1, B);
  }
  // every copy now holds the swept iterate: each CTA writes its share
  for (int k = rank * (int)blockDim.x + (int)threadIdx.x; k < 4 * n; k += cs * (int)blockDim.x)
    x[k] = xs[k];
  if constexpr (!ONE) cg::this_cluster().sync();   // no CTA leaves while others may store
}

// The largest cluster of `cs` CTAs with `smem` bytes each that can be resident
// (0: cannot launch).
template <typename T, int G, typename V>
int gs_cluster_fits(int cs, int smem) {
  constexpr int U = gs_cl_unroll<T, G, V>();
  if (cs == 1) {
    auto one = k_gs_cluster<T, G, U, V, true>;
    max_dynamic_smem((const void*)one, kGsClSmemBytes);
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, one, kGsClThreads, smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return per;
  }
  auto kern = k_gs_cluster<T, G, U, V, false>;
  max_dynamic_smem((const void*)kern, kGsClSmemBytes);
  if (cs > 8 &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(kGsClThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

template <typename T, int G, typename V>
void launch_gs_cluster_g(const Level& lv, int cs, bool post, bool x_zero, const V* val, T* x,
                         const T* b, const T* dinv, int* err, cudaStream_t s) {
  constexpr int U = gs_cl_unroll<T, G, V>();
  // the shared-memory and cluster-size attributes were set by gs_cluster_fits
  // when the level's cluster size was chosen
  GsColours cp;
  for (int c = 0; c <= lv.ncolours; ++c) cp.ptr[c] = lv.colour_ptr[c];
  if (cs == 1) {
    k_gs_cluster<T, G, U, V, true><<<1, kGsClThreads, (size_t)gs_cl_smem<T>(lv.n), s>>>(
        lv.n, lv.ncolours, cp, (int)post, (int)x_zero, lv.k_rows(), lv.k_rowptr(), lv.k_col(),
        val, lv.nnzb, x, b, dinv, (const double*)lv.wt, err);
    return;
  }
  auto kern = k_gs_cluster<T, G, U, V, false>;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(kGsClThreads);
  cfg.dynamicSmemBytes = (size_t)gs_cl_smem<T>(lv.n);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  AMG_CUDA(cudaLaunchKernelEx(&cfg, kern, lv.n, lv.ncolours, cp, (int)post, (int)x_zero,
                              lv.k_rows(), lv.k_rowptr(), lv.k_col(), val, lv.nnzb, x, b, dinv,
                              (const double*)lv.wt, err));
}

template <typename T, typename V>
void launch_gs_cluster_v(const Level& lv, int cs, int G, bool post, bool x_zero, const V* val,
                         T* x, const T* b, const T* dinv, int* err, cudaStream_t s) {
  switch (G) {
    case 4: launch_gs_cluster_g<T, 4, V>(lv, cs, post, x_zero, val, x, b, dinv, err, s); break;
    case 8: launch_gs_cluster_g<T, 8, V>(lv, cs, post, x_zero, val, x, b, dinv, err, s); break;
    case 16: launch_gs_cluster_g<T, 16, V>(lv, cs, post, x_zero, val, x, b, dinv, err, s); break;
    default: launch_gs_cluster_g<T, 32, V>(lv, cs, post, x_zero, val, x, b, dinv, err, s); break;
  }
}

// A level can sweep in one cluster when it is coloured, stored in colour order,
// has at most kGsClMaxColours colours and its iterate, right-hand side, row ids
// and block offsets fit in shared memory.
template <typename T>
bool gs_cluster_eligible(const Level& lv) {
  return lv.ncolours > 0 && lv.ncolours <= kGsClMaxColours && lv.k_rows() && lv.np == 0 &&
         gs_cl_smem<T>(lv.n) <= kGsClSmemBytes;
}

template <typename T>
int gs_cluster_fits_level(const Level& lv, int cs, int G) {
  const int smem = (int)gs_cl_smem<T>(lv.n);
  if constexpr (std::is_same<T, float>::value) {
    if (lv.val16.p) {
      switch (G) {
        case 4: return gs_cluster_fits<float, 4, __nv_bfloat16>(cs, smem);
        case 8: return gs_cluster_fits<float, 8, __nv_bfloat16>(cs, smem);
        case 16: return gs_cluster_fits<float, 16, __nv_bfloat16>(cs, smem);
        default: return gs_cluster_fits<float, 32, __nv_bfloat16>(cs, smem);
      }
    }
  }
  switch (G) {
    case 4: return gs_cluster_fits<T, 4, T>(cs, smem);
    case 8: return gs_cluster_fits<T, 8, T>(cs, smem);
    case 16: return gs_cluster_fits<T, 16, T>(cs, smem);
    default: return gs_cluster_fits<T, 32, T>(cs, smem);
  }
}

// ------------------------------------------------------------------- FP32-pair operator

// The Krylov operator y = K_0 x without FP64 arithmetic (FP64 instructions issue
// at a small fraction of the FP32 rate on this GPU, and the FP64 product kernel
// is bound by them, not by memory).  Every value a = a_hi + a_lo and vector
// entry x = x_hi + x_lo is a pair of floats (the FP64 number to about 2^-48).
// A product is a_hi x_hi exactly (rounded product p plus its error
// fma(a_hi, x_hi, -p)) plus the cross terms a_hi x_lo + a_lo x_hi; a_lo x_lo
// (about 2^-48 of the product) is dropped.  The rounded products are summed
// with TwoSum (Knuth), whose error terms join the low-order accumulator, so the
// row sum S + s carries about 2^-48 of sum |a_ij x_j| (pair_fma, pair_add).
//
// One group of G lanes per block row (rows in the level's kernel layout, as the
// FP64 operator kernel); each lane takes U blocks per step; x gathers are two
// 16-byte loads (hi and lo of the node).
template <int G, int U>
__global__ void __launch_bounds__(256) k_apply_pair(int nrows, const int* __restrict__ rows,
                                                    const int* __restrict__ rowptr,
                                                    const int* __restrict__ col,
                                                    const float2* __restrict__ val, int64_t nnzb,
                                                    const float* __restrict__ xp,
                                                    double* __restrict__ y) {
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31, sub = lane / G, gl = lane & (G - 1);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const float4* xv = reinterpret_cast<const float4*>(xp);
  for (int base = warp * RPW; base < nrows; base += nwarps * RPW) {
    const int g = base + sub;
    const bool active = g < nrows;
    float S0 = 0.f, s0 = 0.f, S1 = 0.f, s1 = 0.f, S2 = 0.f, s2 = 0.f;
    if (active) {
      const int a = __ldg(rowptr + g), e = __ldg(rowptr + g + 1);
      for (int k0 = a + gl; k0 < e; k0 += U * G) {
        int j[U];
        float2 v[U][9];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int k = k0 + u * G;
          if (k < e) {
            j[u] = __ldcs(col + k);
#pragma unroll
            for (int q = 0; q < 9; ++q) v[u][q] = __ldcs(val + q * nnzb + k);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (k0 + u * G >= e) continue;
          const float4 hi = __ldg(xv + 2 * (int64_t)j[u]);
          const float4 lo = __ldg(xv + 2 * (int64_t)j[u] + 1);
          pair_fma(S0, s0, v[u][0], hi.x, lo.x);
          pair_fma(S0, s0, v[u][1], hi.y, lo.y);
          pair_fma(S0, s0, v[u][2], hi.z, lo.z);
          pair_fma(S1, s1, v[u][3], hi.x, lo.x);
          pair_fma(S1, s1, v[u][4], hi.y, lo.y);
          pair_fma(S1, s1, v[u][5], hi.z, lo.z);
          pair_fma(S2, s2, v[u][6], hi.x, lo.x);
          pair_fma(S2, s2, v[u][7], hi.y, lo.y);
          pair_fma(S2, s2, v[u][8], hi.z, lo.z);
        }
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      float T = __shfl_xor_sync(0xffffffffu, S0, o), t = __shfl_xor_sync(0xffffffffu, s0, o);
      pair_add(S0, s0, T, t);
      T = __shfl_xor_sync(0xffffffffu, S1, o); t = __shfl_xor_sync(0xffffffffu, s1, o);
      pair_add(S1, s1, T, t);
      T = __shfl_xor_sync(0xffffffffu, S2, o); t = __shfl_xor_sync(0xffffffffu, s2, o);
      pair_add(S2, s2, T, t);
    }
    if (!active || gl != 0) continue;
    const int i = rows ? __ldg(rows + g) : g;
    st3(y, i, (double)S0 + (double)s0, (double)S1 + (double)s1, (double)S2 + (double)s2);
  }
}

template <int G>
void launch_apply_pair(const Level& lv, const float* xp, double* y, cudaStream_t s) {
  constexpr int U = G >= 16 ? 1 : 2;
  const int grid = (int)std::max<int64_t>(1, ((int64_t)lv.n * G + 255) / 256);
  k_apply_pair<G, U><<<grid, 256, 0, s>>>(lv.n, lv.k_rows(), lv.k_rowptr(), lv.k_col(),
                                          lv.val2.p, lv.nnzb, xp, y);
}

// Residual r = b - K x restricted to the unknowns of one Vanka colour: the velocity
// nodes of its patches (warp per node, one block of the node's A row and one entry
// of its B^T row per lane and step) and the pressure unknowns of its patches (the
// last npres warps' work).  Reads x only, so every patch of the colour then sees the
// residual of the colour's start.
template <typename T>
__global__ void __launch_bounds__(256) k_vk_resid(
    int nnodes, const int* __restrict__ nodes, int npres, const int* __restrict__ pres,
    const int* __restrict__ rowptr, const int* __restrict__ col, const T* __restrict__ val,
    int64_t nnzb, const int* __restrict__ btrow, const int* __restrict__ btcol,
    const T* __restrict__ btval, const int* __restrict__ brow, const int* __restrict__ bcol,
    const T* __restrict__ bval, int64_t bnnz, const int* __restrict__ crow,
    const int* __restrict__ ccol, const T* __restrict__ cval, const T* x, const T* b, T* r,
    int n4) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nnodes + npres; w += nwarps) {
    if (w < nnodes) {
      const int i = nodes[w];
      T s0 = T(0), s1 = T(0), s2 = T(0);
      for (int k = rowptr[i] + lane; k < rowptr[i + 1]; k += 32) {
        T x0, x1, x2;
        ld3(x, col[k], x0, x1, x2);
        s0 = fma(val[k], x0, fma(val[nnzb + k], x1, fma(val[2 * nnzb + k], x2, s0)));
        s1 = fma(val[3 * nnzb + k], x0, fma(val[4 * nnzb + k], x1, fma(val[5 * nnzb + k], x2, s1)));
        s2 = fma(val[6 * nnzb + k], x0, fma(val[7 * nnzb + k], x1, fma(val[8 * nnzb + k], x2, s2)));
      }
      for (int q = btrow[i] + lane; q < btrow[i + 1]; q += 32) {
        const T pk = x[n4 + btcol[q]];
        s0 = fma(btval[q], pk, s0);
        s1 = fma(btval[bnnz + q], pk, s1);
        s2 = fma(btval[2 * bnnz + q], pk, s2);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      }
      if (lane == 0) {
        T b0, b1, b2;
        ld3(b, i, b0, b1, b2);
        st3(r, i, b0 - s0, b1 - s1, b2 - s2);
      }
    } else {
      const int k = pres[w - nnodes];
      T acc = T(0);
      for (int q = brow[k] + lane; q < brow[k + 1]; q += 32) {
        T u0, u1, u2;
        ld3(x, bcol[q], u0, u1, u2);
        acc = fma(bval[q], u0, fma(bval[bnnz + q], u1, fma(bval[2 * bnnz + q], u2, acc)));
      }
      for (int q = crow[k] + lane; q < crow[k + 1]; q += 32) acc -= cval[q] * x[n4 + ccol[q]];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) r[n4 + k] = b[n4 + k] - acc;
    }
  }
}

// one operation as its own kernel
template <typename T>
__global__ void __launch_bounds__(256) k_phase(const Phase P) {
  exec_phase<T, false>(P, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// the block-row operations as their own specialised kernels (the hot path)
template <typename T, int G, int MODE, typename V = T>
__global__ void __launch_bounds__(256) k_rows(const Phase P) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  rows_body<T, G, MODE, false, V>(P.n, P.rows, P.rowptr, P.col, (const V*)P.val, P.nnz,
                               (const T*)P.x, (const T*)P.b, (T*)P.y, (const T*)P.dinv,
                               (T)P.omega, P.wt, tid >> 5, (gridDim.x * blockDim.x) >> 5);
}

template <typename T, int G, typename V>
void launch_rows_mode(const Phase& P, int grid, cudaStream_t s) {
  switch (P.mode) {
    case kApply: k_rows<T, G, kApply, V><<<grid, 256, 0, s>>>(P); break;
    case kResid: k_rows<T, G, kResid, V><<<grid, 256, 0, s>>>(P); break;
    case kGS: k_rows<T, G, kGS, V><<<grid, 256, 0, s>>>(P); break;
    default: k_rows<T, G, kJacobi, V><<<grid, 256, 0, s>>>(P); break;
  }
}

// Multicolour Gauss-Seidel for one colour as a grid-stride kernel over a grid
// of `sctas` CTAs per SM, launched with programmatic dependent launch.  Each warp
// keeps two register sets of row operands (block columns, the values of U blocks
// per lane, D_i^{-1}): the next row group's are loaded, straight from HBM and
// without any dependence on x, while the current group gathers x and updates,
// so the value stream does not stop at each group's x gathers, and the grid
// leaves room on every SM for the next colour's kernel to start its prologue.
// The loop runs in two halves with the sets' roles swapped (no register copy).
// As in k_gs_pdl only setup constants are read before griddepcontrol.wait.
template <typename T, int G, int U>
struct GsSet {
  int i, a, e;
  int j[U];
  T v[U][9];
  T d[9];
};

template <typename T, int G, int U>
__device__ __forceinline__ void gs_set_load(GsSet<T, G, U>& o, int g, int nrows,
                                            const int* __restrict__ rows,
                                            const int* __restrict__ rowptr,
                                            const int* __restrict__ col,
                                            const T* __restrict__ val, int64_t nnzb,
                                            const T* __restrict__ dinv, int gl) {
  o.a = o.e = 0;
#pragma unroll
  for (int u = 0; u < U; ++u) o.j[u] = -1;
  if (g >= nrows) return;
  o.i = ldg(rows + g);
  o.a = ldg(rowptr + g);
  o.e = ldg(rowptr + g + 1);
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int k = o.a + gl + u * G;
    if (k < o.e) {
      o.j[u] = __ldcs(col + k);
#pragma unroll
      for (int q = 0; q < 9; ++q) o.v[u][q] = __ldcs(val + q * nnzb + k);
    }
  }
  if (gl == 0) {
    const T* dp = dinv + 12 * (int64_t)o.i;
    ld3(dp, 0, o.d[0], o.d[1], o.d[2]);
    ld3(dp, 1, o.d[3], o.d[4], o.d[5]);
    ld3(dp, 2, o.d[6], o.d[7], o.d[8]);
  }
}

template <typename T, int G, int U>
__device__ __forceinline__ void gs_set_update(const GsSet<T, G, U>& o, bool active,
                                              const int* __restrict__ col,
                                              const T* __restrict__ val, int64_t nnzb, T* x,
                                              const T* __restrict__ b, T om, int gl) {
  T s0 = T(0), s1 = T(0), s2 = T(0);
  T b0 = T(0), b1 = T(0), b2 = T(0), xi0 = T(0), xi1 = T(0), xi2 = T(0);
  if (active) {
    if (gl == 0) {
      ld3(b, o.i, b0, b1, b2);
      VL<true>::node(x, o.i, xi0, xi1, xi2);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (o.j[u] < 0) continue;
      T x0, x1, x2;
      VL<true>::node(x, o.j[u], x0, x1, x2);
      s0 = fma(o.v[u][0], x0, s0); s0 = fma(o.v[u][1], x1, s0); s0 = fma(o.v[u][2], x2, s0);
      s1 = fma(o.v[u][3], x0, s1); s1 = fma(o.v[u][4], x1, s1); s1 = fma(o.v[u][5], x2, s1);
      s2 = fma(o.v[u][6], x0, s2); s2 = fma(o.v[u][7], x1, s2); s2 = fma(o.v[u][8], x2, s2);
    }
    for (int k = o.a + gl + U * G; k < o.e; k += G) {   // blocks beyond the set
      const int jj = ldg(col + k);
      T x0, x1, x2;
      VL<true>::node(x, jj, x0, x1, x2);
      const T* vv = val + k;
      s0 = fma(ldg(vv), x0, s0);
      s0 = fma(ldg(vv + nnzb), x1, s0);
      s0 = fma(ldg(vv + 2 * nnzb), x2, s0);
      s1 = fma(ldg(vv + 3 * nnzb), x0, s1);
      s1 = fma(ldg(vv + 4 * nnzb), x1, s1);
      s1 = fma(ldg(vv + 5 * nnzb), x2, s1);
      s2 = fma(ldg(vv + 6 * nnzb), x0, s2);
      s2 = fma(ldg(vv + 7 * nnzb), x1, s2);
      s2 = fma(ldg(vv + 8 * nnzb), x2, s2);
    }
  }
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  }
  if (!active || gl != 0) return;
  const T r0 = b0 - s0, r1 = b1 - s1, r2 = b2 - s2;
  const T* d = o.d;
  st3(x, o.i, xi0 + om * (d[0] * r0 + d[1] * r1 + d[2] * r2),
      xi1 + om * (d[3] * r0 + d[4] * r1 + d[5] * r2), xi2 + om * (d[6] * r0 + d[7] * r1 + d[8] * r2));
}

template <typename T, int G, int U>
__global__ void __launch_bounds__(256) k_gs_stream(int nrows, const int* __restrict__ rows,
                                                   const int* __restrict__ rowptr,
                                                   const int* __restrict__ col,
                                                   const T* __restrict__ val, int64_t nnzb, T* x,
                                                   const T* __restrict__ b,
                                                   const T* __restrict__ dinv,
                                                   const double* __restrict__ wt) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  constexpr int R = 32 / G;
  const int lane = threadIdx.x & 31, sub = lane / G, gl = lane & (G - 1);
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int step = (int)((gridDim.x * blockDim.x) >> 5) * R;
  GsSet<T, G, U> A, Bs;
  int g = warp * R + sub;
  gs_set_load(A, g, nrows, rows, rowptr, col, val, nnzb, dinv, gl);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const T om = wt ? (T)wt[0] : T(1);   // learned relaxation multiplier (1: plain)
  // rows of one colour are not neighbours: the x gathers read only earlier
  // colours' values (L2-coherent loads all the same, the kernel writes x)
  for (int base = warp * R; base < nrows; base += 2 * step) {
    gs_set_load(Bs, g + step, nrows, rows, rowptr, col, val, nnzb, dinv, gl);
    gs_set_update(A, g < nrows, col, val, nnzb, x, b, om, gl);
    if (base + step >= nrows) break;
    gs_set_load(A, g + 2 * step, nrows, rows, rowptr, col, val, nnzb, dinv, gl);
    gs_set_update(Bs, g + step < nrows, col, val, nnzb, x, b, om, gl);
    g += 2 * step;
  }
}

template <typename T, int G>
void launch_gs_stream(const Phase& P, cudaStream_t s) {
  constexpr int U = 2;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    AMG_CUDA(cudaGetDevice(&dev));
    AMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const int64_t want = ((int64_t)P.n * G + 255) / 256;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)P.sctas * sms)));
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  AMG_CUDA(cudaLaunchKernelEx(&cfg, k_gs_stream<T, G, U>, P.n, P.rows, P.rowptr, P.col,
                              (const T*)P.val, P.nnz, (T*)P.y, (const T*)P.b,
                              (const T*)P.dinv, P.wt));
}

// ------------------------------------------------- TMA-staged colour kernel (FP32)

// The colour kernel with the block values and columns of a CTA's rows staged in shared
// memory by 1-D bulk copies (cp.async.bulk, the TMA's linear mode), issued before
// griddepcontrol.wait since they are setup constants.  A colour's rows are consecutive
// in the kernel layout, so the blocks of a CTA's R = 256 / G rows are one range [A, E)
// of each of the 9 value planes and of the column array.  The copies hold no registers:
// more rows are in flight per SM than with k_gs_pdl's register prefetch, whose
// registers cap its occupancy.  Up to kTmaBlocksPerRow * R blocks are staged; blocks
// beyond that (rows far longer than a level's average) are read from global memory.
// A plane's copy starts at the 16-byte boundary at or below its first element and
// ends at the boundary at or below its last; the up to 3 elements after that are
// loaded by threads.  A row's sums run in k_gs_pdl's order for the same G (lane gl
// takes blocks a + gl, a + gl + G, ...), so both kernels give the same bits.  The
// one mbarrier wait is bounded: a CTA that gives up sets *err, waits (bounded) once
// more for its copies and returns.
constexpr int kTmaBlocksPerRow = 36;
constexpr unsigned kTmaSpins = 1u << 20;
template <int G>
constexpr int tma_cap() { return (256 / G) * kTmaBlocksPerRow; }   // a multiple of 4
template <int G>
constexpr int tma_smem() { return 10 * (tma_cap<G>() + 4) * (int)sizeof(float); }

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool tma_wait(uint32_t bar) {
  for (unsigned i = 0; i < kTmaSpins; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <int G, bool XNC>
__global__ void __launch_bounds__(256) k_gs_tma(int nrows, const int* __restrict__ rows,
                                                const int* __restrict__ rowptr,
                                                const int* __restrict__ col,
                                                const float* __restrict__ val, int64_t nnzb,
                                                float* x, const float* __restrict__ b,
                                                const float* __restrict__ dinv,
                                                const double* __restrict__ wt,
                                                int* __restrict__ err) {
  extern __shared__ __align__(128) float tma_sm[];
  __shared__ __align__(8) uint64_t tbar;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  constexpr int R = 256 / G;
  constexpr int CAP = tma_cap<G>();
  constexpr int PL = CAP + 4;                  // plane stride in shared memory
  const int g0 = blockIdx.x * R;
  const int g1 = min(g0 + R, nrows);
  const int A = __ldg(rowptr + g0), E = __ldg(rowptr + g1);
  const int Es = min(E, A + CAP);              // staged blocks [A, Es)
  const uint32_t bar = smem_addr(&tbar);
  const uint32_t sm0 = smem_addr(tma_sm);
  // plane p: values p < 9 (element base p * nnzb of val), the columns p = 9 (base 0 of
  // col); global elements [fs, fe) by bulk copy, fs = floor4(base + A),
  // fe = floor4(base + Es); block k sits at position k - A + (base + A - fs)
  if (threadIdx.x == 0) {
    mbar_init(bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();   // the barrier is initialised before any thread polls it
  if (threadIdx.x == 0) {
    uint32_t total = 0;
    for (int p = 0; p < 10; ++p) {
      const int64_t base = p < 9 ? (int64_t)p * nnzb : 0;
      const int64_t fs = (base + A) & ~int64_t(3), fe = (base + Es) & ~int64_t(3);
      if (fe > fs) total += (uint32_t)(fe - fs) * 4u;
    }
    mbar_expect(bar, total);
    for (int p = 0; p < 10; ++p) {
      const int64_t base = p < 9 ? (int64_t)p * nnzb : 0;
      const int64_t fs = (base + A) & ~int64_t(3), fe = (base + Es) & ~int64_t(3);
      const float* src = p < 9 ? val + fs : reinterpret_cast<const float*>(col) + fs;
      if (fe > fs) bulk_g2s(sm0 + (uint32_t)(p * PL) * 4u, src, (uint32_t)(fe - fs) * 4u, bar);
    }
  }
  // the tails: at most 3 elements a plane past the last 16-byte boundary
  if (threadIdx.x < 40) {
    const int p = threadIdx.x >> 2, t = threadIdx.x & 3;
    const int64_t base = p < 9 ? (int64_t)p * nnzb : 0;
    const int64_t gs = base + A, ge = base + Es;
    const int64_t fs = gs & ~int64_t(3), fe = ge & ~int64_t(3);
    const int64_t idx = (fe > gs ? fe : gs) + t;
    if (idx < ge) {
      const float* src = p < 9 ? val : reinterpret_cast<const float*>(col);
      tma_sm[p * PL + (int)(idx - fs)] = __ldg(src + idx);
    }
  }
  const int g = g0 + (int)(threadIdx.x / G);
  const int gl = threadIdx.x & (G - 1);
  const bool active = g < g1;
  int i = 0, a = 0, e = 0;
  float d[9];
  if (active) {
    i = __ldg(rows + g);
    a = __ldg(rowptr + g);
    e = __ldg(rowptr + g + 1);
    if (gl == 0) {
      const float* dp = dinv + 12 * (int64_t)i;
      ld3(dp, 0, d[0], d[1], d[2]);
      ld3(dp, 1, d[3], d[4], d[5]);
      ld3(dp, 2, d[6], d[7], d[8]);
    }
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const bool ok = tma_wait(bar);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicExch(err, 1);
      tma_wait(bar);
    }
    return;
  }
  const float om = wt ? (float)wt[0] : 1.f;   // learned relaxation multiplier (1: plain)
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  float b0 = 0.f, b1 = 0.f, b2 = 0.f, xi0 = 0.f, xi1 = 0.f, xi2 = 0.f;
  if (active) {
    if (gl == 0) {
      ld3(b, i, b0, b1, b2);
      VL<!XNC>::node(x, i, xi0, xi1, xi2);
    }
    int off[10];
#pragma unroll
    for (int p = 0; p < 10; ++p) {
      const int64_t base = p < 9 ? (int64_t)p * nnzb : 0;
      off[p] = p * PL + (int)((base + A) & 3) - A;   // position of block k: k + off[p]
    }
    for (int k = a + gl; k < e; k += G) {
      int jj;
      float v[9];
      if (k < Es) {
        jj = __float_as_int(tma_sm[k + off[9]]);
#pragma unroll
        for (int q = 0; q < 9; ++q) v[q] = tma_sm[k + off[q]];
      } else {
        jj = __ldg(col + k);
#pragma unroll
        for (int q = 0; q < 9; ++q) v[q] = __ldg(val + q * nnzb + k);
      }
      float x0, x1, x2;
      VL<!XNC>::node(x, jj, x0, x1, x2);
      s0 = fmaf(v[0], x0, s0); s0 = fmaf(v[1], x1, s0); s0 = fmaf(v[2], x2, s0);
      s1 = fmaf(v[3], x0, s1); s1 = fmaf(v[4], x1, s1); s1 = fmaf(v[5], x2, s1);
      s2 = fmaf(v[6], x0, s2); s2 = fmaf(v[7], x1, s2); s2 = fmaf(v[8], x2, s2);
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (!active || gl != 0) return;
  const float r0 = b0 - s0, r1 = b1 - s1, r2 = b2 - s2;
  st3(x, i, xi0 + om * (d[0] * r0 + d[1] * r1 + d[2] * r2),
      xi1 + om * (d[3] * r0 + d[4] * r1 + d[5] * r2), xi2 + om * (d[6] * r0 + d[7] * r1 + d[8] * r2));
}

template <int G, bool XNC>
void launch_gs_tma_x(const Phase& P, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    AMG_CUDA(cudaFuncSetAttribute(k_gs_tma<G, XNC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tma_smem<G>()));
    attr = true;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(((int64_t)P.n * G + 255) / 256));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = tma_smem<G>();
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  AMG_CUDA(cudaLaunchKernelEx(&cfg, k_gs_tma<G, XNC>, P.n, P.rows, P.rowptr, P.col,
                              (const float*)P.val, P.nnz, (float*)P.y, (const float*)P.b,
                              (const float*)P.dinv, P.wt, P.err));
}

template <int G>
void launch_gs_tma(const Phase& P, cudaStream_t s) {
  if (P.xnc) launch_gs_tma_x<G, true>(P, s);
  else launch_gs_tma_x<G, false>(P, s);
}

template <typename T, typename V>
void launch_rows_v(const Phase& P, cudaStream_t s, bool pdl) {
  if constexpr (std::is_same<T, V>::value) {
    if (pdl && P.mode == kGS && P.rows && P.sctas > 0) {
      switch (P.G) {
        case 4: launch_gs_stream<T, 4>(P, s); return;
        case 8: launch_gs_stream<T, 8>(P, s); return;
        case 16: launch_gs_stream<T, 16>(P, s); return;
        default: launch_gs_stream<T, 32>(P, s); return;
      }
    }
  }
  if constexpr (std::is_same<T, float>::value && std::is_same<V, float>::value) {
    if (pdl && P.mode == kGS && P.rows && P.tma && P.n > 0) {
      switch (P.G) {
        case 4: launch_gs_tma<4>(P, s); return;
        case 8: launch_gs_tma<8>(P, s); return;
        case 16: launch_gs_tma<16>(P, s); return;
        default: launch_gs_tma<32>(P, s); return;
      }
    }
  }
  if (pdl && P.mode == kGS && P.rows) {
    switch (P.G) {
      case 4: launch_gs_pdl<T, 4, V>(P, s); return;
      case 8: launch_gs_pdl<T, 8, V>(P, s); return;
      case 16: launch_gs_pdl<T, 16, V>(P, s); return;
      default: launch_gs_pdl<T, 32, V>(P, s); return;
    }
  }
  // one group of G lanes per row: nrows * G threads
  const int grid = (int)(((int64_t)P.n * P.G + 255) / 256);
  switch (P.G) {
    case 4: launch_rows_mode<T, 4, V>(P, grid, s); break;
    case 8: launch_rows_mode<T, 8, V>(P, grid, s); break;
    case 16: launch_rows_mode<T, 16, V>(P, grid, s); break;
    default: launch_rows_mode<T, 32, V>(P, grid, s); break;
  }
}

template <typename T>
void launch_rows(const Phase& P, cudaStream_t s, bool pdl) {
  if constexpr (std::is_same<T, float>::value) {
    if (P.vbf) {
      launch_rows_v<float, __nv_bfloat16>(P, s, pdl);
      return;
    }
  }
  launch_rows_v<T, T>(P, s, pdl);
}

// The recorded phases of the small coarse levels in one thread-block cluster.
// The cluster barrier (arrive.release / wait.acquire) orders every phase's
// writes before the next phase's reads; vectors are read through L2.
constexpr int kSubThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kSubThreads, 1) k_subcycle(const Phase* __restrict__ ph,
                                                               int nph) {
  cg::cluster_group cl = cg::this_cluster();
  const int nthr = blockDim.x * (int)cl.num_blocks();
  const int tid = (int)cl.block_rank() * blockDim.x + threadIdx.x;
  for (int p = 0; p < nph; ++p) {
    const Phase P = ph[p];
    exec_phase<T, true>(P, tid, nthr);
    cl.sync();
  }
}

// Grid-wide barrier of the persistent cycle kernel (all CTAs co-resident by
// cooperative launch).  `count` only grows during a launch: barrier number k
// completes when it reaches k * gridDim.x.  Every wait is bounded: after
// kBarrierSpins polls the CTA records a timeout in *err and stops waiting; once
// *err is set no CTA waits any more, so the kernel always ends.
constexpr unsigned kBarrierSpins = 1u << 22;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void grid_barrier(unsigned* count, unsigned target, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    unsigned spins = 0;
    while (ld_acquire(count) < target) {
      if (++spins > kBarrierSpins) { atomicOr(err, 1); break; }
      if ((spins & 1023u) == 0 && *((volatile int*)err)) break;
    }
    __threadfence();
  }
  __syncthreads();
}

// The whole recorded cycle as one persistent launch over all SMs.
constexpr int kGridThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kGridThreads, 1) k_grid_cycle(const Phase* __restrict__ ph,
                                                                  int nph, unsigned* bar,
                                                                  int* err) {
  const int nthr = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int p = 0; p < nph; ++p) {
    const Phase P = ph[p];
    exec_phase<T, true>(P, tid, nthr);
    if (p + 1 < nph) grid_barrier(bar, (unsigned)(p + 1) * gridDim.x, err);
  }
}

// ------------------------------------------------------------------- emitter

inline int gridn(int64_t n, int t = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 152 * 16));
}

template <typename T> struct LvVec;
template <> struct LvVec<double> {
  static double* x(Level& l) { return l.x64; }
  static double* b(Level& l) { return l.b64; }
  static double* r(Level& l) { return l.r64; }
  static double* t(Level& l) { return l.t64; }
  static const double* val(Level& l) { return l.k_val(); }
  static const double* dinv(Level& l) { return l.dinv; }
  static const double* pval(Level& l) { return l.p_val; }
  static const double* rval(Level& l) { return l.r_val; }
  static const double* bval(Level& l) { return l.b_val; }
  static const double* btval(Level& l) { return l.bt_val; }
  static const double* cval(Level& l) { return l.c_val; }
  static const double* hval(Level& l) { return l.h_val; }
  static const double* htval(Level& l) { return l.ht_val; }
  static const double* schur(Level& l) { return l.schur; }
};
template <> struct LvVec<float> {
  static float* x(Level& l) { return l.x32; }
  static float* b(Level& l) { return l.b32; }
  static float* r(Level& l) { return l.r32; }
  static float* t(Level& l) { return l.t32; }
  static const float* val(Level& l) { return l.val32; }
  static const float* dinv(Level& l) { return l.dinv32; }
  static const float* pval(Level& l) { return l.p_val32; }
  static const float* rval(Level& l) { return l.r_val32; }
  static const float* bval(Level& l) { return l.b_val32; }
  static const float* btval(Level& l) { return l.bt_val32; }
  static const float* cval(Level& l) { return l.c_val32; }
  static const float* hval(Level& l) { return l.h_val32; }
  static const float* htval(Level& l) { return l.ht_val32; }
  static const float* schur(Level& l) { return l.schur32; }
};

template <typename T> struct SVec;
template <> struct SVec<double> {
  static double* x(SLevel& q) { return q.x64; }
  static double* b(SLevel& q) { return q.b64; }
  static double* r(SLevel& q) { return q.r64; }
  static const double* val(SLevel& q) { return q.val; }
  static const double* dinv(SLevel& q) { return q.dinv; }
  static const double* ahinv(Level& l) { return l.ahinv; }
};
template <> struct SVec<float> {
  static float* x(SLevel& q) { return q.x32; }
  static float* b(SLevel& q) { return q.b32; }
  static float* r(SLevel& q) { return q.r32; }
  static const float* val(SLevel& q) { return q.val32; }
  static const float* dinv(SLevel& q) { return q.dinv32; }
  static const float* ahinv(Level& l) { return l.ahinv32; }
};

template <typename T> struct VkVec;
template <> struct VkVec<double> {
  static const double* ainv(Level& l) { return l.vk_ainv; }
  static const double* w(Level& l) { return l.vk_w; }
  static const double* s(Level& l) { return l.vk_s; }
};
template <> struct VkVec<float> {
  static const float* ainv(Level& l) { return l.vk_ainv32; }
  static const float* w(Level& l) { return l.vk_w32; }
  static const float* s(Level& l) { return l.vk_s32; }
};

// damping of the Vanka correction (the paper gives none; 0.7 is the reading)
constexpr double kVankaOmega = 0.7;

// damping of the scalar Jacobi smoother of the S-cycle (Braess-Sarazin)
constexpr double kBsJacobi = 0.5;

// lanes per block row: the autotuned value, else from the average row length
inline int group_for(const Level& lv) {
  if (lv.group) return lv.group;
  if (lv.avg_row_blocks > 20.0) return 32;
  if (lv.avg_row_blocks > 10.0) return 16;
  if (lv.avg_row_blocks > 5.0) return 8;
  return 4;
}

// Launches each operation as a kernel (rec == nullptr) or appends it to `rec`.
template <typename T>
struct Emit {
  amg_handle* h;
  std::vector<Phase>* rec = nullptr;

  void put(const Phase& P, int64_t work, int threads_per_item = 1) {
    if (rec) {
      rec->push_back(P);
      return;
    }
    if (work <= 0) return;
    if (P.type == PH_ROWS) launch_rows<T>(P, h->stream, h->use_pdl);
    else if (P.type == PH_VANKA)
      k_vanka<T><<<(unsigned)std::min<int64_t>(work, 152 * 8), 256, 0, h->stream>>>(
          P.n, P.rows, P.rowptr, P.col, (const T*)P.val, P.nnz, P.off, (const T*)P.dinv,
          (const T*)P.cval, (const T*)P.sd, (const T*)P.x, (T*)P.y, P.n3, (T)P.omega);
    else k_phase<T><<<gridn(work * threads_per_item), 256, 0, h->stream>>>(P);
    h->launches++;
  }
  static Phase blank(int type) {
    Phase P;
    std::memset(&P, 0, sizeof(P));
    P.type = type;
    return P;
  }
  // block rows [first, first + nrows) of the level's kernel layout
  void rows(int mode, const Level& lv, int G, int first, int nrows, const T* val, const T* x,
            const T* b, T* y, const T* dinv, T omega) {
    Phase P = blank(PH_ROWS);
    P.wt = (mode == kGS || mode == kJacobi) ? lv.wt : nullptr;
    const int* order = lv.k_rows();
    P.mode = mode; P.G = G; P.n = nrows; P.rows = order ? order + first : nullptr;
    P.rowptr = lv.k_rowptr() + first; P.col = lv.k_col();
    P.val = val; P.nnz = lv.nnzb; P.x = x; P.b = b; P.y = y; P.dinv = dinv; P.omega = omega;
    P.sctas = mode == kGS ? lv.gs_stream : 0;
    P.xnc = mode == kGS ? lv.gs_xnc : 0;
    P.tma = mode == kGS ? lv.gs_tma : 0;
    P.err = h->flag.p;
    if (sizeof(T) == 4 && lv.val16.p && (const void*)val == (const void*)lv.val32.p) {
      P.val = lv.val16.p;   // BF16 storage of this level's values
      P.vbf = 1;
    }
    put(P, nrows, G);
  }
  // a level's whole colour sweep as one cluster launch (never recorded)
  void gs_cluster(Level& lv, T* x, const T* b, bool post, bool x_zero) {
    const T* dinv = LvVec<T>::dinv(lv);
    if constexpr (std::is_same<T, float>::value) {
      if (lv.val16.p) {
        launch_gs_cluster_v<float, __nv_bfloat16>(
            lv, lv.gs_cl, lv.gs_cl_g, post, x_zero,
            reinterpret_cast<const __nv_bfloat16*>(lv.val16.p), x, b, dinv, h->flag.p,
            h->stream);
        h->launches++;
        return;
      }
    }
    launch_gs_cluster_v<T, T>(lv, lv.gs_cl, lv.gs_cl_g, post, x_zero, LvVec<T>::val(lv), x, b,
                              dinv, h->flag.p, h->stream);
    h->launches++;
  }
  // a level's whole colour sweep as one dataflow launch (never recorded)
  void gs_flow(Level& lv, T* x, const T* b, bool reverse) {
    launch_gs_flow<T>(h, lv, x, b, LvVec<T>::val(lv), LvVec<T>::dinv(lv), reverse);
  }
  void zero(T* a, int64_t n) {
    Phase P = blank(PH_ZERO);
    P.y = a; P.n = (int)n;
    put(P, n);
  }
  void copy(const T* a, T* b, int64_t n) {
    Phase P = blank(PH_COPY);
    P.x = a; P.y = b; P.n = (int)n;
    put(P, n);
  }
  void transfer(int type, int n, const int* row, const int* col, const T* val, const T* src,
                T* dst, const double* wt = nullptr) {
    Phase P = blank(type);
    P.n = n; P.rowptr = row; P.col = col; P.val = val; P.x = src; P.y = dst; P.wt = wt;
    put(P, n);
  }
  void coarse(const T* b, T* x) {
    Phase P = blank(PH_COARSE);
    P.m = h->coarse_m; P.n3 = 3 * h->L.back()->n; P.X = h->coarse_inv; P.b = b; P.y = x;
    put(P, P.m, 32);
  }
  void bt_add(Level& lv, const T* p, T sign, T* y) {
    Phase P = blank(PH_BT_ADD);
    P.n = lv.n; P.rowptr = lv.bt_rowptr; P.col = lv.bt_col; P.val = LvVec<T>::btval(lv);
    P.nnz = lv.b_nnz; P.x = p; P.omega = (double)sign; P.y = y;
    put(P, lv.n);
  }
  void srows(int mode, SLevel& q, const T* x, const T* b, T* y, T omega) {
    Phase P = blank(PH_SROWS);
    P.mode = mode; P.n = q.n; P.rowptr = q.rowptr; P.col = q.col; P.val = SVec<T>::val(q);
    P.nnz = q.nnz; P.x = x; P.b = b; P.y = y; P.dinv = SVec<T>::dinv(q); P.omega = (double)omega;
    put(P, q.n);
  }
  void vec(int mode, int64_t n, const T* d, const T* x, const T* b, T omega, T* y) {
    Phase P = blank(PH_VEC);
    P.mode = mode; P.n = (int)n; P.dinv = d; P.x = x; P.b = b; P.omega = (double)omega; P.y = y;
    put(P, n);
  }
  void vanka_resid(Level& lv, int c, const T* x, const T* b, T* r) {
    if (rec) fail(AMG_ERR_UNSUPPORTED, "the Vanka smoother runs with per-operation launches");
    const int a = lv.vk_colour_ptr[c], np = lv.vk_colour_ptr[c + 1] - a;
    const int na = lv.vk_cnode_ptr[c], nn = lv.vk_cnode_ptr[c + 1] - na;
    if (nn + np <= 0) return;
    k_vk_resid<T><<<gridn((int64_t)(nn + np) * 32), 256, 0, h->stream>>>(
        nn, lv.vk_cnodes.p + na, np, lv.vk_rows.p + a, lv.rowptr, lv.col, LvVec<T>::val(lv),
        lv.nnzb, lv.bt_rowptr, lv.bt_col, LvVec<T>::btval(lv), lv.b_rowptr, lv.b_col,
        LvVec<T>::bval(lv), lv.b_nnz, lv.c_rowptr, lv.c_col, LvVec<T>::cval(lv), x, b, r,
        4 * lv.n);
    h->launches++;
  }
  void vanka(Level& lv, int c, const T* r, T* x) {
    if (rec) fail(AMG_ERR_UNSUPPORTED, "the Vanka smoother runs with per-operation launches");
    Phase P = blank(PH_VANKA);
    const int a = lv.vk_colour_ptr[c];
    P.n = lv.vk_colour_ptr[c + 1] - a; P.rows = lv.vk_rows.p + a;
    P.rowptr = lv.b_rowptr; P.col = lv.b_col; P.val = LvVec<T>::bval(lv); P.nnz = lv.b_nnz;
    P.off = lv.vk_off; P.dinv = VkVec<T>::ainv(lv); P.cval = VkVec<T>::w(lv);
    P.sd = VkVec<T>::s(lv); P.x = r; P.y = x; P.n3 = 4 * lv.n; P.omega = kVankaOmega;
    put(P, P.n, 32);
  }
  void coarse_s(Level& lv, const T* b, T* x) {
    Phase P = blank(PH_COARSE);
    P.m = lv.s_coarse_m; P.n3 = 0; P.X = lv.s_coarse_inv; P.b = b; P.y = x;
    put(P, P.m, 32);
  }
  void prows(int mode, Level& lv, const T* u, const T* p, const T* g, T* yp, T omega) {
    Phase P = blank(PH_PROWS);
    P.mode = mode; P.n = lv.np; P.rowptr = lv.b_rowptr; P.col = lv.b_col;
    P.val = LvVec<T>::bval(lv); P.nnz = lv.b_nnz; P.crow = lv.c_rowptr; P.ccol = lv.c_col;
    P.cval = LvVec<T>::cval(lv); P.x = u; P.p = p; P.b = g; P.y = yp;
    P.sd = LvVec<T>::schur(lv); P.omega = (double)omega;
    P.wt = mode == 2 ? lv.wt : nullptr;
    put(P, lv.np, kProwLanes);
  }
};

// ------------------------------------------------------------------- level operations

template <typename T>
void e_apply(Emit<T>& e, Level& lv, const T* x, T* y, bool saddle) {
  const int G = (sizeof(T) == 8 && lv.group64) ? lv.group64 : group_for(lv);
  e.rows(kApply, lv, G, 0, lv.n, LvVec<T>::val(lv), x, nullptr, y, nullptr, T(0));
  if (saddle && lv.np > 0) {
    const T* p = x + 4 * lv.n;
    e.bt_add(lv, p, T(1), y);
    e.prows(0, lv, x, p, nullptr, y + 4 * lv.n, T(0));
  }
}

template <typename T>
void e_residual(Emit<T>& e, Level& lv, const T* x, const T* b, T* r, bool saddle) {
  e.rows(kResid, lv, group_for(lv), 0, lv.n, LvVec<T>::val(lv), x, b, r, nullptr, T(0));
  if (saddle && lv.np > 0) {
    const T* p = x + 4 * lv.n;
    e.bt_add(lv, p, T(-1), r);
    e.prows(1, lv, x, p, b + 4 * lv.n, r + 4 * lv.n, T(0));
  }
}

// One V(1,1)-cycle on the S hierarchy of level l from a zero initial guess
// (Braess-Sarazin: S^{-1} of Eq. (bssmpre)); the result is left in S_k.x.
template <typename T>
void e_scycle(Emit<T>& e, amg_handle* h, int l, int k, const T* rhs) {
  Level& lv = *h->L[l];
  SLevel& q = *lv.S[k];
  T* x = SVec<T>::x(q);
  if (k + 1 == (int)lv.S.size()) {
    e.coarse_s(lv, rhs, x);
    return;
  }
  T* r = SVec<T>::r(q);
  SLevel& nx = *lv.S[k + 1];
  Level& pk = *h->L[l + k];
  e.vec(0, q.n, SVec<T>::dinv(q), rhs, nullptr, T(kBsJacobi), x);   // x = w D^{-1} rhs
  e.srows(0, q, x, rhs, r, T(0));                                    // r = rhs - S x
  e.transfer(PH_RESTRICT1, nx.n, pk.ht_rowptr, pk.ht_col, LvVec<T>::htval(pk), r, SVec<T>::b(nx));
  e_scycle<T>(e, h, l, k + 1, SVec<T>::b(nx));
  e.transfer(PH_PROLONG1, q.n, pk.h_rowptr, pk.h_col, LvVec<T>::hval(pk), SVec<T>::x(nx), x);
  e.srows(1, q, x, rhs, r, T(kBsJacobi));                            // Jacobi into r
  e.copy(r, x, q.n);
}

// One Braess-Sarazin step, Eq. (bssm) with K^ of Eq. (bssmpre):
// r = b - K x; w = A^{-1} r_u; dp = S^{-1}(B w - r_p); x_u += w - A^{-1} B^T dp; p += dp.
template <typename T>
void e_smooth_bs(Emit<T>& e, amg_handle* h, int l, T* x, const T* b) {
  Level& lv = *h->L[l];
  const int64_t n4 = 4 * (int64_t)lv.n;
  T* r = LvVec<T>::r(lv);
  T* t = LvVec<T>::t(lv);
  const T* ah = SVec<T>::ahinv(lv);
  e_residual<T>(e, lv, x, b, r, true);
  e.vec(0, n4, ah, r, nullptr, T(1), t);                   // t_u = w
  e.prows(3, lv, t, nullptr, r + n4, t + n4, T(0));         // t_p = B w - r_p
  e_scycle<T>(e, h, l, 0, t + n4);
  const T* dp = SVec<T>::x(*lv.S[0]);
  e.zero(r, n4);
  e.bt_add(lv, dp, T(1), r);                                // r_u = B^T dp
  e.vec(2, n4, ah, t, r, T(1), x);                          // x_u += w - A^{-1} B^T dp
  e.vec(1, lv.np, nullptr, dp, nullptr, T(1), x + n4);      // p += dp
}

// One smoothing sweep (Sec. 3.3).  SPD: multicolour block GS (colours ascending,
// or descending when `post` is set: the post-smoothing order of the symmetric
// cycle) or damped block Jacobi.  Saddle: segregated Gauss-Seidel, Eq. (uzsm),
// Braess-Sarazin or Vanka (patch colours in the same order as GS).
template <typename T>
void e_smooth(Emit<T>& e, amg_handle* h, Level& lv, T* x, const T* b, bool post,
              bool x_is_zero) {
  const int dofs = lv.dofs4();
  if (!e.rec && lv.gs_cl > 0 && lv.gs_cl_bytes == (int)sizeof(T) && !h->saddle &&
      h->opt.smoother == AMG_SMOOTHER_GS) {
    e.gs_cluster(lv, x, b, post, x_is_zero);
    return;
  }
  if (x_is_zero) e.zero(x, dofs);
  if (!e.rec && lv.flow > 0 && !h->saddle && h->opt.smoother == AMG_SMOOTHER_GS &&
      !(sizeof(T) == 4 && lv.val16.p)) {
    e.gs_flow(lv, x, b, post);
    return;
  }
  const int G = group_for(lv);
  const T* val = LvVec<T>::val(lv);
  const T* dinv = LvVec<T>::dinv(lv);
  if (h->saddle && h->opt.smoother == AMG_SMOOTHER_BS) {
    int l = 0;
    while (h->L[l].get() != &lv) ++l;
    e_smooth_bs<T>(e, h, l, x, b);
    return;
  }
  if (h->saddle && h->opt.smoother == AMG_SMOOTHER_VANKA) {
    // multiplicative over the patch colours: the residual at the colour's unknowns
    // before each
    T* r = LvVec<T>::r(lv);
    for (int q = 0; q < lv.vk_ncolours; ++q) {
      const int c = post ? lv.vk_ncolours - 1 - q : q;
      e.vanka_resid(lv, c, x, b, r);     // the residual at the colour's unknowns
      e.vanka(lv, c, r, x);
    }
    return;
  }
  if (h->saddle) {
    T* t = LvVec<T>::t(lv);
    T* r = LvVec<T>::r(lv);
    const T* p = x + 4 * lv.n;
    // u <- u + omega D^{-1} (f - B^T p - A u)    (M_A = damped block Jacobi)
    e.copy(b, r, 4 * (int64_t)lv.n);
    e.bt_add(lv, p, T(-1), r);
    e.rows(kJacobi, lv, G, 0, lv.n, val, x, r, t, dinv, (T)h->opt.omega);
    e.copy(t, x, 4 * (int64_t)lv.n);
    // p <- p + omega_p S_D^{-1} (B u_new - C p - g)
    e.prows(2, lv, x, x + 4 * lv.n, b + 4 * lv.n, t + 4 * lv.n, (T)h->opt.omega_p);
    e.copy(t + 4 * lv.n, x + 4 * lv.n, lv.np);
    return;
  }
  if (h->opt.smoother == AMG_SMOOTHER_JACOBI) {
    T* t = LvVec<T>::t(lv);
    e.rows(kJacobi, lv, G, 0, lv.n, val, x, b, t, dinv, (T)h->opt.omega);
    e.copy(t, x, dofs);
    return;
  }
  const int Ggs = lv.group_gs ? lv.group_gs : G;
  for (int q = 0; q < lv.ncolours; ++q) {
    const int c = post ? lv.ncolours - 1 - q : q;
    const int a = lv.colour_ptr[c], e2 = lv.colour_ptr[c + 1];
    e.rows(kGS, lv, Ggs, a, e2 - a, val, x, b, x, dinv, T(1));
  }
}

template <typename T>
void e_restrict(Emit<T>& e, amg_handle* h, int l, const T* r, T* bc) {
  Level& lv = *h->L[l];
  Level& nx = *h->L[l + 1];
  e.transfer(PH_RESTRICT, nx.n, lv.r_rowptr, lv.r_col, LvVec<T>::rval(lv), r, bc);
  if (h->saddle && nx.np > 0)
    e.transfer(PH_RESTRICT1, nx.np, lv.ht_rowptr, lv.ht_col, LvVec<T>::htval(lv), r + 4 * lv.n,
               bc + 4 * nx.n);
}

template <typename T>
void e_prolong(Emit<T>& e, amg_handle* h, int l, const T* xc, T* x) {
  Level& lv = *h->L[l];
  Level& nx = *h->L[l + 1];
  e.transfer(PH_PROLONG, lv.n, lv.p_rowptr, lv.p_col, LvVec<T>::pval(lv), xc, x, lv.wt);
  if (h->saddle && lv.np > 0)
    e.transfer(PH_PROLONG1, lv.np, lv.h_rowptr, lv.h_col, LvVec<T>::hval(lv), xc + 4 * nx.n,
               x + 4 * lv.n, lv.wt);
}

template <typename T>
struct SubCycle;

template <typename T>
void cycle_rec(Emit<T>& e, amg_handle* h, int l, T* x, const T* b, bool x_is_zero);

// Steps 5-11 of Algorithm 1 seen from level l-1: the coarse solve when l is the
// coarsest level, else nu recursive calls from x_l = 0.  From the cluster level
// down they run as one recorded launch.
template <typename T>
void coarse_calls(Emit<T>& e, amg_handle* h, int l, T* xc, const T* bc) {
  const int L = (int)h->L.size() - 1;
  if (!e.rec && h->sub_from > 0 && l == h->sub_from) {
    SubCycle<T>::launch(h);
    return;
  }
  if (l == L) {
    e.coarse(bc, xc);
    return;
  }
  for (int k = 0; k < std::max(1, h->opt.nu); ++k) cycle_rec<T>(e, h, l, xc, bc, k == 0);
}

template <typename T>
void cycle_rec(Emit<T>& e, amg_handle* h, int l, T* x, const T* b, bool x_is_zero) {
  const int L = (int)h->L.size() - 1;
  if (l == L) {
    e.coarse(b, x);
    return;
  }
  Level& lv = *h->L[l];
  Level& nx = *h->L[l + 1];
  const amg_options& o = h->opt;
  bool zero = x_is_zero;
  for (int k = 0; k < o.m_pre; ++k) {
    e_smooth<T>(e, h, lv, x, b, false, zero);
    zero = false;
  }
  if (zero) e.zero(x, lv.dofs4());   // no pre-smoothing: x is still the zero initial guess
  T* r = LvVec<T>::r(lv);
  e_residual<T>(e, lv, x, b, r, h->saddle);
  T* bc = LvVec<T>::b(nx);
  T* xc = LvVec<T>::x(nx);
  e_restrict<T>(e, h, l, r, bc);
  coarse_calls<T>(e, h, l + 1, xc, bc);
  e_prolong<T>(e, h, l, xc, x);
  // post-smoothing: colours descending (symmetric cycle) or, with post_order = 1,
  // ascending as in pre-smoothing
  const bool reverse = o.post_order != 1;
  for (int k = 0; k < o.m_post; ++k) e_smooth<T>(e, h, lv, x, b, reverse, false);
}

template <typename T>
DBuf<unsigned char>& sub_buf(amg_handle* h);
template <>
DBuf<unsigned char>& sub_buf<float>(amg_handle* h) { return h->sub_ph32; }
template <>
DBuf<unsigned char>& sub_buf<double>(amg_handle* h) { return h->sub_ph64; }
template <typename T>
int& sub_count(amg_handle* h);
template <>
int& sub_count<float>(amg_handle* h) { return h->sub_n32; }
template <>
int& sub_count<double>(amg_handle* h) { return h->sub_n64; }

template <typename T>
struct SubCycle {
  // records what coarse_calls(from) does, on the level's own vectors
  static void record(amg_handle* h, int from) {
    std::vector<Phase> ph;
    Emit<T> e{h, &ph};
    Level& lv = *h->L[from];
    coarse_calls<T>(e, h, from, LvVec<T>::x(lv), LvVec<T>::b(lv));
    DBuf<unsigned char>& d = sub_buf<T>(h);
    d.alloc(ph.size() * sizeof(Phase));
    AMG_CUDA(cudaMemcpyAsync(d.p, ph.data(), ph.size() * sizeof(Phase), cudaMemcpyHostToDevice,
                             h->stream));
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    sub_count<T>(h) = (int)ph.size();
  }

  static void launch(amg_handle* h) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(h->sub_cluster);
    cfg.blockDim = dim3(kSubThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = h->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = h->sub_cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    AMG_CUDA(cudaLaunchKernelEx(&cfg, k_subcycle<T>,
                                reinterpret_cast<const Phase*>(sub_buf<T>(h).p), sub_count<T>(h)));
    h->launches++;
  }
};

template <typename T>
DBuf<unsigned char>& full_buf(amg_handle* h);
template <>
DBuf<unsigned char>& full_buf<float>(amg_handle* h) { return h->full_ph32; }
template <>
DBuf<unsigned char>& full_buf<double>(amg_handle* h) { return h->full_ph64; }
template <typename T>
int& full_count(amg_handle* h);
template <>
int& full_count<float>(amg_handle* h) { return h->full_n32; }
template <>
int& full_count<double>(amg_handle* h) { return h->full_n64; }

// The whole preconditioner application (opt.cycles cycles of Algorithm 1 from
// zero on the level-0 work vectors), recorded for the persistent kernel.
template <typename T>
struct FullCycle {
  static void record(amg_handle* h) {
    std::vector<Phase> ph;
    Emit<T> e{h, &ph};
    Level& lv = *h->L[0];
    const int sub = h->sub_from;
    h->sub_from = 0;   // record every level's operations
    for (int c = 0; c < std::max(1, h->opt.cycles); ++c)
      cycle_rec<T>(e, h, 0, LvVec<T>::x(lv), LvVec<T>::b(lv), c == 0);
    h->sub_from = sub;
    DBuf<unsigned char>& d = full_buf<T>(h);
    d.alloc(ph.size() * sizeof(Phase));
    AMG_CUDA(cudaMemcpyAsync(d.p, ph.data(), ph.size() * sizeof(Phase), cudaMemcpyHostToDevice,
                             h->stream));
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    full_count<T>(h) = (int)ph.size();
  }

  static void launch(amg_handle* h) {
    AMG_CUDA(cudaMemsetAsync(h->grid_bar.p, 0, sizeof(unsigned), h->stream));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(h->grid_ctas);
    cfg.blockDim = dim3(kGridThreads);
    cfg.stream = h->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    AMG_CUDA(cudaLaunchKernelEx(&cfg, k_grid_cycle<T>,
                                reinterpret_cast<const Phase*>(full_buf<T>(h).p),
                                full_count<T>(h), h->grid_bar.p, h->flag.p));
    h->launches++;
  }
};

template <typename T>
int grid_ctas() {
  int dev = 0, sms = 0, per = 0;
  AMG_CUDA(cudaGetDevice(&dev));
  AMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int coop = 0;
  AMG_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_grid_cycle<T>, kGridThreads, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms * std::min(per, 1);
}

template <typename T>
int max_clusters(int size) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(size);
  cfg.blockDim = dim3(kSubThreads);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = size;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (size > 8 &&
      cudaFuncSetAttribute(k_subcycle<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_subcycle<T>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

// ------------------------------------------------------------------- entry points

template <typename T>
void level_apply(amg_handle* h, int l, const T* x, T* y) {
  Emit<T> e{h};
  e_apply<T>(e, *h->L[l], x, y, h->saddle);
}

template <typename T>
void level_residual(amg_handle* h, int l, const T* x, const T* b, T* r) {
  Emit<T> e{h};
  e_residual<T>(e, *h->L[l], x, b, r, h->saddle);
}

template <typename T>
void level_smooth(amg_handle* h, int l, T* x, const T* b, bool post, bool x_is_zero) {
  Emit<T> e{h};
  e_smooth<T>(e, h, *h->L[l], x, b, post, x_is_zero);
}

template <typename T>
void vcycle(amg_handle* h, int l, bool x_is_zero) {
  Emit<T> e{h};
  Level& lv = *h->L[l];
  cycle_rec<T>(e, h, l, LvVec<T>::x(lv), LvVec<T>::b(lv), x_is_zero);
}

// z = M^{-1} r: opt.cycles applications of Algorithm 1 from zero.
template <>
void precondition_device<double>(amg_handle* h, const double* r, double* z) {
  if (h->use_full) {
    Level& lv = *h->L[0];
    launch_copy(r, lv.b64, lv.dofs4(), h->stream, h);
    FullCycle<double>::launch(h);
    launch_copy(lv.x64, z, lv.dofs4(), h->stream, h);
    return;
  }
  Emit<double> e{h};
  for (int c = 0; c < std::max(1, h->opt.cycles); ++c) cycle_rec<double>(e, h, 0, z, r, c == 0);
}

template <>
void precondition_device<float>(amg_handle* h, const double* r, double* z) {
  Level& lv = *h->L[0];
  const int64_t n = lv.dofs4();
  launch_to_float(r, lv.b32, n, h->stream, h);
  if (h->use_full) {
    FullCycle<float>::launch(h);
  } else {
    Emit<float> e{h};
    for (int c = 0; c < std::max(1, h->opt.cycles); ++c)
      cycle_rec<float>(e, h, 0, lv.x32.p, lv.b32.p, c == 0);
  }
  launch_to_double(lv.x32, z, n, h->stream, h);
}

void apply_pair(amg_handle* h, const float* xp, double* y) {
  const Level& lv = *h->L[0];
  if (!lv.val2.p)
    fail(AMG_ERR_INVALID, "the FP32-pair operator needs an FP32 handle with outer_pair");
  switch (lv.group_pair) {
    case 4: launch_apply_pair<4>(lv, xp, y, h->stream); break;
    case 8: launch_apply_pair<8>(lv, xp, y, h->stream); break;
    case 32: launch_apply_pair<32>(lv, xp, y, h->stream); break;
    default: launch_apply_pair<16>(lv, xp, y, h->stream); break;
  }
  h->launches++;
}

// y = K_0 x with the velocity block in FP32-pair arithmetic (x split into xp, 8 floats a
// node, first) and, on saddle levels, B^T p and B u - C p added in FP64
void apply_K_pair(amg_handle* h, const double* x, float* xp, double* y) {
  Level& lv = *h->L[0];
  launch_split_pair(x, xp, 4 * (int64_t)lv.n, h->stream, h);
  apply_pair(h, xp, y);
  if (h->saddle && lv.np > 0) {
    Emit<double> e{h};
    const double* p = x + 4 * lv.n;
    e.bt_add(lv, p, 1.0, y);
    e.prows(0, lv, x, p, nullptr, y + 4 * lv.n, 0.0);
  }
}

void level_transfer(amg_handle* h, int l, bool restrict_, bool f32) {
  Level& lv = *h->L[l];
  Level& nx = *h->L[l + 1];
  if (f32) {
    Emit<float> e{h};
    if (restrict_) e_restrict<float>(e, h, l, lv.r32.p, nx.b32.p);
    else e_prolong<float>(e, h, l, nx.x32.p, lv.x32.p);
  } else {
    Emit<double> e{h};
    if (restrict_) e_restrict<double>(e, h, l, lv.r64.p, nx.b64.p);
    else e_prolong<double>(e, h, l, nx.x64.p, lv.x64.p);
  }
}

void set_subcycle(amg_handle* h, int from) {
  h->sub_from = 0;
  if (from <= 0 || from >= (int)h->L.size() || h->sub_cluster <= 0) return;
  if (h->opt.precision == AMG_FP32) SubCycle<float>::record(h, from);
  else SubCycle<double>::record(h, from);
  h->sub_from = from;
}

// Lanes per block row (4, 8, 16 or 32) of every level, from timing the operator
// kernel and, separately, one colour sweep; then the level from which the cycle
// runs as one cluster launch, from timing whole preconditioner applications.
void autotune_levels(amg_handle* h) {
  cudaStream_t s = h->stream;
  cudaEvent_t e0, e1;
  AMG_CUDA(cudaEventCreate(&e0));
  AMG_CUDA(cudaEventCreate(&e1));
  auto elapsed = [&]() {
    AMG_CUDA(cudaEventRecord(e1, s));
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms;
  };
  const bool f32 = h->opt.precision == AMG_FP32;
  for (size_t l = 0; l < h->L.size(); ++l) {
    Level& lv = *h->L[l];
    lv.gs_cl = 0;
    int best = 0;
    float best_ms = 1e30f;
    for (int G : {4, 8, 16, 32}) {
      lv.group = G;
      for (int r = 0; r < 7; ++r) {
        if (r == 2) AMG_CUDA(cudaEventRecord(e0, s));
        if (f32) level_apply<float>(h, (int)l, lv.x32.p, lv.r32.p);
        else level_apply<double>(h, (int)l, lv.x64.p, lv.r64.p);
      }
      const float ms = elapsed();
      if (ms < best_ms) { best_ms = ms; best = G; }
    }
    lv.group = best;
    if (f32 && l == 0) {   // the outer Krylov operator is FP64 on level 0
      best = 0;
      best_ms = 1e30f;
      for (int G : {4, 8, 16, 32}) {
        lv.group64 = G;
        for (int r = 0; r < 7; ++r) {
          if (r == 2) AMG_CUDA(cudaEventRecord(e0, s));
          level_apply<double>(h, 0, lv.x64.p, lv.r64.p);
        }
        const float ms = elapsed();
        if (ms < best_ms) { best_ms = ms; best = G; }
      }
      lv.group64 = best;
    }
    if (l == 0 && lv.val2.p) {   // the FP32-pair Krylov operator
      DBuf<float> xp;
      xp.alloc(8 * (size_t)lv.n);
      AMG_CUDA(cudaMemsetAsync(xp.p, 0, xp.bytes(), s));
      best = 0;
      best_ms = 1e30f;
      for (int G : {4, 8, 16, 32}) {
        lv.group_pair = G;
        for (int r = 0; r < 7; ++r) {
          if (r == 2) AMG_CUDA(cudaEventRecord(e0, s));
          apply_pair(h, xp.p, lv.r64.p);
        }
        const float ms = elapsed();
        if (ms < best_ms) { best_ms = ms; best = G; }
      }
      lv.group_pair = best;
      AMG_CUDA(cudaStreamSynchronize(s));
    }
    if (lv.ncolours == 0 || h->saddle || h->opt.smoother != AMG_SMOOTHER_GS) continue;
    best = 0;
    best_ms = 1e30f;
    for (int G : {4, 8, 16, 32}) {
      lv.group_gs = G;
      for (int r = 0; r < 3; ++r) {
        if (r == 1) AMG_CUDA(cudaEventRecord(e0, s));
        if (f32) level_smooth<float>(h, (int)l, lv.x32.p, lv.b32.p, false, false);
        else level_smooth<double>(h, (int)l, lv.x64.p, lv.b64.p, false, false);
      }
      const float ms = elapsed();
      if (ms < best_ms) { best_ms = ms; best = G; }
    }
    lv.group_gs = best;
    lv.gs_stream = 0;
    // the colour kernel's x gathers through L1 or L2 only: the faster
    {
      lv.gs_xnc = 0;
      float t_l2 = 0.f, t_l1 = 0.f;
      for (int xnc : {0, 1}) {
        lv.gs_xnc = xnc;
        for (int r = 0; r < 7; ++r) {
          if (r == 2) AMG_CUDA(cudaEventRecord(e0, s));
          if (f32) level_smooth<float>(h, (int)l, lv.x32.p, lv.b32.p, false, false);
          else level_smooth<double>(h, (int)l, lv.x64.p, lv.b64.p, false, false);
        }
        (xnc ? t_l1 : t_l2) = elapsed();
      }
      lv.gs_xnc = t_l1 < t_l2 ? 1 : 0;
    }
    auto sweep_ms = [&]() {
      for (int r = 0; r < 7; ++r) {
        if (r == 2) AMG_CUDA(cudaEventRecord(e0, s));
        if (f32) level_smooth<float>(h, (int)l, lv.x32.p, lv.b32.p, false, false);
        else level_smooth<double>(h, (int)l, lv.x64.p, lv.b64.p, false, false);
      }
      return elapsed();
    };
    // the grid-stride colour kernel (register double buffering, a grid of a few
    // CTAs per SM), for the cycle's precision: kept with its (CTAs per SM, lanes
    // per row) if it beats one group of lanes per row
    if (h->opt.gs_stream > 0) {
      lv.gs_stream = h->opt.gs_stream;
    } else if (h->opt.gs_stream < 0) {
      float t_best = sweep_ms();
      int c_best = 0, g_best = lv.group_gs;
      const int g_keep = lv.group_gs;
      for (int G : {8, 16, 32}) {
        for (int cps : {1, 2, 3, 4}) {
          lv.group_gs = G;
          lv.gs_stream = cps;
          const float t = sweep_ms();
          if (t < t_best) { t_best = t; c_best = cps; g_best = G; }
        }
      }
      lv.gs_stream = c_best;
      lv.group_gs = c_best ? g_best : g_keep;
    }
    // the TMA-staged colour kernel (FP32 values): forced with the chain's lanes per row
    // (gs_tma = 1), else kept with the fastest lanes per row if it beats the chain
    lv.gs_tma = 0;
    if (f32 && !lv.val16.p && lv.gs_stream == 0 && h->opt.gs_tma != 0) {
      if (h->opt.gs_tma > 0) {
        lv.gs_tma = 1;
      } else {
        float t_best = sweep_ms();
        int g_best = 0;
        const int g_keep = lv.group_gs;
        for (int G : {4, 8, 16, 32}) {
          lv.group_gs = G;
          lv.gs_tma = 1;
          const float t = sweep_ms();
          if (t < t_best) { t_best = t; g_best = G; }
        }
        lv.gs_tma = g_best ? 1 : 0;
        lv.group_gs = g_best ? g_best : g_keep;
      }
    }
    // the sweep as one dataflow launch: forced on with the chain's lanes per row
    // (gs_flow = 1), or the fastest lanes per row if it beats the colour chain
    lv.flow = 0;
    if (h->opt.gs_flow != 0 && !(f32 && lv.val16.p) && flow_prepare(h, lv)) {
      if (h->opt.gs_flow > 0) {
        flow_set_group(h, lv, lv.group_gs);
      } else {
        float t_best = sweep_ms();
        int g_best = 0;
        for (int G : {4, 8, 16, 32}) {
          flow_set_group(h, lv, G);
          const float t = sweep_ms();
          if (t < t_best) { t_best = t; g_best = G; }
        }
        if (g_best) flow_set_group(h, lv, g_best);
        else lv.flow = 0;
      }
    }
    // the sweep as one cluster launch with the iterate in shared memory: the
    // forced cluster size, else the fastest (cluster size, lanes per row) if it
    // beats one launch per colour
    const bool elig = f32 ? gs_cluster_eligible<float>(lv) : gs_cluster_eligible<double>(lv);
    if (!elig || h->opt.gs_cluster == 0) continue;
    lv.gs_cl_bytes = f32 ? 4 : 8;
    auto fits = [&](int cs, int G) {
      return f32 ? gs_cluster_fits_level<float>(lv, cs, G)
                 : gs_cluster_fits_level<double>(lv, cs, G);
    };
    auto sweeps_ms = [&]() {
      for (int r = 0; r < 7; ++r) {
        if (r == 2) AMG_CUDA(cudaEventRecord(e0, s));
        if (f32) level_smooth<float>(h, (int)l, lv.x32.p, lv.b32.p, false, false);
        else level_smooth<double>(h, (int)l, lv.x64.p, lv.b64.p, false, false);
      }
      return elapsed();
    };
    if (h->opt.gs_cluster > 0) {
      const int G = lv.group_gs;
      if (fits(h->opt.gs_cluster, G) >= 1) {
        lv.gs_cl = h->opt.gs_cluster;
        lv.gs_cl_g = G;
      }
      continue;
    }
    float t_best = sweeps_ms();
    int cs_best = 0, g_best = 0;
    for (int cs : {1, 2, 4, 8, 16}) {
      for (int G : {8, 16, 32}) {
        if (fits(cs, G) < 1) continue;
        lv.gs_cl = cs;
        lv.gs_cl_g = G;
        const float t = sweeps_ms();
        if (t < t_best) { t_best = t; cs_best = cs; g_best = G; }
      }
    }
    lv.gs_cl = cs_best;
    lv.gs_cl_g = g_best;
  }
  // A one-launch sweep chosen above by timing the sweep alone is kept only if
  // the whole preconditioner application is faster with it: between the
  // per-colour and row kernels of the cycle it can cost more than alone.
  if (h->opt.gs_cluster < 0) {
    DBuf<double> r, z;
    const int64_t n4 = h->L[0]->dofs4();
    r.alloc(n4);
    z.alloc(n4);
    AMG_CUDA(cudaMemsetAsync(r.p, 0, r.bytes(), s));
    auto precond_ms = [&]() {
      for (int rep = 0; rep < 6; ++rep) {
        if (rep == 2) AMG_CUDA(cudaEventRecord(e0, s));
        if (f32) precondition_device<float>(h, r, z);
        else precondition_device<double>(h, r, z);
      }
      return elapsed();
    };
    for (size_t l = 0; l < h->L.size(); ++l) {
      Level& lv = *h->L[l];
      if (lv.gs_cl <= 0) continue;
      const float t_on = precond_ms();
      const int keep = lv.gs_cl;
      lv.gs_cl = 0;
      const float t_off = precond_ms();
      if (t_on < 0.99f * t_off) lv.gs_cl = keep;
    }
  }
  // the same rule for the dataflow sweep, where it runs (no cluster sweep)
  if (h->opt.gs_flow < 0) {
    DBuf<double> r, z;
    const int64_t n4 = h->L[0]->dofs4();
    r.alloc(n4);
    z.alloc(n4);
    AMG_CUDA(cudaMemsetAsync(r.p, 0, r.bytes(), s));
    auto precond_ms = [&]() {
      for (int rep = 0; rep < 6; ++rep) {
        if (rep == 2) AMG_CUDA(cudaEventRecord(e0, s));
        if (f32) precondition_device<float>(h, r, z);
        else precondition_device<double>(h, r, z);
      }
      return elapsed();
    };
    for (size_t l = 0; l < h->L.size(); ++l) {
      Level& lv = *h->L[l];
      if (lv.flow <= 0 || lv.gs_cl > 0) continue;
      const float t_on = precond_ms();
      const int keep = lv.flow;
      lv.flow = 0;
      const float t_off = precond_ms();
      if (t_on < 0.99f * t_off) lv.flow = keep;
    }
  }
  {
    int ferr = 0;
    AMG_CUDA(cudaMemcpy(&ferr, h->flag.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (ferr)
      fail(AMG_ERR_TIMEOUT, "a bounded wait of a one-launch colour sweep (mbarrier or dataflow "
                            "flag) timed out during setup tuning");
  }
  // cluster sub-cycle: the largest cluster that fits (16, else 8 CTAs), then the
  // fastest start level among 1..L (or none)
  const int L = (int)h->L.size() - 1;
  h->sub_cluster = 0;
  if (L >= 1 && h->opt.cluster_from != 0) {
    for (int size : {16, 8}) {
      const int n = f32 ? max_clusters<float>(size) : max_clusters<double>(size);
      if (n >= 1) { h->sub_cluster = size; break; }
    }
  }
  if (h->sub_cluster > 0 && h->opt.cluster_from >= 0) {
    set_subcycle(h, std::min(h->opt.cluster_from, L));
  } else if (h->sub_cluster > 0) {
    DBuf<double> r, z;
    const int64_t n4 = h->L[0]->dofs4();
    r.alloc(n4);
    z.alloc(n4);
    AMG_CUDA(cudaMemsetAsync(r.p, 0, r.bytes(), s));
    int best_from = 0;
    float best_ms = 1e30f;
    for (int from = 0; from <= L; ++from) {
      set_subcycle(h, from);
      for (int rep = 0; rep < 5; ++rep) {
        if (rep == 2) AMG_CUDA(cudaEventRecord(e0, s));
        if (f32) precondition_device<float>(h, r, z);
        else precondition_device<double>(h, r, z);
      }
      const float ms = elapsed();
      if (ms < best_ms * 0.98f) { best_ms = ms; best_from = from; }
    }
    set_subcycle(h, best_from);
  }
  // the whole cycle as one persistent cooperative launch, if it is faster
  h->use_full = false;
  h->grid_ctas = (h->opt.cycle_kernel != 1) ? (f32 ? grid_ctas<float>() : grid_ctas<double>()) : 0;
  if (h->grid_ctas > 0) {
    if (!h->grid_bar.p) h->grid_bar.alloc(1);
    if (f32) FullCycle<float>::record(h);
    else FullCycle<double>::record(h);
    if (h->opt.cycle_kernel == 2) {
      h->use_full = true;
    } else {
      DBuf<double> r, z;
      const int64_t n4 = h->L[0]->dofs4();
      r.alloc(n4);
      z.alloc(n4);
      AMG_CUDA(cudaMemsetAsync(r.p, 0, r.bytes(), s));
      float t[2];
      for (int mode = 0; mode < 2; ++mode) {
        h->use_full = mode == 1;
        for (int rep = 0; rep < 5; ++rep) {
          if (rep == 2) AMG_CUDA(cudaEventRecord(e0, s));
          if (f32) precondition_device<float>(h, r, z);
          else precondition_device<double>(h, r, z);
        }
        t[mode] = elapsed();
      }
      h->use_full = t[1] < t[0];
    }
    int ferr = 0;
    AMG_CUDA(cudaMemcpy(&ferr, h->flag.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (ferr) fail(AMG_ERR_TIMEOUT, "grid barrier of the persistent cycle kernel timed out");
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

template void level_apply<double>(amg_handle*, int, const double*, double*);
template void level_apply<float>(amg_handle*, int, const float*, float*);
template void level_residual<double>(amg_handle*, int, const double*, const double*, double*);
template void level_residual<float>(amg_handle*, int, const float*, const float*, float*);
template void level_smooth<double>(amg_handle*, int, double*, const double*, bool, bool);
template void level_smooth<float>(amg_handle*, int, float*, const float*, bool, bool);
template void vcycle<double>(amg_handle*, int, bool);
template void vcycle<float>(amg_handle*, int, bool);

}  // namespace amgp2
