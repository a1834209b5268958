// The AMG cycle of Algorithm 1 on the GPU: 3x3-block row kernels (operator
// application, residual, multicolour block Gauss-Seidel, damped block Jacobi),
// transfers P / R = P^T, the dense coarsest solve, and the saddle-point
// segregated Gauss-Seidel sweep of Eq. (uzsm).
#include <algorithm>

#include "amg_internal.cuh"
#include "vec.cuh"

namespace amgp2 {

namespace {

enum RowMode { kApply = 0, kResid = 1, kGS = 2, kJacobi = 3 };

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// One group of G lanes per block row.  Each lane walks the row's blocks with
// stride G; block values come from the 9 planes (consecutive lanes read
// consecutive addresses of each plane), x_j is one vector load of the padded
// node; the three partial sums are reduced with shuffles inside the group.
//   kApply : y_i = (A x)_i
//   kResid : y_i = b_i - (A x)_i
//   kGS    : x_i += D_i^{-1} (b_i - (A x)_i)   for the rows listed in `rows`
//   kJacobi: y_i = x_i + omega D_i^{-1} (b_i - (A x)_i)
// D^{-1} is stored as 3 padded rows per node (12 values).
template <typename T, int G, int MODE>
__global__ void __launch_bounds__(256) k_block_rows(
    int nrows, const int* __restrict__ rows, const int* __restrict__ rowptr,
    const int* __restrict__ col, const T* __restrict__ val, int64_t nnzb, const T* x,
    const T* __restrict__ b, T* y, const T* __restrict__ dinv, T omega) {
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int lane = threadIdx.x & (G - 1);
  const bool active = g < nrows;
  int i = 0;
  T s0 = T(0), s1 = T(0), s2 = T(0);
  if (active) {
    i = rows ? ldg(rows + g) : g;
    const int a = ldg(rowptr + i), e = ldg(rowptr + i + 1);
    for (int k = a + lane; k < e; k += G) {
      const int j = ldg(col + k);
      T x0, x1, x2;
      ld3(x, j, x0, x1, x2);
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
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (!active || lane != 0) return;
  if (MODE == kApply) {
    st3(y, i, s0, s1, s2);
    return;
  }
  T b0, b1, b2;
  ld3(b, i, b0, b1, b2);
  const T r0 = b0 - s0, r1 = b1 - s1, r2 = b2 - s2;
  if (MODE == kResid) {
    st3(y, i, r0, r1, r2);
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
  ld3(x, i, x0, x1, x2);
  if (MODE == kGS) {
    st3(y, i, x0 + c0, x1 + c1, x2 + c2);
  } else {
    st3(y, i, x0 + omega * c0, x1 + omega * c1, x2 + omega * c2);
  }
}

// R = P^T gather: bc_I = sum_t w_t r_{i_t} (3 components, same weight)
template <typename T>
__global__ void k_restrict(int nc, const int* __restrict__ rrow, const int* __restrict__ rcol,
                           const T* __restrict__ rval, const T* __restrict__ r, T* __restrict__ bc) {
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int t = rrow[I]; t < rrow[I + 1]; ++t) {
      const int i = rcol[t];
      const T w = rval[t];
      T r0, r1, r2;
      ld3(r, i, r0, r1, r2);
      s0 = fma(w, r0, s0);
      s1 = fma(w, r1, s1);
      s2 = fma(w, r2, s2);
    }
    st3(bc, I, s0, s1, s2);
  }
}

// x_i += sum_q P_iq xc_q
template <typename T>
__global__ void k_prolong(int n, const int* __restrict__ prow, const int* __restrict__ pcol,
                          const T* __restrict__ pval, const T* __restrict__ xc, T* __restrict__ x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int q = prow[i]; q < prow[i + 1]; ++q) {
      const int J = pcol[q];
      const T w = pval[q];
      T c0, c1, c2;
      ld3(xc, J, c0, c1, c2);
      s0 = fma(w, c0, s0);
      s1 = fma(w, c1, s1);
      s2 = fma(w, c2, s2);
    }
    T x0, x1, x2;
    ld3(x, i, x0, x1, x2);
    st3(x, i, x0 + s0, x1 + s1, x2 + s2);
  }
}

// scalar versions for the pressure (H, H^T)
template <typename T>
__global__ void k_restrict1(int nc, const int* __restrict__ rrow, const int* __restrict__ rcol,
                            const T* __restrict__ rval, const T* __restrict__ r, T* __restrict__ bc) {
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
    T s = T(0);
    for (int t = rrow[I]; t < rrow[I + 1]; ++t) s = fma(rval[t], r[rcol[t]], s);
    bc[I] = s;
  }
}

template <typename T>
__global__ void k_prolong1(int n, const int* __restrict__ prow, const int* __restrict__ pcol,
                           const T* __restrict__ pval, const T* __restrict__ xc, T* __restrict__ x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    T s = T(0);
    for (int q = prow[i]; q < prow[i + 1]; ++q) s = fma(pval[q], xc[pcol[q]], s);
    x[i] += s;
  }
}

// x = X b with the FP64 generalised inverse of the coarsest matrix (warp per row).
// X is indexed in the unpadded order (3 per node, then pressure); n3 = 3 n.
__device__ __forceinline__ int pad_index(int j, int n3) {
  return j < n3 ? 4 * (j / 3) + j % 3 : j + n3 / 3;
}

template <typename T>
__global__ void k_coarse_solve(int m, int n3, const double* __restrict__ X,
                               const T* __restrict__ b, T* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = w; i < m; i += nw) {
    double s = 0.0;
    for (int j = lane; j < m; j += 32)
      s = fma(X[(int64_t)i * m + j], (double)b[pad_index(j, n3)], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[pad_index(i, n3)] = (T)s;
  }
}

template <typename T>
__global__ void k_zero(T* a, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    a[k] = T(0);
}

template <typename T>
__global__ void k_copyT(const T* __restrict__ a, T* __restrict__ b, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = a[k];
}

// ---- saddle-point parts: y_u (+)= B^T p per velocity node, y_p = B u - C p ---------

// yu_i += sum_k B_ki^T p_k (rows of B^T are velocity nodes)
template <typename T>
__global__ void k_bt_add(int n, const int* __restrict__ row, const int* __restrict__ col,
                         const T* __restrict__ val, int64_t nnz, const T* __restrict__ p,
                         T sign, T* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int q = row[i]; q < row[i + 1]; ++q) {
      const T pk = p[col[q]];
      s0 = fma(val[q], pk, s0);
      s1 = fma(val[nnz + q], pk, s1);
      s2 = fma(val[2 * nnz + q], pk, s2);
    }
    T y0, y1, y2;
    ld3(y, i, y0, y1, y2);
    st3(y, i, y0 + sign * s0, y1 + sign * s1, y2 + sign * s2);
  }
}

// MODE 0: yp = B u - C p;  MODE 1: yp = g - B u + C p (residual);
// MODE 2: p += omega * (B u - C p - g) / S_D (sGS pressure step, in place)
template <typename T, int MODE>
__global__ void k_pressure_rows(int np, const int* __restrict__ brow, const int* __restrict__ bcol,
                                const T* __restrict__ bval, int64_t bnnz,
                                const int* __restrict__ crow, const int* __restrict__ ccol,
                                const T* __restrict__ cval, const T* __restrict__ u,
                                const T* p, const T* __restrict__ g, T* yp,
                                const T* __restrict__ sd, T omega) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
    T s = T(0);
    for (int q = brow[k]; q < brow[k + 1]; ++q) {
      const int j = bcol[q];
      T u0, u1, u2;
      ld3(u, j, u0, u1, u2);
      s = fma(bval[q], u0, s);
      s = fma(bval[bnnz + q], u1, s);
      s = fma(bval[2 * bnnz + q], u2, s);
    }
    T cp = T(0);
    for (int q = crow[k]; q < crow[k + 1]; ++q) cp = fma(cval[q], p[ccol[q]], cp);
    if (MODE == 0) {
      yp[k] = s - cp;
    } else if (MODE == 1) {
      yp[k] = g[k] - s + cp;
    } else {
      const T d = sd[k];
      const T r = s - cp - g[k];
      yp[k] = p[k] + (d != T(0) ? omega * r / d : T(0));
    }
  }
}

template <typename T> struct LvVec;
template <> struct LvVec<double> {
  static double* x(Level& l) { return l.x64; }
  static double* b(Level& l) { return l.b64; }
  static double* r(Level& l) { return l.r64; }
  static double* t(Level& l) { return l.t64; }
  static const double* val(Level& l) { return l.val; }
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

inline int gridn(int64_t n, int t = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 152 * 16));
}

// lanes per block row: the autotuned value, else from the average row length
inline int group_for(const Level& lv) {
  if (lv.group) return lv.group;
  if (lv.avg_row_blocks > 20.0) return 32;
  if (lv.avg_row_blocks > 10.0) return 16;
  if (lv.avg_row_blocks > 5.0) return 8;
  return 4;
}

template <typename T, int MODE>
void launch_rows_g(int G, cudaStream_t s, int nrows, const int* rows, const Level& lv,
                   const T* val, const T* x, const T* b, T* y, const T* dinv, T omega) {
  if (nrows <= 0) return;
  int64_t threads = (int64_t)nrows * G;
  int grid = (int)((threads + 255) / 256);
#define AMG_ROWS_CASE(GG)                                                                   \
  case GG:                                                                                  \
    k_block_rows<T, GG, MODE><<<grid, 256, 0, s>>>(nrows, rows, lv.rowptr, lv.col, val,      \
                                                   lv.nnzb, x, b, y, dinv, omega);          \
    break;
  switch (G) {
    AMG_ROWS_CASE(4)
    AMG_ROWS_CASE(8)
    AMG_ROWS_CASE(16)
    default:
    AMG_ROWS_CASE(32)
  }
#undef AMG_ROWS_CASE
}

}  // namespace

// y = K_l x (saddle: [A B^T; B -C])
template <typename T>
void level_apply(amg_handle* h, int l, const T* x, T* y) {
  Level& lv = *h->L[l];
  cudaStream_t s = h->stream;
  launch_rows_g<T, kApply>(group_for(lv), s, lv.n, nullptr, lv, LvVec<T>::val(lv), x, nullptr, y,
                           nullptr, T(0));
  h->launches++;
  if (h->saddle && lv.np > 0) {
    const T* p = x + 4 * lv.n;
    k_bt_add<T><<<gridn(lv.n), 256, 0, s>>>(lv.n, lv.bt_rowptr, lv.bt_col, LvVec<T>::btval(lv),
                                            lv.b_nnz, p, T(1), y);
    k_pressure_rows<T, 0><<<gridn(lv.np), 256, 0, s>>>(
        lv.np, lv.b_rowptr, lv.b_col, LvVec<T>::bval(lv), lv.b_nnz, lv.c_rowptr, lv.c_col,
        LvVec<T>::cval(lv), x, p, nullptr, y + 4 * lv.n, nullptr, T(0));
    h->launches += 2;
  }
}

template <typename T>
void level_residual(amg_handle* h, int l, const T* x, const T* b, T* r) {
  Level& lv = *h->L[l];
  cudaStream_t s = h->stream;
  launch_rows_g<T, kResid>(group_for(lv), s, lv.n, nullptr, lv, LvVec<T>::val(lv), x, b, r,
                           nullptr, T(0));
  h->launches++;
  if (h->saddle && lv.np > 0) {
    const T* p = x + 4 * lv.n;
    k_bt_add<T><<<gridn(lv.n), 256, 0, s>>>(lv.n, lv.bt_rowptr, lv.bt_col, LvVec<T>::btval(lv),
                                            lv.b_nnz, p, T(-1), r);
    k_pressure_rows<T, 1><<<gridn(lv.np), 256, 0, s>>>(
        lv.np, lv.b_rowptr, lv.b_col, LvVec<T>::bval(lv), lv.b_nnz, lv.c_rowptr, lv.c_col,
        LvVec<T>::cval(lv), x, p, b + 4 * lv.n, r + 4 * lv.n, nullptr, T(0));
    h->launches += 2;
  }
}

// One smoothing sweep (Sec. 3.3).  SPD: symmetric multicolour block GS (colours
// ascending before the coarse correction, descending after it) or damped block
// Jacobi.  Saddle: segregated Gauss-Seidel, Eq. (uzsm).
template <typename T>
void level_smooth(amg_handle* h, int l, T* x, const T* b, bool post, bool x_is_zero) {
  Level& lv = *h->L[l];
  cudaStream_t s = h->stream;
  const int dofs = lv.dofs4();
  if (x_is_zero) {
    k_zero<T><<<gridn(dofs), 256, 0, s>>>(x, dofs);
    h->launches++;
  }
  const int G = group_for(lv);
  const T* val = LvVec<T>::val(lv);
  const T* dinv = LvVec<T>::dinv(lv);
  if (h->saddle) {
    // u <- u + omega D^{-1} (f - A u - B^T p)   (M_A = damped block Jacobi)
    T* t = LvVec<T>::t(lv);
    T* r = LvVec<T>::r(lv);
    const T* p = x + 4 * lv.n;
    // r_u = f - B^T p, then t_u = u + omega D^{-1} (r_u - A u)
    k_copyT<T><<<gridn(4 * lv.n), 256, 0, s>>>(b, r, 4 * (int64_t)lv.n);
    k_bt_add<T><<<gridn(lv.n), 256, 0, s>>>(lv.n, lv.bt_rowptr, lv.bt_col, LvVec<T>::btval(lv),
                                            lv.b_nnz, p, T(-1), r);
    launch_rows_g<T, kJacobi>(G, s, lv.n, nullptr, lv, val, x, r, t, dinv, (T)h->opt.omega);
    k_copyT<T><<<gridn(4 * lv.n), 256, 0, s>>>(t, x, 4 * (int64_t)lv.n);
    // p <- p + omega_p S_D^{-1} (B u_new - C p - g)
    k_pressure_rows<T, 2><<<gridn(lv.np), 256, 0, s>>>(
        lv.np, lv.b_rowptr, lv.b_col, LvVec<T>::bval(lv), lv.b_nnz, lv.c_rowptr, lv.c_col,
        LvVec<T>::cval(lv), x, x + 4 * lv.n, b + 4 * lv.n, t + 4 * lv.n, LvVec<T>::schur(lv),
        (T)h->opt.omega_p);
    k_copyT<T><<<gridn(lv.np), 256, 0, s>>>(t + 4 * lv.n, x + 4 * lv.n, lv.np);
    h->launches += 6;
    return;
  }
  if (h->opt.smoother == AMG_SMOOTHER_JACOBI) {
    T* t = LvVec<T>::t(lv);
    launch_rows_g<T, kJacobi>(G, s, lv.n, nullptr, lv, val, x, b, t, dinv, (T)h->opt.omega);
    k_copyT<T><<<gridn(dofs), 256, 0, s>>>(t, x, dofs);
    h->launches += 2;
    return;
  }
  const int Ggs = lv.group_gs ? lv.group_gs : G;
  for (int q = 0; q < lv.ncolours; ++q) {
    const int c = post ? lv.ncolours - 1 - q : q;
    const int a = lv.colour_ptr[c], e = lv.colour_ptr[c + 1];
    launch_rows_g<T, kGS>(Ggs, s, e - a, lv.colour_rows.p + a, lv, val, x, b, x, dinv, T(0));
    h->launches++;
  }
}

template <typename T>
static void coarse_solve(amg_handle* h, const T* b, T* x) {
  const int m = h->coarse_m;
  const int n3 = 3 * h->L.back()->n;
  k_coarse_solve<T><<<gridn((int64_t)m * 32), 256, 0, h->stream>>>(m, n3, h->coarse_inv, b, x);
  h->launches++;
}

template <typename T>
static void restrict_to(amg_handle* h, int l, const T* r, T* bc) {
  Level& lv = *h->L[l];
  Level& nx = *h->L[l + 1];
  cudaStream_t s = h->stream;
  k_restrict<T><<<gridn(nx.n), 256, 0, s>>>(nx.n, lv.r_rowptr, lv.r_col, LvVec<T>::rval(lv), r, bc);
  h->launches++;
  if (h->saddle && nx.np > 0) {
    k_restrict1<T><<<gridn(nx.np), 256, 0, s>>>(nx.np, lv.ht_rowptr, lv.ht_col,
                                                 LvVec<T>::htval(lv), r + 4 * lv.n, bc + 4 * nx.n);
    h->launches++;
  }
}

template <typename T>
static void prolong_add(amg_handle* h, int l, const T* xc, T* x) {
  Level& lv = *h->L[l];
  Level& nx = *h->L[l + 1];
  cudaStream_t s = h->stream;
  k_prolong<T><<<gridn(lv.n), 256, 0, s>>>(lv.n, lv.p_rowptr, lv.p_col, LvVec<T>::pval(lv), xc, x);
  h->launches++;
  if (h->saddle && lv.np > 0) {
    k_prolong1<T><<<gridn(lv.np), 256, 0, s>>>(lv.np, lv.h_rowptr, lv.h_col, LvVec<T>::hval(lv),
                                               xc + 4 * nx.n, x + 4 * lv.n);
    h->launches++;
  }
}

// Algorithm 1 on level l with iterate x and right-hand side b.
template <typename T>
static void cycle_rec(amg_handle* h, int l, T* x, const T* b, bool x_is_zero) {
  const int L = (int)h->L.size() - 1;
  if (l == L) {
    coarse_solve<T>(h, b, x);
    return;
  }
  Level& lv = *h->L[l];
  Level& nx = *h->L[l + 1];
  const amg_options& o = h->opt;
  bool zero = x_is_zero;
  for (int k = 0; k < o.m_pre; ++k) {
    level_smooth<T>(h, l, x, b, false, zero);
    zero = false;
  }
  if (zero) {   // no pre-smoothing: x is still the zero initial guess
    k_zero<T><<<gridn(lv.dofs4()), 256, 0, h->stream>>>(x, lv.dofs4());
    h->launches++;
  }
  T* r = LvVec<T>::r(lv);
  level_residual<T>(h, l, x, b, r);
  T* bc = LvVec<T>::b(nx);
  T* xc = LvVec<T>::x(nx);
  restrict_to<T>(h, l, r, bc);
  if (l + 1 == L) {
    coarse_solve<T>(h, bc, xc);
  } else {
    for (int k = 0; k < std::max(1, o.nu); ++k) cycle_rec<T>(h, l + 1, xc, bc, k == 0);
  }
  prolong_add<T>(h, l, xc, x);
  for (int k = 0; k < o.m_post; ++k) level_smooth<T>(h, l, x, b, true, false);
}

template <typename T>
void vcycle(amg_handle* h, int l, bool x_is_zero) {
  Level& lv = *h->L[l];
  cycle_rec<T>(h, l, LvVec<T>::x(lv), LvVec<T>::b(lv), x_is_zero);
}

// z = M^{-1} r: opt.cycles applications of Algorithm 1 from zero.
template <>
void precondition_device<double>(amg_handle* h, const double* r, double* z) {
  for (int c = 0; c < std::max(1, h->opt.cycles); ++c) cycle_rec<double>(h, 0, z, r, c == 0);
}

template <>
void precondition_device<float>(amg_handle* h, const double* r, double* z) {
  Level& lv = *h->L[0];
  const int64_t n = lv.dofs4();
  launch_to_float(r, lv.b32, n, h->stream, h);
  for (int c = 0; c < std::max(1, h->opt.cycles); ++c)
    cycle_rec<float>(h, 0, lv.x32.p, lv.b32.p, c == 0);
  launch_to_double(lv.x32, z, n, h->stream, h);
}

void level_transfer(amg_handle* h, int l, bool restrict_, bool f32) {
  Level& lv = *h->L[l];
  Level& nx = *h->L[l + 1];
  if (f32) {
    if (restrict_) restrict_to<float>(h, l, lv.r32.p, nx.b32.p);
    else prolong_add<float>(h, l, nx.x32.p, lv.x32.p);
  } else {
    if (restrict_) restrict_to<double>(h, l, lv.r64.p, nx.b64.p);
    else prolong_add<double>(h, l, nx.x64.p, lv.x64.p);
  }
}

// Times the operator kernel of every level with 4, 8, 16 and 32 lanes per block
// row (in the precision the cycle uses) and keeps the fastest.  The row kernels
// of one level share its access pattern, so one choice serves all modes.
void autotune_levels(amg_handle* h) {
  cudaStream_t s = h->stream;
  cudaEvent_t e0, e1;
  AMG_CUDA(cudaEventCreate(&e0));
  AMG_CUDA(cudaEventCreate(&e1));
  const bool f32 = h->opt.precision == AMG_FP32;
  for (auto& lp : h->L) {
    Level& lv = *lp;
    int best = 0;
    float best_ms = 1e30f;
    for (int G : {4, 8, 16, 32}) {
      const int reps = 5;
      for (int r = 0; r < reps + 2; ++r) {
        if (r == 2) AMG_CUDA(cudaEventRecord(e0, s));
        if (f32)
          launch_rows_g<float, kApply>(G, s, lv.n, nullptr, lv, lv.val32.p, lv.x32.p, nullptr,
                                       lv.r32.p, nullptr, 0.f);
        else
          launch_rows_g<double, kApply>(G, s, lv.n, nullptr, lv, lv.val.p, lv.x64.p, nullptr,
                                        lv.r64.p, nullptr, 0.0);
      }
      AMG_CUDA(cudaEventRecord(e1, s));
      AMG_LAUNCH_CHECK();
      AMG_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      h->launches += reps + 2;
      if (ms < best_ms) { best_ms = ms; best = G; }
    }
    lv.group = best;
    if (lv.ncolours == 0 || h->saddle || h->opt.smoother != AMG_SMOOTHER_GS) continue;
    // one full colour sweep per candidate
    best = 0;
    best_ms = 1e30f;
    for (int G : {4, 8, 16, 32}) {
      lv.group_gs = G;
      for (int r = 0; r < 3; ++r) {
        if (r == 1) AMG_CUDA(cudaEventRecord(e0, s));
        if (f32) level_smooth<float>(h, (int)(&lp - &h->L[0]), lv.x32.p, lv.b32.p, false, false);
        else level_smooth<double>(h, (int)(&lp - &h->L[0]), lv.x64.p, lv.b64.p, false, false);
      }
      AMG_CUDA(cudaEventRecord(e1, s));
      AMG_LAUNCH_CHECK();
      AMG_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) { best_ms = ms; best = G; }
    }
    lv.group_gs = best;
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
