// AMG setup phase on the GPU (Sec. 3.2 of the paper):
//   coarsening graphs -> greedy independent set (C/F split) -> prolongation
//   (Eqs. disprolongmat / mixprolongmat) -> Galerkin product P^T K P ->
//   colouring + 3x3 diagonal-block inverses -> coarsest factorisation.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>

#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "amg_internal.cuh"

namespace amgp2 {

// ============================================================================ scan

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ int block_exclusive_scan(int v, int* sh) {
  // warp inclusive scan
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < (blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  int base = wid ? sh[wid - 1] : 0;
  int total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  sh[32] = total;
  return base + x - v;
}

__global__ void k_scan_tiles(const int* __restrict__ in, int* __restrict__ out, int n,
                             int* __restrict__ tile_sums) {
  __shared__ int sh[33];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int ex = block_exclusive_scan(s, sh);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = sh[32];
}

__global__ void k_scan_sums(int* sums, int ntiles, long long* total) {
  // one block: sequential over chunks of blockDim
  __shared__ int sh[33];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int c = 0; c < ntiles; c += blockDim.x) {
    int i = c + threadIdx.x;
    int v = i < ntiles ? sums[i] : 0;
    int ex = block_exclusive_scan(v, sh);
    if (i < ntiles) sums[i] = (int)(carry + ex);
    __syncthreads();
    if (threadIdx.x == 0) carry += sh[32];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int* out, int n, const int* sums, const long long* total) {
  int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  int add = sums[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k, i += kScanThreads)
    if (i < n) out[i] += add;
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (int)*total;
}

}  // namespace

int64_t exclusive_scan(const int* in, int* out, int n, cudaStream_t s, amg_handle* h) {
  int ntiles = std::max(1, div_up(n, kScanTile));
  DBuf<int> sums;
  sums.alloc(ntiles);
  DBuf<long long> total;
  total.alloc(1);
  k_scan_tiles<<<ntiles, kScanThreads, 0, s>>>(in, out, n, sums);
  k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, ntiles, total);
  k_scan_add<<<ntiles, kScanThreads, 0, s>>>(out, n, sums, total);
  AMG_LAUNCH_CHECK();
  h->launches += 3;
  long long t = 0;
  AMG_CUDA(cudaMemcpyAsync(&t, total.p, sizeof(t), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  if (t > INT32_MAX) fail(AMG_ERR_UNSUPPORTED, "index range exceeds int32");
  return t;
}

// ============================================================================ small kernels

namespace {

__global__ void k_aos9_to_planes(const double* __restrict__ aos, double* __restrict__ planes,
                                 int64_t nnzb) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnzb;
       k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int e = 0; e < 9; ++e) planes[e * nnzb + k] = aos[9 * k + e];
  }
}

__global__ void k_aos3_to_planes(const double* __restrict__ aos, double* __restrict__ planes,
                                 int64_t nnz) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int e = 0; e < 3; ++e) planes[e * nnz + k] = aos[3 * k + e];
  }
}

// FP64 -> BF16 bit patterns, rounded to nearest even
__global__ void k_to_bf16(const double* __restrict__ a, unsigned short* __restrict__ b,
                          int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = __bfloat16_as_ushort(__double2bfloat16(a[k]));
}

// FP64 -> (hi, lo) float pairs: hi = fl32(a), lo = fl32(a - hi); hi + lo equals
// a to about 2^-48 relative (a - hi is exact in FP64)
__global__ void k_split_pair(const double* __restrict__ a, float2* __restrict__ b, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double v = a[k];
    const float hi = (float)v;
    b[k] = make_float2(hi, (float)(v - (double)hi));
  }
}

// a padded FP64 vector (4 entries a node) -> 8 floats a node: the hi parts of
// the node's 4 entries, then the lo parts
__global__ void k_split_vec(const double* __restrict__ x, float* __restrict__ xp, int64_t n4) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n4;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[k];
    const float hi = (float)v;
    const int64_t o = 8 * (k >> 2) + (k & 3);
    xp[o] = hi;
    xp[o + 4] = (float)(v - (double)hi);
  }
}

__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = (float)a[k];
}

__global__ void k_f2d(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = (double)a[k];
}

__global__ void k_copy(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = a[k];
}

__global__ void k_fill(double* a, double v, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    a[k] = v;
}

// Structural checks of a block-CSR matrix: rowptr monotone, columns in range and
// strictly ascending, diagonal block present (square case), values finite.
__global__ void k_check_csr(int nrows, int ncols, const int* __restrict__ rowptr,
                            const int* __restrict__ col, const double* __restrict__ val,
                            int64_t nval_per_row_entry, int64_t nnz, int need_diag,
                            int* __restrict__ flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += gridDim.x * blockDim.x) {
    int a = rowptr[i], b = rowptr[i + 1];
    if (b < a || a < 0 || b > nnz) { atomicOr(flag, 1); continue; }
    bool diag = false;
    for (int k = a; k < b; ++k) {
      int j = col[k];
      if (j < 0 || j >= ncols) { atomicOr(flag, 2); break; }
      if (k > a && j <= col[k - 1]) { atomicOr(flag, 4); break; }
      if (j == i) diag = true;
      for (int e = 0; e < nval_per_row_entry; ++e)
        if (!isfinite(val[e * nnz + k])) atomicOr(flag, 8);
    }
    if (need_diag && !diag) atomicOr(flag, 16);
  }
}

}  // namespace

static inline int grid_for(int64_t n, int threads = 256) {
  int64_t g = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

namespace {
__global__ void k_to_padded(const double* __restrict__ u, double* __restrict__ p, int n, int np) {
  const int64_t tot = 4 * (int64_t)n + np;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < tot;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (k < 4 * (int64_t)n) {
      const int64_t node = k >> 2, c = k & 3;
      p[k] = c < 3 ? u[3 * node + c] : 0.0;
    } else {
      p[k] = u[k - n];
    }
  }
}
__global__ void k_from_padded(const double* __restrict__ p, double* __restrict__ u, int n, int np) {
  const int64_t tot = 3 * (int64_t)n + np;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < tot;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (k < 3 * (int64_t)n) u[k] = p[4 * (k / 3) + k % 3];
    else u[k] = p[k + n];
  }
}
}  // namespace

void launch_to_padded(const double* u, double* p, int n, int np, cudaStream_t s, amg_handle* h) {
  k_to_padded<<<grid_for(4 * (int64_t)n + np), 256, 0, s>>>(u, p, n, np);
  h->launches++;
}
void launch_from_padded(const double* p, double* u, int n, int np, cudaStream_t s, amg_handle* h) {
  k_from_padded<<<grid_for(3 * (int64_t)n + np), 256, 0, s>>>(p, u, n, np);
  h->launches++;
}

void launch_copy(const double* a, double* b, int64_t n, cudaStream_t s, amg_handle* h) {
  if (n <= 0) return;
  k_copy<<<grid_for(n), 256, 0, s>>>(a, b, n);
  h->launches++;
}
void launch_to_float(const double* a, float* b, int64_t n, cudaStream_t s, amg_handle* h) {
  if (n <= 0) return;
  k_d2f<<<grid_for(n), 256, 0, s>>>(a, b, n);
  h->launches++;
}
void launch_split_pair(const double* x, float* xp, int64_t n4, cudaStream_t s, amg_handle* h) {
  if (n4 <= 0) return;
  k_split_vec<<<grid_for(n4), 256, 0, s>>>(x, xp, n4);
  h->launches++;
}
void launch_to_double(const float* a, double* b, int64_t n, cudaStream_t s, amg_handle* h) {
  if (n <= 0) return;
  k_f2d<<<grid_for(n), 256, 0, s>>>(a, b, n);
  h->launches++;
}
void launch_fill(double* a, double v, int64_t n, cudaStream_t s, amg_handle* h) {
  if (n <= 0) return;
  k_fill<<<grid_for(n), 256, 0, s>>>(a, v, n);
  h->launches++;
}

// ============================================================================ C/F splitting

namespace {

constexpr int kUndecided = 0, kC = 1, kF = 2;

// One round of the greedy independent set in increasing index order.  A node is
// C iff none of its lower-index neighbours (in the coarsening graph) is C, so it
// is decided as soon as a lower neighbour is C (-> F) or all lower neighbours
// are F (-> C).  States only move from undecided to final, so reading values
// written earlier in the same round is safe and speeds up propagation.
__global__ void k_mis_round(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                            const int* __restrict__ tags, int separate, int* state,
                            int* remaining) {
  volatile int* vs = state;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (vs[i] != kUndecided) continue;
    int ti = tags ? (tags[i] & 0xF) : 0;
    bool all_f = true, any_c = false;
    for (int k = rowptr[i], e = rowptr[i + 1]; k < e; ++k) {
      int j = col[k];
      if (j >= i) break;
      if (separate && tags && (tags[j] & 0xF) != ti) continue;
      int sj = vs[j];
      if (sj == kC) { any_c = true; break; }
      if (sj == kUndecided) all_f = false;
    }
    if (any_c) vs[i] = kF;
    else if (all_f) vs[i] = kC;
    else atomicAdd(remaining, 1);
  }
}

__global__ void k_is_c(int n, const int* __restrict__ state, int* __restrict__ flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    flag[i] = state[i] == kC ? 1 : 0;
}

__global__ void k_cid(int n, const int* __restrict__ state, int* __restrict__ cid) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (state[i] != kC) cid[i] = -1;
}

// Number of prolongation entries of each fine row: 1 for C, k (its C neighbours
// of the same type) for F.
__global__ void k_p_count(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                          const int* __restrict__ tags, int separate,
                          const int* __restrict__ state, int* __restrict__ count,
                          int* __restrict__ flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (state[i] == kC) { count[i] = 1; continue; }
    int ti = tags ? (tags[i] & 0xF) : 0;
    int k = 0;
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      int j = col[q];
      if (j == i) continue;
      if (separate && tags && (tags[j] & 0xF) != ti) continue;
      if (state[j] == kC) ++k;
    }
    if (k == 0) atomicOr(flag, 32);   // not maximal: cannot happen after the rounds
    count[i] = k;
  }
}

// Prolongation rows: C -> weight 1 on its own coarse id; F -> 1/k on each of its
// k C-neighbours (ascending, which is ascending coarse id).  Entries in rows of
// Dirichlet fine nodes and in columns of Dirichlet coarse nodes are zero.
__global__ void k_p_fill(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                         const int* __restrict__ tags, int separate,
                         const int* __restrict__ state, const int* __restrict__ cid,
                         const int* __restrict__ p_rowptr, int* __restrict__ p_col,
                         double* __restrict__ p_val) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    bool di = tags ? (tags[i] & AMG_NODE_DIRICHLET) != 0 : false;
    int o = p_rowptr[i];
    if (state[i] == kC) {
      p_col[o] = cid[i];
      p_val[o] = di ? 0.0 : 1.0;
      continue;
    }
    int k = p_rowptr[i + 1] - o;
    double w = 1.0 / (double)k;
    int ti = tags ? (tags[i] & 0xF) : 0;
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      int j = col[q];
      if (j == i) continue;
      if (separate && tags && (tags[j] & 0xF) != ti) continue;
      if (state[j] != kC) continue;
      bool dj = tags ? (tags[j] & AMG_NODE_DIRICHLET) != 0 : false;
      p_col[o] = cid[j];
      p_val[o] = (di || dj) ? 0.0 : w;
      ++o;
    }
  }
}

__global__ void k_gather_tags(int n, const int* __restrict__ tags, const int* __restrict__ cid,
                              int* __restrict__ ctags) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (cid[i] >= 0) ctags[cid[i]] = tags ? tags[i] : 0;
}

// ---- transpose of a scalar-weight CSR (P -> R = P^T), rows sorted afterwards
__global__ void k_t_count(int nnz, const int* __restrict__ pcol, int* __restrict__ cnt) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x)
    atomicAdd(&cnt[pcol[k]], 1);
}

__global__ void k_t_fill(int n, const int* __restrict__ prow, const int* __restrict__ pcol,
                         const double* __restrict__ pval, int nplanes, int64_t pnnz,
                         const int* __restrict__ rrow, int* __restrict__ cursor,
                         int* __restrict__ rcol, double* __restrict__ rval, int64_t rnnz) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int k = prow[i]; k < prow[i + 1]; ++k) {
      int c = pcol[k];
      int pos = rrow[c] + atomicAdd(&cursor[c], 1);
      rcol[pos] = i;
      for (int e = 0; e < nplanes; ++e) rval[e * rnnz + pos] = pval[e * pnnz + k];
    }
  }
}

__global__ void k_sort_rows(int n, const int* __restrict__ row, int* __restrict__ colv,
                            double* __restrict__ val, int nplanes, int64_t nnz) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int a = row[i], b = row[i + 1];
    for (int k = a + 1; k < b; ++k) {   // insertion sort: rows are short
      int key = colv[k];
      double v[3];
      for (int e = 0; e < nplanes; ++e) v[e] = val[e * nnz + k];
      int m = k - 1;
      while (m >= a && colv[m] > key) {
        colv[m + 1] = colv[m];
        for (int e = 0; e < nplanes; ++e) val[e * nnz + m + 1] = val[e * nnz + m];
        --m;
      }
      colv[m + 1] = key;
      for (int e = 0; e < nplanes; ++e) val[e * nnz + m + 1] = v[e];
    }
  }
}

// ============================================================================ Galerkin product
//
// C = R M P for R (coarse rows -> fine rows, scalar weights), M (fine rows ->
// fine cols, NV value planes) and P (fine cols -> coarse cols, scalar weights).
// One warp owns one coarse row and keeps the set of its coarse columns in a
// shared-memory open-addressing table.  The symbolic passes use every stored
// entry of R, M and P (the structural pattern, zero weights included).

constexpr int kHashSize = 4096;        // slots per warp
constexpr int kGalWarps = 4;            // warps per CTA

__device__ __forceinline__ unsigned hash_slot(int key) {
  return ((unsigned)key * 2654435761u) & (kHashSize - 1);
}

// insert key; returns 1 if it was new, -1 if the table is full
__device__ __forceinline__ int hash_insert(int* tab, int key) {
  unsigned s = hash_slot(key);
  for (int probe = 0; probe < kHashSize; ++probe) {
    int old = atomicCAS(&tab[s], -1, key);
    if (old == -1) return 1;
    if (old == key) return 0;
    s = (s + 1) & (kHashSize - 1);
  }
  return -1;
}

__device__ void gal_collect(int I, const int* __restrict__ rrow, const int* __restrict__ rcol,
                            const int* __restrict__ mrow, const int* __restrict__ mcol,
                            const int* __restrict__ prow, const int* __restrict__ pcol,
                            int* tab, int* count, int* overflow) {
  int lane = threadIdx.x & 31;
  for (int t = rrow[I]; t < rrow[I + 1]; ++t) {
    int i = rcol[t];
    for (int k = mrow[i] + lane; k < mrow[i + 1]; k += 32) {
      int j = mcol[k];
      for (int q = prow[j]; q < prow[j + 1]; ++q) {
        int r = hash_insert(tab, pcol[q]);
        if (r == 1) atomicAdd(count, 1);
        else if (r < 0) atomicOr(overflow, 1);
      }
    }
  }
}

__global__ void k_gal_count(int nc, const int* __restrict__ rrow, const int* __restrict__ rcol,
                            const int* __restrict__ mrow, const int* __restrict__ mcol,
                            const int* __restrict__ prow, const int* __restrict__ pcol,
                            int* __restrict__ out_count, int* __restrict__ flag) {
  extern __shared__ int sh[];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* tab = sh + w * kHashSize;
  __shared__ int cnt[kGalWarps];
  for (int I = blockIdx.x * kGalWarps + w; I < nc; I += gridDim.x * kGalWarps) {
    for (int s = lane; s < kHashSize; s += 32) tab[s] = -1;
    if (lane == 0) cnt[w] = 0;
    __syncwarp();
    gal_collect(I, rrow, rcol, mrow, mcol, prow, pcol, tab, &cnt[w], flag);
    __syncwarp();
    if (lane == 0) out_count[I] = cnt[w];
    __syncwarp();
  }
}

__global__ void k_gal_fill(int nc, const int* __restrict__ rrow, const int* __restrict__ rcol,
                           const int* __restrict__ mrow, const int* __restrict__ mcol,
                           const int* __restrict__ prow, const int* __restrict__ pcol,
                           const int* __restrict__ crow, int* __restrict__ ccol,
                           int* __restrict__ flag) {
  extern __shared__ int sh[];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* tab = sh + w * kHashSize;
  __shared__ int cnt[kGalWarps];
  for (int I = blockIdx.x * kGalWarps + w; I < nc; I += gridDim.x * kGalWarps) {
    for (int s = lane; s < kHashSize; s += 32) tab[s] = -1;
    if (lane == 0) cnt[w] = 0;
    __syncwarp();
    gal_collect(I, rrow, rcol, mrow, mcol, prow, pcol, tab, &cnt[w], flag);
    __syncwarp();
    // compact the keys into the front of the table region's tail copy, then rank
    int base = crow[I];
    int m = crow[I + 1] - base;
    // write keys unsorted into ccol, then rank-sort in place via the table
    int pos = 0;
    for (int s0 = 0; s0 < kHashSize; s0 += 32) {
      int key = tab[s0 + lane];
      unsigned bal = __ballot_sync(0xffffffffu, key >= 0);
      if (key >= 0) {
        int off = __popc(bal & ((1u << lane) - 1));
        ccol[base + pos + off] = key;
      }
      pos += __popc(bal);
    }
    __syncwarp();
    // rank sort: the final position of each key is the number of smaller keys
    // (the table region is reused to hold the sorted row)
    for (int a = lane; a < m; a += 32) {
      int key = ccol[base + a];
      int r = 0;
      for (int b = 0; b < m; ++b) r += ccol[base + b] < key;
      tab[r] = key;
    }
    __syncwarp();
    for (int a = lane; a < m; a += 32) ccol[base + a] = tab[a];
    __syncwarp();
  }
}

template <int NV>
__global__ void k_gal_numeric(int nc, const int* __restrict__ rrow, const int* __restrict__ rcol,
                              const double* __restrict__ rval, const int* __restrict__ mrow,
                              const int* __restrict__ mcol, const double* __restrict__ mval,
                              int64_t mnnz, const int* __restrict__ prow,
                              const int* __restrict__ pcol, const double* __restrict__ pval,
                              const int* __restrict__ crow, const int* __restrict__ ccol,
                              double* __restrict__ cval, int64_t cnnz) {
  int lane = threadIdx.x & 31;
  int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int nw = (gridDim.x * blockDim.x) >> 5;
  for (int I = gw; I < nc; I += nw) {
    int base = crow[I], m = crow[I + 1] - base;
    const int* cc = ccol + base;
    for (int t = rrow[I]; t < rrow[I + 1]; ++t) {
      int i = rcol[t];
      double wi = rval[t];
      if (wi == 0.0) continue;
      for (int k = mrow[i] + lane; k < mrow[i + 1]; k += 32) {
        int j = mcol[k];
        double a[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) a[e] = mval[e * mnnz + k];
        for (int q = prow[j]; q < prow[j + 1]; ++q) {
          double w = wi * pval[q];
          if (w == 0.0) continue;
          int J = pcol[q];
          int lo = 0, hi = m - 1;
          while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (cc[mid] < J) lo = mid + 1; else hi = mid;
          }
#pragma unroll
          for (int e = 0; e < NV; ++e) atomicAdd(&cval[e * cnnz + base + lo], w * a[e]);
        }
      }
    }
  }
}

// Dirichlet coarse nodes: identity diagonal block (their rows/columns are zero).
__global__ void k_dirichlet_diag(int n, const int* __restrict__ tags, const int* __restrict__ row,
                                 const int* __restrict__ col, double* __restrict__ val,
                                 int64_t nnzb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (!(tags[i] & AMG_NODE_DIRICHLET)) continue;
    for (int k = row[i]; k < row[i + 1]; ++k) {
      if (col[k] != i) continue;
#pragma unroll
      for (int e = 0; e < 9; ++e) val[e * nnzb + k] = (e % 4 == 0) ? 1.0 : 0.0;
    }
  }
}

// ============================================================================ colouring

// One round of first-fit colouring in increasing index order: a node is coloured
// once all its lower-index neighbours are, with the smallest colour none of them
// uses.
__global__ void k_colour_round(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                               int* colour, int* remaining) {
  volatile int* vc = colour;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (vc[i] >= 0) continue;
    int a = rowptr[i], b = rowptr[i + 1];
    bool ready = true;
    for (int k = a; k < b; ++k) {
      int j = col[k];
      if (j >= i) break;
      if (vc[j] < 0) { ready = false; break; }
    }
    if (!ready) { atomicAdd(remaining, 1); continue; }
    for (int base = 0; base <= b - a; base += 32) {
      unsigned used = 0;
      for (int k = a; k < b; ++k) {
        int j = col[k];
        if (j >= i) break;
        int c = vc[j] - base;
        if (c >= 0 && c < 32) used |= 1u << c;
      }
      if (used != 0xffffffffu) {
        vc[i] = base + __ffs(~used) - 1;
        break;
      }
    }
  }
}

__global__ void k_colour_flag(int n, const int* __restrict__ colour, int c, int* __restrict__ f) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    f[i] = colour[i] == c ? 1 : 0;
}

__global__ void k_colour_scatter(int n, const int* __restrict__ colour, int c,
                                 const int* __restrict__ pos, int offset, int* __restrict__ rows) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (colour[i] == c) rows[offset + pos[i]] = i;
}

// stored-row lengths and block copy into colour order
__global__ void k_stored_len(int n, const int* __restrict__ order, const int* __restrict__ rowptr,
                             int* __restrict__ len) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int i = order[k];
    len[k] = rowptr[i + 1] - rowptr[i];
  }
}

__global__ void k_stored_copy(int n, const int* __restrict__ order, const int* __restrict__ rowptr,
                              const int* __restrict__ col, const double* __restrict__ val,
                              int64_t nnzb, const int* __restrict__ srowptr, int* __restrict__ scol,
                              double* __restrict__ sval) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int k = w; k < n; k += nw) {
    const int i = order[k];
    const int a = rowptr[i], len = rowptr[i + 1] - a, o = srowptr[k];
    for (int q = lane; q < len; q += 32) {
      scol[o + q] = col[a + q];
#pragma unroll
      for (int e = 0; e < 9; ++e) sval[e * nnzb + o + q] = val[e * nnzb + a + q];
    }
  }
}

// ============================================================================ block inverses

__global__ void k_dinv(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                       const double* __restrict__ val, int64_t nnzb, double* __restrict__ dinv,
                       int* __restrict__ flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int lo = rowptr[i], hi = rowptr[i + 1] - 1;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (col[mid] < i) lo = mid + 1; else hi = mid;
    }
    double a[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) a[e] = val[e * nnzb + lo];
    // inverse by cofactors: inv = adj(a) / det(a)
    double c00 = a[4] * a[8] - a[5] * a[7];
    double c01 = a[5] * a[6] - a[3] * a[8];
    double c02 = a[3] * a[7] - a[4] * a[6];
    double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    if (!(fabs(det) > 0.0) || !isfinite(det)) { atomicOr(flag, 64); continue; }
    double r = 1.0 / det;
    double* o = dinv + 12 * (int64_t)i;
    o[0] = c00 * r;
    o[1] = (a[2] * a[7] - a[1] * a[8]) * r;
    o[2] = (a[1] * a[5] - a[2] * a[4]) * r;
    o[3] = 0.0;
    o[4] = c01 * r;
    o[5] = (a[0] * a[8] - a[2] * a[6]) * r;
    o[6] = (a[2] * a[3] - a[0] * a[5]) * r;
    o[7] = 0.0;
    o[8] = c02 * r;
    o[9] = (a[1] * a[6] - a[0] * a[7]) * r;
    o[10] = (a[0] * a[4] - a[1] * a[3]) * r;
    o[11] = 0.0;
  }
}

// sGS pressure scaling S_D[k] = C_kk + omega * sum_j b_kj^T D_j^{-1} b_kj
__global__ void k_schur_diag(int np, const int* __restrict__ brow, const int* __restrict__ bcol,
                             const double* __restrict__ bval, int64_t bnnz,
                             const int* __restrict__ crow, const int* __restrict__ ccol,
                             const double* __restrict__ cval, const double* __restrict__ dinv,
                             double omega, double* __restrict__ out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = crow[k]; q < crow[k + 1]; ++q)
      if (ccol[q] == k) s = cval[q];
    double acc = 0.0;
    for (int q = brow[k]; q < brow[k + 1]; ++q) {
      int j = bcol[q];
      double b0 = bval[q], b1 = bval[bnnz + q], b2 = bval[2 * bnnz + q];
      const double* d = dinv + 12 * (int64_t)j;
      acc += b0 * (d[0] * b0 + d[1] * b1 + d[2] * b2) + b1 * (d[4] * b0 + d[5] * b1 + d[6] * b2) +
             b2 * (d[8] * b0 + d[9] * b1 + d[10] * b2);
    }
    out[k] = s + omega * acc;
  }
}

// ============================================================================ coarsest level

// dense K = [A B^T; B -C] (row-major m x m, m = 3n + np)
__global__ void k_dense_A(int n, const int* __restrict__ row, const int* __restrict__ col,
                          const double* __restrict__ val, int64_t nnzb, int m,
                          double* __restrict__ K) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int k = row[i]; k < row[i + 1]; ++k) {
      int j = col[k];
      for (int e = 0; e < 9; ++e)
        K[(int64_t)(3 * i + e / 3) * m + 3 * j + e % 3] = val[e * nnzb + k];
    }
}

__global__ void k_dense_BC(int np, int n3, const int* __restrict__ brow,
                           const int* __restrict__ bcol, const double* __restrict__ bval,
                           int64_t bnnz, const int* __restrict__ crow,
                           const int* __restrict__ ccol, const double* __restrict__ cval, int m,
                           double* __restrict__ K) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
    for (int q = brow[k]; q < brow[k + 1]; ++q) {
      int j = bcol[q];
      for (int c = 0; c < 3; ++c) {
        double v = bval[c * bnnz + q];
        K[(int64_t)(n3 + k) * m + 3 * j + c] = v;   // B
        K[(int64_t)(3 * j + c) * m + n3 + k] = v;   // B^T
      }
    }
    for (int q = crow[k]; q < crow[k + 1]; ++q)
      K[(int64_t)(n3 + k) * m + n3 + ccol[q]] = -cval[q];
  }
}

// Entries within this relative window of the largest remaining magnitude count
// as tied pivots, broken by row-major position: exact ties of a structured
// coarse matrix then resolve the same way whatever rounding the Galerkin
// products left in them.
constexpr double kPivotTie = 1e-9;

// Gaussian elimination with complete pivoting in one CTA, stopped at the
// numerical rank (Algorithm 1, step 6: the coarsest direct solve): step k takes
// the largest magnitude M of the trailing block, pivots on its first entry in
// row-major order with magnitude >= (1 - kPivotTie) M, swaps it to (k, k) and
// eliminates.  It stops when M <= rtol * max|K|.

__global__ void k_cplu(int m, double* __restrict__ A, int* __restrict__ rp, int* __restrict__ cp,
                       double rtol, int* __restrict__ rank_out) {
  __shared__ double sv[1024];
  __shared__ long long si[1024];
  __shared__ int piv_r, piv_c, stop;
  __shared__ double scale;
  int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < m; i += nt) { rp[i] = i; cp[i] = i; }
  // global scale
  double mx = 0.0;
  for (int64_t q = tid; q < (int64_t)m * m; q += nt) mx = fmax(mx, fabs(A[q]));
  sv[tid] = mx;
  __syncthreads();
  for (int s = nt / 2; s > 0; s >>= 1) {
    if (tid < s) sv[tid] = fmax(sv[tid], sv[tid + s]);
    __syncthreads();
  }
  if (tid == 0) { scale = sv[0]; stop = 0; }
  __syncthreads();
  int rank = 0;
  for (int k = 0; k < m; ++k) {
    int w = m - k;
    // the largest magnitude M of the remaining block ...
    double bv = 0.0;
    for (long long q = tid; q < (long long)w * w; q += nt) {
      int i = (int)(q / w), j = (int)(q % w);
      bv = fmax(bv, fabs(A[(int64_t)(k + i) * m + k + j]));
    }
    sv[tid] = bv;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) {
      if (tid < s) sv[tid] = fmax(sv[tid], sv[tid + s]);
      __syncthreads();
    }
    const double big = sv[0];
    __syncthreads();
    // ... and the pivot: the first entry in row-major order whose magnitude is
    // within the relative tie window of M (rounding noise does not reorder ties)
    const double thr = (1.0 - kPivotTie) * big;
    long long bi = LLONG_MAX;
    for (long long q = tid; q < (long long)w * w; q += nt) {
      int i = (int)(q / w), j = (int)(q % w);
      if (fabs(A[(int64_t)(k + i) * m + k + j]) >= thr) { bi = q; break; }
    }
    si[tid] = bi;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) {
      if (tid < s) si[tid] = min(si[tid], si[tid + s]);
      __syncthreads();
    }
    if (tid == 0) {
      if (!(big > rtol * scale)) stop = 1;
      piv_r = k + (int)(si[0] / w);
      piv_c = k + (int)(si[0] % w);
    }
    __syncthreads();
    if (stop) break;
    int pr = piv_r, pc = piv_c;
    if (pr != k) {
      for (int j = tid; j < m; j += nt) {
        double t = A[(int64_t)k * m + j];
        A[(int64_t)k * m + j] = A[(int64_t)pr * m + j];
        A[(int64_t)pr * m + j] = t;
      }
      if (tid == 0) { int t = rp[k]; rp[k] = rp[pr]; rp[pr] = t; }
    }
    __syncthreads();
    if (pc != k) {
      for (int i = tid; i < m; i += nt) {
        double t = A[(int64_t)i * m + k];
        A[(int64_t)i * m + k] = A[(int64_t)i * m + pc];
        A[(int64_t)i * m + pc] = t;
      }
      if (tid == 0) { int t = cp[k]; cp[k] = cp[pc]; cp[pc] = t; }
    }
    __syncthreads();
    double d = A[(int64_t)k * m + k];
    for (int i = k + 1 + tid; i < m; i += nt) A[(int64_t)i * m + k] /= d;
    __syncthreads();
    int w1 = m - k - 1;
    for (long long q = tid; q < (long long)w1 * w1; q += nt) {
      int i = k + 1 + (int)(q / w1), j = k + 1 + (int)(q % w1);
      // product rounded, then the difference (no fused multiply-add)
      A[(int64_t)i * m + j] =
          __dsub_rn(A[(int64_t)i * m + j], __dmul_rn(A[(int64_t)i * m + k], A[(int64_t)k * m + j]));
    }
    __syncthreads();
    rank = k + 1;
  }
  if (tid == 0) *rank_out = rank;
}

// Column j of the generalised inverse X (x = X b solves K x = b): one CTA per
// column, forward substitution with the unit lower factor, back substitution on
// the leading rank x rank upper factor, unknowns beyond the rank set to zero.
__global__ void k_cplu_inverse(int m, const double* __restrict__ LU, const int* __restrict__ rp,
                               const int* __restrict__ cp, const int* __restrict__ rank_p,
                               double* __restrict__ work, double* __restrict__ X) {
  int j = blockIdx.x;
  int r = *rank_p;
  double* y = work + (int64_t)j * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] = (rp[i] == j) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    double yk = y[k];
    if (yk != 0.0)
      for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x)
        y[i] = __dsub_rn(y[i], __dmul_rn(LU[(int64_t)i * m + k], yk));
    __syncthreads();
  }
  for (int k = r - 1; k >= 0; --k) {
    if (threadIdx.x == 0) y[k] /= LU[(int64_t)k * m + k];
    __syncthreads();
    double yk = y[k];
    for (int i = threadIdx.x; i < k; i += blockDim.x)
      y[i] = __dsub_rn(y[i], __dmul_rn(LU[(int64_t)i * m + k], yk));
    __syncthreads();
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    X[(int64_t)cp[i] * m + j] = (i < r) ? y[i] : 0.0;
}

}  // namespace

// ============================================================================ host side

namespace {

struct Flag {
  amg_handle* h;
  explicit Flag(amg_handle* hh) : h(hh) {}
  void reset() { AMG_CUDA(cudaMemsetAsync(h->flag.p, 0, sizeof(int), h->stream)); }
  int read() {
    int v = 0;
    AMG_CUDA(cudaMemcpyAsync(&v, h->flag.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    return v;
  }
};

void upload_i32(DBuf<int>& dst, const int32_t* src, int64_t n, bool dev, cudaStream_t s) {
  dst.alloc(std::max<int64_t>(n, 1));
  if (n > 0)
    AMG_CUDA(cudaMemcpyAsync(dst.p, src, n * sizeof(int), dev ? cudaMemcpyDeviceToDevice
                                                              : cudaMemcpyHostToDevice, s));
}

void upload_planes(DBuf<double>& dst, const double* src, int64_t nnz, int nv, bool dev,
                   cudaStream_t s, amg_handle* h) {
  dst.alloc(std::max<int64_t>(nnz * nv, 1));
  if (nnz == 0) return;
  if (nv == 1) {
    AMG_CUDA(cudaMemcpyAsync(dst.p, src, nnz * sizeof(double),
                             dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return;
  }
  DBuf<double> tmp;
  tmp.alloc(nnz * nv);
  AMG_CUDA(cudaMemcpyAsync(tmp.p, src, nnz * nv * sizeof(double),
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  if (nv == 9) k_aos9_to_planes<<<grid_for(nnz), 256, 0, s>>>(tmp, dst, nnz);
  else k_aos3_to_planes<<<grid_for(nnz), 256, 0, s>>>(tmp, dst, nnz);
  AMG_LAUNCH_CHECK();
  h->launches++;
  AMG_CUDA(cudaStreamSynchronize(s));
}

void check_matrix(amg_handle* h, int nrows, int ncols, const DBuf<int>& row, const DBuf<int>& col,
                  const DBuf<double>& val, int nv, int64_t nnz, bool diag, const char* name) {
  Flag f(h);
  f.reset();
  k_check_csr<<<grid_for(nrows), 256, 0, h->stream>>>(nrows, ncols, row, col, val, nv, nnz,
                                                      diag ? 1 : 0, h->flag);
  AMG_LAUNCH_CHECK();
  h->launches++;
  int v = f.read();
  if (v) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "matrix %s malformed (flags 0x%x: 1 rowptr, 2 column range, 4 unsorted/duplicate "
             "columns, 8 non-finite value, 16 missing diagonal block)", name, v);
    fail(AMG_ERR_INVALID, buf);
  }
}

// greedy independent set by rounds; bounded by n + 1 rounds
void run_mis(amg_handle* h, int n, const DBuf<int>& row, const DBuf<int>& col, const int* tags,
             int separate, DBuf<int>& state) {
  cudaStream_t s = h->stream;
  state.alloc(std::max(n, 1));
  AMG_CUDA(cudaMemsetAsync(state.p, 0, n * sizeof(int), s));
  DBuf<int> rem;
  rem.alloc(1);
  int remaining = n;
  const int batch = 8;
  for (int round = 0; remaining > 0; round += batch) {
    if (round > n + batch) fail(AMG_ERR_TIMEOUT, "independent-set rounds exceeded their bound");
    for (int b = 0; b < batch; ++b) {
      AMG_CUDA(cudaMemsetAsync(rem.p, 0, sizeof(int), s));
      k_mis_round<<<grid_for(n), 256, 0, s>>>(n, row, col, tags, separate, state, rem);
      h->launches++;
    }
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaMemcpyAsync(&remaining, rem.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
  }
}

// prolongation from a C/F state; fills p_rowptr/p_col/p_val, cid; returns coarse count
int build_p(amg_handle* h, int n, const DBuf<int>& row, const DBuf<int>& col, const int* tags,
            int separate, const DBuf<int>& state, DBuf<int>& cid, DBuf<int>& prow,
            DBuf<int>& pcol, DBuf<double>& pval, int64_t& pnnz) {
  cudaStream_t s = h->stream;
  DBuf<int> tmp;
  tmp.alloc(std::max(n, 1));
  cid.alloc(n + 1);
  k_is_c<<<grid_for(n), 256, 0, s>>>(n, state, tmp);
  int nc = (int)exclusive_scan(tmp, cid, n, s, h);
  k_cid<<<grid_for(n), 256, 0, s>>>(n, state, cid);
  Flag f(h);
  f.reset();
  k_p_count<<<grid_for(n), 256, 0, s>>>(n, row, col, tags, separate, state, tmp, h->flag);
  prow.alloc(n + 1);
  pnnz = exclusive_scan(tmp, prow, n, s, h);
  if (f.read()) fail(AMG_ERR_INVALID, "F node without a C neighbour");
  pcol.alloc(std::max<int64_t>(pnnz, 1));
  pval.alloc(std::max<int64_t>(pnnz, 1));
  k_p_fill<<<grid_for(n), 256, 0, s>>>(n, row, col, tags, separate, state, cid, prow, pcol, pval);
  AMG_LAUNCH_CHECK();
  h->launches += 4;
  return nc;
}

void transpose(amg_handle* h, int nrows, int ncols, const DBuf<int>& row, const DBuf<int>& col,
               const DBuf<double>& val, int nplanes, int64_t nnz, DBuf<int>& trow,
               DBuf<int>& tcol, DBuf<double>& tval) {
  cudaStream_t s = h->stream;
  DBuf<int> cnt;
  cnt.alloc(ncols + 1);
  AMG_CUDA(cudaMemsetAsync(cnt.p, 0, (ncols + 1) * sizeof(int), s));
  if (nnz > 0) k_t_count<<<grid_for(nnz), 256, 0, s>>>((int)nnz, col, cnt);
  trow.alloc(ncols + 1);
  exclusive_scan(cnt, trow, ncols, s, h);
  tcol.alloc(std::max<int64_t>(nnz, 1));
  tval.alloc(std::max<int64_t>(nnz * nplanes, 1));
  AMG_CUDA(cudaMemsetAsync(cnt.p, 0, (ncols + 1) * sizeof(int), s));
  k_t_fill<<<grid_for(nrows), 256, 0, s>>>(nrows, row, col, val, nplanes, nnz, trow, cnt, tcol,
                                          tval, nnz);
  k_sort_rows<<<grid_for(ncols), 256, 0, s>>>(ncols, trow, tcol, tval, nplanes, nnz);
  AMG_LAUNCH_CHECK();
  h->launches += 3;
}

// C = R M P, structural pattern; returns nnz of C
template <int NV>
int64_t galerkin(amg_handle* h, int nc, int ncols_c, const DBuf<int>& rrow, const DBuf<int>& rcol,
                 const DBuf<double>& rval, const DBuf<int>& mrow, const DBuf<int>& mcol,
                 const DBuf<double>& mval, int64_t mnnz, const DBuf<int>& prow,
                 const DBuf<int>& pcol, const DBuf<double>& pval, DBuf<int>& crow,
                 DBuf<int>& ccol, DBuf<double>& cval) {
  (void)ncols_c;
  cudaStream_t s = h->stream;
  size_t shm = (size_t)kGalWarps * kHashSize * sizeof(int);
  max_dynamic_smem((const void*)k_gal_count, (int)shm);
  max_dynamic_smem((const void*)k_gal_fill, (int)shm);
  DBuf<int> cnt;
  cnt.alloc(nc + 1);
  Flag f(h);
  f.reset();
  int blocks = std::max(1, std::min(div_up(nc, kGalWarps), 152 * 8));
  k_gal_count<<<blocks, 32 * kGalWarps, shm, s>>>(nc, rrow, rcol, mrow, mcol, prow, pcol, cnt,
                                                   h->flag);
  AMG_LAUNCH_CHECK();
  crow.alloc(nc + 1);
  int64_t cnnz = exclusive_scan(cnt, crow, nc, s, h);
  if (f.read()) fail(AMG_ERR_UNSUPPORTED, "coarse row wider than the Galerkin hash table");
  ccol.alloc(std::max<int64_t>(cnnz, 1));
  cval.alloc(std::max<int64_t>(cnnz * NV, 1));
  AMG_CUDA(cudaMemsetAsync(cval.p, 0, cval.bytes(), s));
  k_gal_fill<<<blocks, 32 * kGalWarps, shm, s>>>(nc, rrow, rcol, mrow, mcol, prow, pcol, crow, ccol,
                                                  h->flag);
  int nblocks = std::max(1, std::min(div_up((int64_t)nc * 32, 256), 152 * 16));
  k_gal_numeric<NV><<<nblocks, 256, 0, s>>>(nc, rrow, rcol, rval, mrow, mcol, mval, mnnz, prow,
                                            pcol, pval, crow, ccol, cval, cnnz);
  AMG_LAUNCH_CHECK();
  h->launches += 3;
  return cnnz;
}

// First-fit greedy colouring of a graph in increasing vertex index (round-based,
// equal to the sequential result); `rows` receives the vertices colour by colour.
void colour_graph(amg_handle* h, int n, const DBuf<int>& rowptr, const DBuf<int>& col,
                  DBuf<int>& colour, int& ncolours, std::vector<int>& colour_ptr,
                  DBuf<int>& rows);

void colour_level(amg_handle* h, Level& lv) {
  colour_graph(h, lv.n, lv.rowptr, lv.col, lv.colour, lv.ncolours, lv.colour_ptr,
               lv.colour_rows);
}

void colour_graph(amg_handle* h, int n, const DBuf<int>& rowptr, const DBuf<int>& col,
                  DBuf<int>& colour, int& ncolours, std::vector<int>& colour_ptr,
                  DBuf<int>& rows) {
  cudaStream_t s = h->stream;
  colour.alloc(std::max(n, 1));
  AMG_CUDA(cudaMemsetAsync(colour.p, 0xff, n * sizeof(int), s));
  DBuf<int> rem;
  rem.alloc(1);
  int remaining = n;
  const int batch = 8;
  for (int round = 0; remaining > 0; round += batch) {
    if (round > n + batch) fail(AMG_ERR_TIMEOUT, "colouring rounds exceeded their bound");
    for (int b = 0; b < batch; ++b) {
      AMG_CUDA(cudaMemsetAsync(rem.p, 0, sizeof(int), s));
      k_colour_round<<<grid_for(n), 256, 0, s>>>(n, rowptr, col, colour, rem);
      h->launches++;
    }
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaMemcpyAsync(&remaining, rem.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<int> hc(n);
  AMG_CUDA(cudaMemcpyAsync(hc.data(), colour.p, n * sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  int nc = 0;
  for (int c : hc) nc = std::max(nc, c + 1);
  ncolours = nc;
  colour_ptr.assign(nc + 1, 0);
  rows.alloc(std::max(n, 1));
  DBuf<int> fl, pos;
  fl.alloc(std::max(n, 1));
  pos.alloc(n + 1);
  int off = 0;
  for (int c = 0; c < nc; ++c) {
    k_colour_flag<<<grid_for(n), 256, 0, s>>>(n, colour, c, fl);
    int cnt = (int)exclusive_scan(fl, pos, n, s, h);
    k_colour_scatter<<<grid_for(n), 256, 0, s>>>(n, colour, c, pos, off, rows);
    h->launches += 2;
    off += cnt;
    colour_ptr[c + 1] = off;
  }
  AMG_LAUNCH_CHECK();
}

void row_stats(amg_handle* h, Level& lv) {
  std::vector<int> r(lv.n + 1);
  AMG_CUDA(cudaMemcpyAsync(r.data(), lv.rowptr.p, (lv.n + 1) * sizeof(int),
                           cudaMemcpyDeviceToHost, h->stream));
  AMG_CUDA(cudaStreamSynchronize(h->stream));
  int mx = 0;
  for (int i = 0; i < lv.n; ++i) mx = std::max(mx, r[i + 1] - r[i]);
  lv.max_row_blocks = mx;
  lv.avg_row_blocks = lv.n ? (double)r[lv.n] / lv.n : 0.0;
}

void finish_level(amg_handle* h, Level& lv, bool coarsest) {
  cudaStream_t s = h->stream;
  int n = lv.n;
  row_stats(h, lv);
  lv.dinv.alloc(12 * (size_t)std::max(n, 1));
  Flag f(h);
  f.reset();
  k_dinv<<<grid_for(n), 256, 0, s>>>(n, lv.rowptr, lv.col, lv.val, lv.nnzb, lv.dinv, h->flag);
  AMG_LAUNCH_CHECK();
  h->launches++;
  if (f.read()) fail(AMG_ERR_BREAKDOWN, "singular or non-finite 3x3 diagonal block");
  if (!coarsest && !h->saddle) {
    colour_level(h, lv);
    // colour-major copy of A for the cycle kernels
    DBuf<int> len;
    len.alloc(std::max(n, 1));
    k_stored_len<<<grid_for(n), 256, 0, s>>>(n, lv.colour_rows, lv.rowptr, len);
    lv.srowptr.alloc(n + 1);
    exclusive_scan(len, lv.srowptr, n, s, h);
    lv.scol.alloc(std::max<int64_t>(lv.nnzb, 1));
    lv.sval.alloc(9 * (size_t)std::max<int64_t>(lv.nnzb, 1));
    k_stored_copy<<<grid_for((int64_t)n * 32), 256, 0, s>>>(n, lv.colour_rows, lv.rowptr, lv.col,
                                                          lv.val, lv.nnzb, lv.srowptr, lv.scol,
                                                          lv.sval);
    AMG_LAUNCH_CHECK();
    h->launches += 2;
    lv.stored = true;
  }
  bool fp32 = h->opt.precision == AMG_FP32;
  const int dofs = lv.dofs4();
  auto zalloc64 = [&](DBuf<double>& v) {
    v.alloc(std::max(dofs, 1));
    AMG_CUDA(cudaMemsetAsync(v.p, 0, v.bytes(), s));
  };
  auto zalloc32 = [&](DBuf<float>& v) {
    v.alloc(std::max(dofs, 1));
    AMG_CUDA(cudaMemsetAsync(v.p, 0, v.bytes(), s));
  };
  zalloc64(lv.x64); zalloc64(lv.b64); zalloc64(lv.r64); zalloc64(lv.t64);
  if (fp32) {
    lv.val32.alloc(9 * (size_t)std::max<int64_t>(lv.nnzb, 1));
    launch_to_float(lv.k_val(), lv.val32, 9 * lv.nnzb, s, h);
    if (h->bf16_coarse && &lv != h->L[0].get() && lv.nnzb > 0) {
      lv.val16.alloc(9 * (size_t)lv.nnzb);
      k_to_bf16<<<grid_for(9 * lv.nnzb), 256, 0, s>>>(lv.k_val(), lv.val16, 9 * lv.nnzb);
      AMG_LAUNCH_CHECK();
      h->launches++;
    }
    if (&lv == h->L[0].get() && h->opt.outer_pair && lv.nnzb > 0) {
      lv.val2.alloc(9 * (size_t)lv.nnzb);
      k_split_pair<<<grid_for(9 * lv.nnzb), 256, 0, s>>>(lv.k_val(), lv.val2, 9 * lv.nnzb);
      AMG_LAUNCH_CHECK();
      h->launches++;
    }
    lv.dinv32.alloc(12 * (size_t)std::max(n, 1));
    launch_to_float(lv.dinv, lv.dinv32, 12 * (int64_t)n, s, h);
    if (!coarsest) {
      lv.p_val32.alloc(std::max<int64_t>(lv.p_nnz, 1));
      launch_to_float(lv.p_val, lv.p_val32, lv.p_nnz, s, h);
      lv.r_val32.alloc(std::max<int64_t>(lv.p_nnz, 1));
      launch_to_float(lv.r_val, lv.r_val32, lv.p_nnz, s, h);
    }
    zalloc32(lv.x32); zalloc32(lv.b32); zalloc32(lv.r32); zalloc32(lv.t32);
  }
  if (h->saddle) {
    lv.schur.alloc(std::max(lv.np, 1));
    k_schur_diag<<<grid_for(lv.np), 256, 0, s>>>(lv.np, lv.b_rowptr, lv.b_col, lv.b_val, lv.b_nnz,
                                                lv.c_rowptr, lv.c_col, lv.c_val, lv.dinv,
                                                h->opt.omega, lv.schur);
    h->launches++;
    transpose(h, lv.np, n, lv.b_rowptr, lv.b_col, lv.b_val, 3, lv.b_nnz, lv.bt_rowptr, lv.bt_col,
              lv.bt_val);
    if (fp32) {
      lv.b_val32.alloc(std::max<int64_t>(3 * lv.b_nnz, 1));
      launch_to_float(lv.b_val, lv.b_val32, 3 * lv.b_nnz, s, h);
      lv.bt_val32.alloc(std::max<int64_t>(3 * lv.b_nnz, 1));
      launch_to_float(lv.bt_val, lv.bt_val32, 3 * lv.b_nnz, s, h);
      lv.c_val32.alloc(std::max<int64_t>(lv.c_nnz, 1));
      launch_to_float(lv.c_val, lv.c_val32, lv.c_nnz, s, h);
      lv.schur32.alloc(std::max(lv.np, 1));
      launch_to_float(lv.schur, lv.schur32, lv.np, s, h);
      if (!coarsest) {
        lv.h_val32.alloc(std::max<int64_t>(lv.h_nnz, 1));
        launch_to_float(lv.h_val, lv.h_val32, lv.h_nnz, s, h);
        lv.ht_val32.alloc(std::max<int64_t>(lv.h_nnz, 1));
        launch_to_float(lv.ht_val, lv.ht_val32, lv.h_nnz, s, h);
      }
    }
  }
  AMG_LAUNCH_CHECK();
}

std::unique_ptr<Level> coarsen(amg_handle* h, Level& lv) {
  cudaStream_t s = h->stream;
  int separate = h->opt.separate ? 1 : 0;
  run_mis(h, lv.n, lv.rowptr, lv.col, lv.tags, separate, lv.state);
  int nc = build_p(h, lv.n, lv.rowptr, lv.col, lv.tags, separate, lv.state, lv.cid, lv.p_rowptr,
                   lv.p_col, lv.p_val, lv.p_nnz);
  transpose(h, lv.n, nc, lv.p_rowptr, lv.p_col, lv.p_val, 1, lv.p_nnz, lv.r_rowptr, lv.r_col,
            lv.r_val);
  auto nx = std::make_unique<Level>();
  nx->n = nc;
  nx->tags.alloc(std::max(nc, 1));
  k_gather_tags<<<grid_for(lv.n), 256, 0, s>>>(lv.n, lv.tags, lv.cid, nx->tags);
  h->launches++;
  nx->nnzb = galerkin<9>(h, nc, nc, lv.r_rowptr, lv.r_col, lv.r_val, lv.rowptr, lv.col, lv.val,
                         lv.nnzb, lv.p_rowptr, lv.p_col, lv.p_val, nx->rowptr, nx->col, nx->val);
  k_dirichlet_diag<<<grid_for(nc), 256, 0, s>>>(nc, nx->tags, nx->rowptr, nx->col, nx->val,
                                                nx->nnzb);
  h->launches++;
  AMG_LAUNCH_CHECK();
  if (h->saddle) {
    // pressure: greedy set on the P1 graph (pattern of C), H, then B and C through H
    run_mis(h, lv.np, lv.c_rowptr, lv.c_col, nullptr, 0, lv.pstate);
    int npc = build_p(h, lv.np, lv.c_rowptr, lv.c_col, nullptr, 0, lv.pstate, lv.pcid,
                      lv.h_rowptr, lv.h_col, lv.h_val, lv.h_nnz);
    transpose(h, lv.np, npc, lv.h_rowptr, lv.h_col, lv.h_val, 1, lv.h_nnz, lv.ht_rowptr,
              lv.ht_col, lv.ht_val);
    nx->np = npc;
    nx->b_nnz = galerkin<3>(h, npc, nc, lv.ht_rowptr, lv.ht_col, lv.ht_val, lv.b_rowptr, lv.b_col,
                            lv.b_val, lv.b_nnz, lv.p_rowptr, lv.p_col, lv.p_val, nx->b_rowptr,
                            nx->b_col, nx->b_val);
    nx->c_nnz = galerkin<1>(h, npc, npc, lv.ht_rowptr, lv.ht_col, lv.ht_val, lv.c_rowptr,
                            lv.c_col, lv.c_val, lv.c_nnz, lv.h_rowptr, lv.h_col, lv.h_val,
                            nx->c_rowptr, nx->c_col, nx->c_val);
  }
  AMG_CUDA(cudaStreamSynchronize(s));
  return nx;
}

// ============================================================================ Braess-Sarazin setup
//
// S = C + B A^{-1} B^T with A^ = 2 diag(A) (scalar diagonal), formed as one
// triple product R M R^T with R = [B | I] (pressure rows; columns: the 3n
// velocity unknowns, then the pressure unknowns) and M = diag(A^{-1}) (+) C.

// 1 / (2 A_ii,cc) in the padded layout (pad entries 0)
__global__ void k_bs_ahinv(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                           const double* __restrict__ val, int64_t nnzb,
                           double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double d[3] = {0.0, 0.0, 0.0};
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] == i)
        for (int c = 0; c < 3; ++c) d[c] = val[(4 * c) * nnzb + k];
    for (int c = 0; c < 3; ++c) out[4 * (int64_t)i + c] = d[c] != 0.0 ? 0.5 / d[c] : 0.0;
    out[4 * (int64_t)i + 3] = 0.0;
  }
}

// rows of R = [B | I]: row k holds 3 entries per block of B row k, then (n3 + k, 1)
__global__ void k_bs_rrow(int np, const int* __restrict__ brow, int* __restrict__ cnt) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x)
    cnt[k] = 3 * (brow[k + 1] - brow[k]) + 1;
}

__global__ void k_bs_rfill(int np, int n3, const int* __restrict__ brow,
                           const int* __restrict__ bcol, const double* __restrict__ bval,
                           int64_t bnnz, const int* __restrict__ rrow, int* __restrict__ rcol,
                           double* __restrict__ rval) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
    int o = rrow[k];
    for (int q = brow[k]; q < brow[k + 1]; ++q)
      for (int c = 0; c < 3; ++c) {
        rcol[o] = 3 * bcol[q] + c;
        rval[o] = bval[c * bnnz + q];
        ++o;
      }
    rcol[o] = n3 + k;
    rval[o] = 1.0;
  }
}

// rows of M = diag(A^{-1}) (+) C: rows i < n3 hold (i, A^{-1}_i); row n3 + k holds
// C row k shifted by n3
__global__ void k_bs_mrow(int n3, int np, const int* __restrict__ crow, int* __restrict__ cnt) {
  const int m = n3 + np;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    cnt[i] = i < n3 ? 1 : crow[i - n3 + 1] - crow[i - n3];
}

__global__ void k_bs_mfill(int n3, int np, const double* __restrict__ ahinv,
                           const int* __restrict__ crow, const int* __restrict__ ccol,
                           const double* __restrict__ cval, const int* __restrict__ mrow,
                           int* __restrict__ mcol, double* __restrict__ mval) {
  const int m = n3 + np;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    int o = mrow[i];
    if (i < n3) {
      mcol[o] = i;
      mval[o] = ahinv[4 * (i / 3) + i % 3];
    } else {
      const int k = i - n3;
      for (int q = crow[k]; q < crow[k + 1]; ++q, ++o) {
        mcol[o] = n3 + ccol[q];
        mval[o] = cval[q];
      }
    }
  }
}

__global__ void k_s_dinv(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                         const double* __restrict__ val, double* __restrict__ dinv) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int q = rowptr[k]; q < rowptr[k + 1]; ++q)
      if (col[q] == k) d = val[q];
    dinv[k] = d != 0.0 ? 1.0 / d : 0.0;
  }
}

__global__ void k_dense_csr(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                            const double* __restrict__ val, double* __restrict__ K) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    for (int q = rowptr[k]; q < rowptr[k + 1]; ++q) K[(int64_t)k * n + col[q]] = val[q];
}

// The S hierarchy of every non-coarsest saddle level (Braess-Sarazin smoother).
void bs_setup(amg_handle* h) {
  cudaStream_t s = h->stream;
  const bool fp32 = h->opt.precision == AMG_FP32;
  const int L = (int)h->L.size() - 1;
  for (int l = 0; l < L; ++l) {
    Level& lv = *h->L[l];
    const int n3 = 3 * lv.n, np = lv.np;
    lv.ahinv.alloc(4 * (size_t)std::max(lv.n, 1));
    k_bs_ahinv<<<grid_for(lv.n), 256, 0, s>>>(lv.n, lv.rowptr, lv.col, lv.val, lv.nnzb, lv.ahinv);
    AMG_LAUNCH_CHECK();
    h->launches++;
    if (fp32) {
      lv.ahinv32.alloc(4 * (size_t)std::max(lv.n, 1));
      launch_to_float(lv.ahinv, lv.ahinv32, 4 * (int64_t)lv.n, s, h);
    }
    // R = [B | I], M = diag(A^{-1}) (+) C, R^T
    DBuf<int> cnt, rrow, rcol, mrow, mcol, trow, tcol;
    DBuf<double> rval, mval, tval;
    cnt.alloc(std::max(n3 + np, 1) + 1);
    k_bs_rrow<<<grid_for(np), 256, 0, s>>>(np, lv.b_rowptr, cnt);
    rrow.alloc(np + 1);
    const int64_t rnnz = exclusive_scan(cnt, rrow, np, s, h);
    rcol.alloc(std::max<int64_t>(rnnz, 1));
    rval.alloc(std::max<int64_t>(rnnz, 1));
    k_bs_rfill<<<grid_for(np), 256, 0, s>>>(np, n3, lv.b_rowptr, lv.b_col, lv.b_val, lv.b_nnz,
                                            rrow, rcol, rval);
    k_bs_mrow<<<grid_for(n3 + np), 256, 0, s>>>(n3, np, lv.c_rowptr, cnt);
    mrow.alloc(n3 + np + 1);
    const int64_t mnnz = exclusive_scan(cnt, mrow, n3 + np, s, h);
    mcol.alloc(std::max<int64_t>(mnnz, 1));
    mval.alloc(std::max<int64_t>(mnnz, 1));
    k_bs_mfill<<<grid_for(n3 + np), 256, 0, s>>>(n3, np, lv.ahinv, lv.c_rowptr, lv.c_col,
                                                lv.c_val, mrow, mcol, mval);
    AMG_LAUNCH_CHECK();
    h->launches += 4;
    transpose(h, np, n3 + np, rrow, rcol, rval, 1, rnnz, trow, tcol, tval);
    lv.S.clear();
    auto s0 = std::make_unique<SLevel>();
    s0->n = np;
    s0->nnz = galerkin<1>(h, np, np, rrow, rcol, rval, mrow, mcol, mval, mnnz, trow, tcol, tval,
                          s0->rowptr, s0->col, s0->val);
    lv.S.push_back(std::move(s0));
    for (int k = l; k < L; ++k) {
      Level& pk = *h->L[k];
      SLevel& cur = *lv.S.back();
      auto nx = std::make_unique<SLevel>();
      nx->n = h->L[k + 1]->np;
      nx->nnz = galerkin<1>(h, nx->n, nx->n, pk.ht_rowptr, pk.ht_col, pk.ht_val, cur.rowptr,
                            cur.col, cur.val, cur.nnz, pk.h_rowptr, pk.h_col, pk.h_val,
                            nx->rowptr, nx->col, nx->val);
      lv.S.push_back(std::move(nx));
    }
    for (auto& sp : lv.S) {
      SLevel& q = *sp;
      const int n = std::max(q.n, 1);
      q.dinv.alloc(n);
      k_s_dinv<<<grid_for(q.n), 256, 0, s>>>(q.n, q.rowptr, q.col, q.val, q.dinv);
      AMG_LAUNCH_CHECK();
      h->launches++;
      q.x64.alloc(n); q.b64.alloc(n); q.r64.alloc(n);
      AMG_CUDA(cudaMemsetAsync(q.x64.p, 0, q.x64.bytes(), s));
      if (fp32) {
        q.val32.alloc(std::max<int64_t>(q.nnz, 1));
        launch_to_float(q.val, q.val32, q.nnz, s, h);
        q.dinv32.alloc(n);
        launch_to_float(q.dinv, q.dinv32, q.n, s, h);
        q.x32.alloc(n); q.b32.alloc(n); q.r32.alloc(n);
        AMG_CUDA(cudaMemsetAsync(q.x32.p, 0, q.x32.bytes(), s));
      }
    }
    // generalised inverse of the coarsest S (complete-pivoting LU, as the coarsest K)
    SLevel& last = *lv.S.back();
    const int m = last.n;
    if (m > 2048) fail(AMG_ERR_UNSUPPORTED, "coarsest S larger than 2048 unknowns");
    lv.s_coarse_m = m;
    if (m > 0) {
      DBuf<double> K, work;
      K.alloc((size_t)m * m);
      AMG_CUDA(cudaMemsetAsync(K.p, 0, K.bytes(), s));
      k_dense_csr<<<grid_for(m), 256, 0, s>>>(m, last.rowptr, last.col, last.val, K);
      DBuf<int> rp, cp, rank;
      rp.alloc(m); cp.alloc(m); rank.alloc(1);
      k_cplu<<<1, 1024, 0, s>>>(m, K, rp, cp, 1e-13, rank);
      lv.s_coarse_inv.alloc((size_t)m * m);
      work.alloc((size_t)m * m);
      k_cplu_inverse<<<m, 256, 0, s>>>(m, K, rp, cp, rank, work, lv.s_coarse_inv);
      AMG_LAUNCH_CHECK();
      h->launches += 3;
      AMG_CUDA(cudaStreamSynchronize(s));
    }
  }
  AMG_CUDA(cudaStreamSynchronize(s));
}

// ============================================================================ Vanka setup
//
// Patch k: pressure unknown k and the velocity nodes b_col[b_rowptr[k] ..] of row
// k of B (ascending), m_k = 3 * (row length) velocity unknowns.  A_k^{-1} is
// formed in place in its slot (row-major m_k x m_k at off[k]).

constexpr int kVankaMax = 512;   // unknowns of a patch (the cycle kernel's register tile)
constexpr int kVankaSmem = 237;  // patches factorised in shared memory: m (m + 1) / 2 + m
                                 // doubles within 227 KB
constexpr int kVkCl = 8;         // CTAs of the cluster that inverts larger patches
constexpr int kVankaCluster = 470;   // ceil(m / 8) m + m doubles within 227 KB a CTA

__device__ __forceinline__ int find_col(const int* __restrict__ col, int a, int e, int j) {
  while (a < e) {
    const int mid = (a + e) >> 1;
    const int c = col[mid];
    if (c == j) return mid;
    if (c < j) a = mid + 1;
    else e = mid;
  }
  return -1;
}

// dense A_k: block (a, b) = A[node_a][node_b] (zero when not stored)
__global__ void k_vk_gather(int np, const int* __restrict__ brow, const int* __restrict__ bcol,
                            const int* __restrict__ rowptr, const int* __restrict__ col,
                            const double* __restrict__ val, int64_t nnzb,
                            const long long* __restrict__ off, double* __restrict__ ainv) {
  for (int k = blockIdx.x; k < np; k += gridDim.x) {
    const int q0 = brow[k], len = brow[k + 1] - q0, m = 3 * len;
    double* M = ainv + off[k];
    for (int t = threadIdx.x; t < len * len; t += blockDim.x) {
      const int a = t / len, b = t % len;
      const int na = bcol[q0 + a], nb = bcol[q0 + b];
      const int q = find_col(col, rowptr[na], rowptr[na + 1], nb);
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
          M[(int64_t)(3 * a + r) * m + 3 * b + c] = q >= 0 ? val[(3 * r + c) * nnzb + q] : 0.0;
    }
  }
}

// Patches above kVankaSmem unknowns: in-place Gauss-Jordan inversion of the SPD A_k
// in global memory (no pivoting: every pivot of an SPD matrix is positive); a
// non-positive pivot sets *flag and leaves the patch.
__global__ void k_vk_invert(int np, const int* __restrict__ brow,
                            const long long* __restrict__ off, double* __restrict__ ainv,
                            int* flag) {
  extern __shared__ int vk_sh[];
  double* colk = reinterpret_cast<double*>(vk_sh);   // column k before the step
  double* rowk = colk + kVankaMax;                     // row k after scaling
  for (int p = blockIdx.x; p < np; p += gridDim.x) {
    const int m = 3 * (brow[p + 1] - brow[p]);
    if (m <= kVankaCluster) continue;  // done by k_vk_chol or k_vk_gj_cluster
    double* M = ainv + off[p];
    bool bad = false;
    for (int k = 0; k < m && !bad; ++k) {
      const double piv = M[(int64_t)k * m + k];
      __syncthreads();
      if (!(piv > 0.0)) {
        if (threadIdx.x == 0) atomicOr(flag, 2);
        bad = true;
        break;
      }
      for (int i = threadIdx.x; i < m; i += blockDim.x) colk[i] = M[(int64_t)i * m + k];
      for (int j = threadIdx.x; j < m; j += blockDim.x)
        rowk[j] = (j == k ? 1.0 : M[(int64_t)k * m + j]) / piv;
      __syncthreads();
      for (int j = threadIdx.x; j < m; j += blockDim.x) M[(int64_t)k * m + j] = rowk[j];
      for (int t = threadIdx.x; t < (m - 1) * m; t += blockDim.x) {
        int i = t / m;
        const int j = t % m;
        if (i >= k) ++i;
        const double base = j == k ? 0.0 : M[(int64_t)i * m + j];
        M[(int64_t)i * m + j] = base - colk[i] * rowk[j];
      }
      __syncthreads();
    }
  }
}

// Patches of at most kVankaSmem unknowns: Cholesky of A_k, inverse of the factor
// and A_k^{-1} = L^{-T} L^{-1}, all in shared memory (packed lower triangle, row i
// at i (i + 1) / 2), then A_k^{-1} written over A_k in its slot.  Larger patches
// are left to k_vk_invert.  A non-positive pivot sets *flag.
__global__ void __launch_bounds__(512) k_vk_chol(int np, const int* __restrict__ brow,
                                                  const long long* __restrict__ off,
                                                  double* __restrict__ ainv, int* flag) {
  extern __shared__ int vk_sh[];
  double* L = reinterpret_cast<double*>(vk_sh);
  __shared__ int bad;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int p = blockIdx.x; p < np; p += gridDim.x) {
    const int m = 3 * (brow[p + 1] - brow[p]);
    if (m > kVankaSmem) continue;
    double* M = ainv + off[p];
    double* tmp = L + m * (m + 1) / 2;
    auto at = [&](int i, int j) -> double& { return L[i * (i + 1) / 2 + j]; };
    for (int i = warp; i < m; i += nwarps)
      for (int j = lane; j <= i; j += 32) at(i, j) = M[(int64_t)i * m + j];
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    // Cholesky, right-looking
    for (int k = 0; k < m; ++k) {
      if (threadIdx.x == 0) {
        const double d = at(k, k);
        if (!(d > 0.0)) bad = 1;
        at(k, k) = d > 0.0 ? sqrt(d) : 1.0;
      }
      __syncthreads();
      const double lkk = at(k, k);
      for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) at(i, k) /= lkk;
      __syncthreads();
      for (int i = k + 1 + warp; i < m; i += nwarps) {
        const double lik = at(i, k);
        for (int j = k + 1 + lane; j <= i; j += 32) at(i, j) -= lik * at(j, k);
      }
      __syncthreads();
    }
    if (bad) {
      if (threadIdx.x == 0) atomicOr(flag, 2);
      __syncthreads();
      continue;
    }
    // L^{-1} in place, column by column from the last:
    // (L^{-1})_ij = -(1 / L_jj) sum_{k=j+1..i} (L^{-1})_ik L_kj
    for (int j = m - 1; j >= 0; --j) {
      for (int i = j + 1 + warp; i < m; i += nwarps) {
        double acc = 0.0;
        for (int k = j + 1 + lane; k <= i; k += 32) acc = fma(at(i, k), at(k, j), acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) tmp[i] = -acc / at(j, j);
      }
      __syncthreads();
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) at(i, j) = tmp[i];
      __syncthreads();
      if (threadIdx.x == 0) at(j, j) = 1.0 / at(j, j);
      __syncthreads();
    }
    // A^{-1}_ij = sum_{k >= max(i, j)} (L^{-1})_ki (L^{-1})_kj
    for (int i = warp; i < m; i += nwarps)
      for (int j = lane; j <= i; j += 32) {
        double acc = 0.0;
        for (int k = i; k < m; ++k) acc = fma(at(k, i), at(k, j), acc);
        M[(int64_t)i * m + j] = acc;
        M[(int64_t)j * m + i] = acc;
      }
    __syncthreads();
  }
}

// Patches above kVankaSmem and up to kVankaCluster unknowns: Gauss-Jordan inversion
// with the matrix spread over the shared memory of an 8-CTA thread-block cluster
// (CTA r holds rows [r R, (r + 1) R), R = ceil(m / 8)).  Step k: the owner of row k
// scales it; every CTA copies it through distributed shared memory and eliminates
// column k from its own rows.  No pivoting (A_k is SPD); a non-positive pivot sets
// *flag and leaves the patch.
__global__ void __launch_bounds__(1024, 1) k_vk_gj_cluster(int np, const int* __restrict__ brow,
                                                          const long long* __restrict__ off,
                                                          double* __restrict__ ainv, int* flag) {
  namespace cgr = cooperative_groups;
  cgr::cluster_group cl = cgr::this_cluster();
  extern __shared__ int vk_sh[];
  double* loc = reinterpret_cast<double*>(vk_sh);
  __shared__ double fcol[64];
  __shared__ int bad;
  const unsigned rank = cl.block_rank();
  const int ncl = gridDim.x / kVkCl, cid = blockIdx.x / kVkCl;
  for (int p = cid; p < np; p += ncl) {
    const int m = 3 * (brow[p + 1] - brow[p]);
    if (m <= kVankaSmem || m > kVankaCluster) continue;
    const int R = (m + kVkCl - 1) / kVkCl;
    const int r0 = (int)rank * R, r1 = min(m, r0 + R), nr = max(0, r1 - r0);
    double* rowk = loc + (size_t)R * m;        // m doubles after the owned rows
    double* M = ainv + off[p];
    for (int t = threadIdx.x; t < nr * m; t += blockDim.x)
      loc[t] = M[(int64_t)(r0 + t / m) * m + t % m];
    if (threadIdx.x == 0) bad = 0;
    cl.sync();
    for (int k = 0; k < m; ++k) {
      const unsigned owner = (unsigned)(k / R);
      if (rank == owner) {
        double* rk = loc + (size_t)(k - r0) * m;
        const double piv = rk[k];
        __syncthreads();
        if (!(piv > 0.0)) {
          if (threadIdx.x == 0) bad = 1;
        } else {
          for (int j = threadIdx.x; j < m; j += blockDim.x) rk[j] = (j == k ? 1.0 : rk[j]) / piv;
        }
      }
      cl.sync();
      const double* src = cl.map_shared_rank(loc, owner) + (size_t)(k - (int)owner * R) * m;
      const int obad = *cl.map_shared_rank(&bad, owner);
      for (int j = threadIdx.x; j < m; j += blockDim.x) rowk[j] = src[j];
      for (int i = threadIdx.x; i < nr; i += blockDim.x) fcol[i] = loc[(size_t)i * m + k];
      __syncthreads();
      if (!obad) {
        for (int t = threadIdx.x; t < nr * m; t += blockDim.x) {
          const int i = t / m, j = t % m;
          if (r0 + i == k) continue;
          const double base = j == k ? 0.0 : loc[t];
          loc[t] = base - fcol[i] * rowk[j];
        }
      }
      cl.sync();
      if (obad) {
        if (threadIdx.x == 0 && rank == 0) atomicOr(flag, 2);
        break;
      }
    }
    for (int t = threadIdx.x; t < nr * m; t += blockDim.x)
      M[(int64_t)(r0 + t / m) * m + t % m] = loc[t];
    cl.sync();
  }
}

// w_k = A_k^{-1} B_k^T, s_k = B_k w_k + C_kk
__global__ void k_vk_ws(int np, const int* __restrict__ brow, const double* __restrict__ bval,
                        int64_t bnnz, const int* __restrict__ crow,
                        const int* __restrict__ ccol, const double* __restrict__ cval,
                        const long long* __restrict__ off, const double* __restrict__ ainv,
                        double* __restrict__ w, double* __restrict__ sk) {
  __shared__ double red[8];
  for (int p = blockIdx.x; p < np; p += gridDim.x) {
    const int q0 = brow[p], m = 3 * (brow[p + 1] - q0);
    const double* M = ainv + off[p];
    double* wp = w + 3 * (int64_t)q0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      double acc = 0.0;
      for (int j = 0; j < m; ++j)
        acc = fma(M[(int64_t)i * m + j], bval[(j % 3) * bnnz + q0 + j / 3], acc);
      wp[i] = acc;
    }
    __syncthreads();
    double part = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x)
      part = fma(bval[(j % 3) * bnnz + q0 + j / 3], wp[j], part);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
      double c = 0.0;
      for (int q = crow[p]; q < crow[p + 1]; ++q)
        if (ccol[q] == p) c = cval[q];
      sk[p] = t + c;
    }
    __syncthreads();
  }
}

__global__ void k_iota(int* a, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    a[k] = k;
}

// Patches, local inverses and the patch colouring of every non-coarsest saddle level.
void vanka_setup(amg_handle* h) {
  cudaStream_t s = h->stream;
  const bool fp32 = h->opt.precision == AMG_FP32;
  const int L = (int)h->L.size() - 1;
  for (int l = 0; l < L; ++l) {
    Level& lv = *h->L[l];
    const int np = lv.np;
    std::vector<int> br(np + 1);
    AMG_CUDA(cudaMemcpyAsync(br.data(), lv.b_rowptr.p, (np + 1) * sizeof(int),
                             cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    std::vector<long long> off(np + 1, 0);
    int mmax = 0;
    for (int k = 0; k < np; ++k) {
      const long long m = 3LL * (br[k + 1] - br[k]);
      mmax = std::max<int>(mmax, (int)m);
      off[k + 1] = off[k] + m * m;
    }
    if (mmax > kVankaMax) fail(AMG_ERR_UNSUPPORTED, "Vanka patch larger than 512 unknowns");
    lv.vk_mmax = mmax;
    lv.vk_off.alloc(np + 1);
    AMG_CUDA(cudaMemcpyAsync(lv.vk_off.p, off.data(), (np + 1) * sizeof(long long),
                             cudaMemcpyHostToDevice, s));
    lv.vk_ainv.alloc(std::max<long long>(off[np], 1));
    lv.vk_w.alloc(std::max<int64_t>(3 * lv.b_nnz, 1));
    lv.vk_s.alloc(std::max(np, 1));
    const int grid = std::max(1, std::min(np, 152 * 8));
    k_vk_gather<<<grid, 256, 0, s>>>(np, lv.b_rowptr, lv.b_col, lv.rowptr, lv.col, lv.val,
                                     lv.nnzb, lv.vk_off, lv.vk_ainv);
    AMG_LAUNCH_CHECK();
    Flag f(h);
    f.reset();
    const int msm = std::min(mmax, kVankaSmem);
    const size_t chol_shm = (size_t)(msm * (msm + 1) / 2 + msm) * sizeof(double);
    max_dynamic_smem((const void*)k_vk_chol,
                     (int)((kVankaSmem * (kVankaSmem + 1) / 2 + kVankaSmem) * sizeof(double)));
    k_vk_chol<<<std::max(1, std::min(np, 152 * 2)), 512, chol_shm, s>>>(np, lv.b_rowptr,
                                                                       lv.vk_off, lv.vk_ainv,
                                                                       h->flag);
    AMG_LAUNCH_CHECK();
    if (mmax > kVankaSmem) {
      const int mc = std::min(mmax, kVankaCluster);
      const int Rc = (mc + kVkCl - 1) / kVkCl;
      const size_t cl_shm = ((size_t)Rc * mc + mc) * sizeof(double);
      const int Rmax = (kVankaCluster + kVkCl - 1) / kVkCl;
      max_dynamic_smem((const void*)k_vk_gj_cluster,
                       (int)(((size_t)Rmax * kVankaCluster + kVankaCluster) * sizeof(double)));
      cudaLaunchConfig_t cfg{};
      const int nclusters = std::max(1, std::min(np, 152 / kVkCl));
      cfg.gridDim = dim3((unsigned)(nclusters * kVkCl));
      cfg.blockDim = dim3(1024);
      cfg.dynamicSmemBytes = cl_shm;
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = kVkCl;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      AMG_CUDA(cudaLaunchKernelEx(&cfg, k_vk_gj_cluster, np, (const int*)lv.b_rowptr.p,
                                  (const long long*)lv.vk_off.p, lv.vk_ainv.p, h->flag.p));
      h->launches++;
    }
    if (mmax > kVankaCluster) {
      k_vk_invert<<<grid, 256, 2 * kVankaMax * sizeof(double), s>>>(np, lv.b_rowptr, lv.vk_off,
                                                                    lv.vk_ainv, h->flag);
      AMG_LAUNCH_CHECK();
    }
    k_vk_ws<<<grid, 256, 0, s>>>(np, lv.b_rowptr, lv.b_val, lv.b_nnz, lv.c_rowptr, lv.c_col,
                                 lv.c_val, lv.vk_off, lv.vk_ainv, lv.vk_w, lv.vk_s);
    AMG_LAUNCH_CHECK();
    h->launches += 3;
    if (f.read()) fail(AMG_ERR_BREAKDOWN, "Vanka patch matrix A_k is not positive definite");
    if (fp32) {
      lv.vk_ainv32.alloc(std::max<long long>(off[np], 1));
      launch_to_float(lv.vk_ainv, lv.vk_ainv32, off[np], s, h);
      lv.vk_w32.alloc(std::max<int64_t>(3 * lv.b_nnz, 1));
      launch_to_float(lv.vk_w, lv.vk_w32, 3 * lv.b_nnz, s, h);
      lv.vk_s32.alloc(std::max(np, 1));
      launch_to_float(lv.vk_s, lv.vk_s32, np, s, h);
    }
    // overlap graph of the patches: the pattern of B B^T (node level)
    DBuf<int> irow, icol, trow, tcol, orow, ocol;
    DBuf<double> ones, ival, tval, oval;
    ones.alloc(std::max<int64_t>(lv.b_nnz, 1));
    launch_fill(ones, 1.0, lv.b_nnz, s, h);
    irow.alloc(lv.n + 1);
    k_iota<<<grid_for(lv.n + 1), 256, 0, s>>>(irow, lv.n + 1);
    icol.alloc(std::max(lv.n, 1));
    k_iota<<<grid_for(lv.n), 256, 0, s>>>(icol, lv.n);
    ival.alloc(std::max(lv.n, 1));
    launch_fill(ival, 1.0, lv.n, s, h);
    h->launches += 2;
    transpose(h, np, lv.n, lv.b_rowptr, lv.b_col, ones, 1, lv.b_nnz, trow, tcol, tval);
    galerkin<1>(h, np, np, lv.b_rowptr, lv.b_col, ones, irow, icol, ival, lv.n, trow, tcol, tval,
                orow, ocol, oval);
    colour_graph(h, np, orow, ocol, lv.vk_colour, lv.vk_ncolours, lv.vk_colour_ptr, lv.vk_rows);
    // velocity nodes of every colour's patches (disjoint within a colour)
    std::vector<int> rows_h(std::max(np, 1)), bcol_h(std::max<int64_t>(lv.b_nnz, 1));
    AMG_CUDA(cudaMemcpyAsync(rows_h.data(), lv.vk_rows.p, np * sizeof(int),
                             cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaMemcpyAsync(bcol_h.data(), lv.b_col.p, lv.b_nnz * sizeof(int),
                             cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    std::vector<int> cn;
    cn.reserve(lv.b_nnz);
    lv.vk_cnode_ptr.assign(lv.vk_ncolours + 1, 0);
    for (int c = 0; c < lv.vk_ncolours; ++c) {
      for (int t = lv.vk_colour_ptr[c]; t < lv.vk_colour_ptr[c + 1]; ++t) {
        const int k = rows_h[t];
        for (int q = br[k]; q < br[k + 1]; ++q) cn.push_back(bcol_h[q]);
      }
      lv.vk_cnode_ptr[c + 1] = (int)cn.size();
    }
    lv.vk_cnodes.alloc(std::max<size_t>(cn.size(), 1));
    AMG_CUDA(cudaMemcpyAsync(lv.vk_cnodes.p, cn.data(), cn.size() * sizeof(int),
                             cudaMemcpyHostToDevice, s));
    AMG_CUDA(cudaStreamSynchronize(s));
  }
}

void factor_coarsest(amg_handle* h) {
  Level& lv = *h->L.back();
  cudaStream_t s = h->stream;
  int m = lv.dofs();
  if (m > 2048) fail(AMG_ERR_UNSUPPORTED, "coarsest level larger than 2048 unknowns");
  h->coarse_m = m;
  DBuf<double> K;
  K.alloc((size_t)m * m);
  AMG_CUDA(cudaMemsetAsync(K.p, 0, K.bytes(), s));
  k_dense_A<<<grid_for(lv.n), 256, 0, s>>>(lv.n, lv.rowptr, lv.col, lv.val, lv.nnzb, m, K);
  if (h->saddle && lv.np > 0)
    k_dense_BC<<<grid_for(lv.np), 256, 0, s>>>(lv.np, 3 * lv.n, lv.b_rowptr, lv.b_col, lv.b_val,
                                              lv.b_nnz, lv.c_rowptr, lv.c_col, lv.c_val, m, K);
  DBuf<int> rp, cp, rank;
  rp.alloc(m); cp.alloc(m); rank.alloc(1);
  k_cplu<<<1, 1024, 0, s>>>(m, K, rp, cp, 1e-13, rank);
  h->coarse_inv.alloc((size_t)m * m);
  DBuf<double> work;
  work.alloc((size_t)m * m);
  k_cplu_inverse<<<m, 256, 0, s>>>(m, K, rp, cp, rank, work, h->coarse_inv);
  AMG_LAUNCH_CHECK();
  h->launches += 4;
  AMG_CUDA(cudaMemcpyAsync(&h->coarse_rank, rank.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

void build_hierarchy(amg_handle* h, const amg_matrix* m, const int32_t* tags) {
  cudaStream_t s = h->stream;
  bool dev = m->device_ptrs != 0;
  auto l0 = std::make_unique<Level>();
  Level& lv = *l0;
  lv.n = m->n_nodes;
  lv.nnzb = m->nnzb;
  upload_i32(lv.rowptr, m->a_rowptr, lv.n + 1, dev, s);
  upload_i32(lv.col, m->a_col, lv.nnzb, dev, s);
  upload_i32(lv.tags, tags, lv.n, dev, s);
  upload_planes(lv.val, m->a_val, lv.nnzb, 9, dev, s, h);
  AMG_CUDA(cudaStreamSynchronize(s));
  check_matrix(h, lv.n, lv.n, lv.rowptr, lv.col, lv.val, 9, lv.nnzb, true, "A");
  if (h->saddle) {
    lv.np = m->n_pres;
    lv.b_nnz = m->b_nnz;
    lv.c_nnz = m->c_nnz;
    upload_i32(lv.b_rowptr, m->b_rowptr, lv.np + 1, dev, s);
    upload_i32(lv.b_col, m->b_col, lv.b_nnz, dev, s);
    upload_planes(lv.b_val, m->b_val, lv.b_nnz, 3, dev, s, h);
    upload_i32(lv.c_rowptr, m->c_rowptr, lv.np + 1, dev, s);
    upload_i32(lv.c_col, m->c_col, lv.c_nnz, dev, s);
    upload_planes(lv.c_val, m->c_val, lv.c_nnz, 1, dev, s, h);
    AMG_CUDA(cudaStreamSynchronize(s));
    check_matrix(h, lv.np, lv.n, lv.b_rowptr, lv.b_col, lv.b_val, 3, lv.b_nnz, false, "B");
    check_matrix(h, lv.np, lv.np, lv.c_rowptr, lv.c_col, lv.c_val, 1, lv.c_nnz, true, "C");
  }
  h->L.clear();
  h->L.push_back(std::move(l0));
  int max_levels = std::max(1, std::min(h->opt.max_levels, AMG_MAX_LEVELS));
  while ((int)h->L.size() < max_levels && h->L.back()->dofs() > h->opt.coarse_dofs) {
    Level& cur = *h->L.back();
    auto nx = coarsen(h, cur);
    if (nx->n == cur.n || nx->n == 0) {
      // no reduction: this level becomes the coarsest; drop its transfer data
      cur.state.release(); cur.cid.release(); cur.p_rowptr.release(); cur.p_col.release();
      cur.p_val.release(); cur.r_rowptr.release(); cur.r_col.release(); cur.r_val.release();
      cur.p_nnz = 0;
      break;
    }
    h->L.push_back(std::move(nx));
  }
  for (size_t l = 0; l < h->L.size(); ++l) finish_level(h, *h->L[l], l + 1 == h->L.size());
  // learned weights start at the plain method's (all 1)
  h->wts.alloc(4 * h->L.size());
  launch_fill(h->wts, 1.0, 4 * (int64_t)h->L.size(), s, h);
  for (size_t l = 0; l < h->L.size(); ++l) h->L[l]->wt = h->wts.p + 4 * l;
  factor_coarsest(h);
  if (h->saddle && h->opt.smoother == AMG_SMOOTHER_BS) bs_setup(h);
  if (h->saddle && h->opt.smoother == AMG_SMOOTHER_VANKA) vanka_setup(h);
  autotune_levels(h);
  AMG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace amgp2
