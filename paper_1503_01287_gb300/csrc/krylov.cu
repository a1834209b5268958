// Krylov accelerators of the AMG preconditioner (Sec. 3.1 and Sec. 4):
// preconditioned CG (SPD, FP64 cycle), flexible CG (SPD, FP32 cycle), right-
// preconditioned flexible GMRES(m) (saddle systems), and the stand-alone AMG
// iteration.  The CG vectors, residuals and inner products are FP64; the FGMRES basis
// and its Gram-Schmidt sweep are FP32 pairs (about 2^-48), its Hessenberg matrix FP64.
// Scalars stay on the device and the host reads one residual estimate per iteration
// for the stopping rule ||b - K x_k|| / ||b|| <= tol.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "amg_internal.cuh"
#include "vec.cuh"

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

constexpr int kMdotG = 8;   // basis rows per block row of the multi-dot

// out[d * ostride + i] = sum over b < nblk of partial[(b * m + i) * nv + d] in block
// order, one warp per (i, d)
__global__ void k_mdot_final(const double* __restrict__ partial, int nblk, int m, int nv,
                             int ostride, double* __restrict__ out) {
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= m * nv) return;
  const int i = t / nv, d = t - i * nv;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += partial[((int64_t)b * m + i) * nv + d];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[d * ostride + i] = s;
}

// The Gram-Schmidt sweep of flexible GMRES with delayed reorthogonalisation (DCGS2:
// Swirydowicz, Langou, Ananthan, Yang and Thomas, Numer. Linear Algebra Appl. 28,
// 2021).  Rows 0..m-1 of the basis are final; row m holds u, the pending vector
// (orthogonalised once and normalised); w is the new Krylov vector K z.  One pass
// over the basis gives p_i = V_i . u and q_i = V_i . w for i < m together with
// u . u and u . w (row m is u itself).
//
// The basis, u and w are FP32 pairs (hi + lo, the FP64 value to about 2^-48) and all
// of the sweep's arithmetic is FP32 (pair_fma: exact products and TwoSum), because
// FP64 instructions issue at a small fraction of the FP32 rate on this GPU: with
// four FP64 FMAs per basis entry and step the sweep was bound by them, far below
// the memory bandwidth.  Only each warp's final sums are converted to FP64.
//
// The basis streams through shared memory in a ring of kStages stages, filled by a
// producer warp with 1-D bulk copies (cp.async.bulk, the TMA's linear mode) of
// kTile-entry pieces of the rows.  Each stage has two mbarriers: "full" completes when
// the stage's bytes have landed; "empty" completes when each of the kConsumers
// consumer warps has arrived on it after using the stage.  The producer refills a
// stage once it is empty, so the copies run ahead of the arithmetic by up to kStages
// stages and a consumer warp waits only for its own next stage, never for the other
// warps.  Every wait is bounded: a warp that gives up raises the CTA's abort flag
// and *err, the others stop at their next wait, and the producer waits (bounded) for
// its copies in flight before the CTA returns.
constexpr int kTile = 256;                 // entries of a row piece (2 KB of pairs)
constexpr int kConsumers = kTile / 32;     // consumer warps: one entry a thread
constexpr int kThreads = kTile + 32;       // and one producer warp
constexpr int kPieces = 10;                // pieces a stage: up to 8 basis rows, u and w
constexpr int kStages = 3;
constexpr unsigned kBulkSpins = 1u << 20;
constexpr int kStreamSmem = kStages * kPieces * kTile * (int)sizeof(float2);   // 60 KB
constexpr int kCtasPerSm = 3;              // CTAs of a sweep kernel an SM (shared memory)

__device__ __forceinline__ uint32_t sm_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(b)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_addr(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_addr(b)),
               "r"(bytes)
               : "memory");
}
// bytes (a multiple of 16, both addresses 16-byte aligned) from global to shared
// memory, counted on mbarrier b
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          sm_addr(dst)),
      "l"(src), "r"(bytes), "r"(sm_addr(b))
      : "memory");
}
// waits for the completion of the phase of parity par; false after kBulkSpins polls
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t par) {
  for (unsigned i = 0; i < kBulkSpins; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(sm_addr(b)), "r"(par)
        : "memory");
    if (done) return true;
  }
  return false;
}
// The ring of one CTA: full and empty mbarriers a stage and the abort flag.
struct Ring {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  int abort;
};
__device__ __forceinline__ void ring_init(Ring& r) {
  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      bar_init(&r.full[st], 1);
      bar_init(&r.empty[st], kConsumers);
    }
    r.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}
// The producer loop (lane 0 of the last warp): load q goes to stage q % kStages once
// the consumers have emptied that stage's previous load; issue(st, q) posts the
// expected bytes on full[st] and starts the copies.  At the end it waits (bounded) for
// the last loads' copies, which are all that can still be in flight.
template <typename Issue>
__device__ void ring_produce(Ring& r, int64_t nq, int* err, Issue issue) {
  int64_t q = 0;
  for (; q < nq; ++q) {
    const int st = (int)(q % kStages);
    if (q >= kStages &&
        !bar_wait(&r.empty[st], (uint32_t)(((q / kStages) - 1) & 1))) {
      atomicExch(&r.abort, 1);
      atomicExch(err, 1);
      break;
    }
    if (*(volatile int*)&r.abort) break;
    issue(st, q);
  }
  for (int64_t d = q > kStages ? q - kStages : 0; d < q; ++d)
    bar_wait(&r.full[d % kStages], (uint32_t)((d / kStages) & 1));
}
// A consumer warp's wait for load q, called by all its lanes; false in every lane
// (abort raised) if a lane gave up or another warp did.
__device__ __forceinline__ bool ring_wait(Ring& r, int64_t q, int* err) {
  bool ok = *(volatile int*)&r.abort == 0;
  if (ok) ok = bar_wait(&r.full[q % kStages], (uint32_t)((q / kStages) & 1));
  ok = __all_sync(0xffffffffu, ok);
  if (!ok && (threadIdx.x & 31) == 0) {
    atomicExch(&r.abort, 1);
    atomicExch(err, 1);
  }
  return ok;
}
// A consumer warp is done with load q's stage.
__device__ __forceinline__ void ring_release(Ring& r, int64_t q) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) bar_arrive(&r.empty[q % kStages]);
}
__device__ __forceinline__ uint32_t piece_bytes(int64_t ld, int64_t k0) {
  return (uint32_t)(min((int64_t)kTile, ld - k0) * (int64_t)sizeof(float2));
}

// partial[(blockIdx.x * rows + i) * 2 + {0, 1}] = sum over the tiles of block column
// blockIdx.x of V_i[k] u[k] and V_i[k] w[k], kMdotG rows per block row (blockIdx.y).
// Rows are ld entries apart; the entries from n to ld are padding (copied, not used).
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_mdot2(int64_t n, int64_t ld, int rows,
                                                    const float2* __restrict__ V,
                                                    const float2* __restrict__ u,
                                                    const float2* __restrict__ w,
                                                    double* __restrict__ partial,
                                                    int* __restrict__ err) {
  extern __shared__ __align__(128) float2 ring[];
  __shared__ Ring R;
  __shared__ double sh[2 * kMdotG][kConsumers];
  const int i0 = blockIdx.y * kMdotG;
  const int gn = min(kMdotG, rows - i0);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  const int64_t nq = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  ring_init(R);
  float Su[kMdotG], su[kMdotG], Sw[kMdotG], sw[kMdotG];
#pragma unroll
  for (int g = 0; g < kMdotG; ++g) Su[g] = su[g] = Sw[g] = sw[g] = 0.f;
  if (threadIdx.x >= kTile) {
    if (threadIdx.x == kTile)
      ring_produce(R, nq, err, [&](int st, int64_t q) {
        const int64_t k0 = (blockIdx.x + q * gridDim.x) * kTile;
        const uint32_t bytes = piece_bytes(ld, k0);
        bar_expect(&R.full[st], bytes * (gn + 2));
        float2* dst = ring + (size_t)st * kPieces * kTile;
        for (int g = 0; g < gn; ++g)
          bulk_load(dst + g * kTile, V + (int64_t)(i0 + g) * ld + k0, bytes, &R.full[st]);
        bulk_load(dst + 8 * kTile, u + k0, bytes, &R.full[st]);
        bulk_load(dst + 9 * kTile, w + k0, bytes, &R.full[st]);
      });
  } else {
    for (int64_t q = 0; q < nq; ++q) {
      if (!ring_wait(R, q, err)) break;
      const float2* sg = ring + (size_t)(q % kStages) * kPieces * kTile;
      const int64_t k = (blockIdx.x + q * gridDim.x) * kTile + threadIdx.x;
      if (k < n) {
        const float2 uk = sg[8 * kTile + threadIdx.x], wk = sg[9 * kTile + threadIdx.x];
#pragma unroll
        for (int g = 0; g < kMdotG; ++g) {
          if (g < gn) {
            const float2 v = sg[g * kTile + threadIdx.x];
            pair_fma(Su[g], su[g], v, uk.x, uk.y);
            pair_fma(Sw[g], sw[g], v, wk.x, wk.y);
          }
        }
      }
      ring_release(R, q);
    }
  }
  __syncthreads();
  // the sums of a warp in pair arithmetic, then in FP64 across the consumer warps
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid < kConsumers) {
#pragma unroll
    for (int q = 0; q < 2 * kMdotG; ++q) {
      float S = q < kMdotG ? Su[q] : Sw[q - kMdotG];
      float e = q < kMdotG ? su[q] : sw[q - kMdotG];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float T = __shfl_xor_sync(0xffffffffu, S, o);
        const float t = __shfl_xor_sync(0xffffffffu, e, o);
        pair_add(S, e, T, t);
      }
      if (lane == 0) sh[q][wid] = (double)S + (double)e;
    }
  }
  __syncthreads();
  const int g = threadIdx.x >> 1, d = threadIdx.x & 1;
  if (threadIdx.x < 2 * kMdotG && g < gn) {
    double t = 0.0;
    for (int q = 0; q < kConsumers; ++q) t += sh[d * kMdotG + g][q];
    partial[(blockIdx.x * (int64_t)rows + i0 + g) * 2 + d] = t;
  }
}

// FP32 pair of an FP64 value (hi = fl32(d), lo = fl32(d - hi)) and back
__device__ __forceinline__ float2 to_pair(double d) {
  const float hi = __double2float_rn(d);
  return make_float2(hi, __double2float_rn(d - (double)hi));
}
__device__ __forceinline__ double from_pair(float2 p) { return (double)p.x + (double)p.y; }
// a leading sum S and a small error sum s as one normalised pair (FastTwoSum)
__device__ __forceinline__ float2 norm_pair(float S, float s) {
  const float hi = __fadd_rn(S, s);
  return make_float2(hi, __fsub_rn(s, __fsub_rn(hi, S)));
}

// Coefficients of the update from the sweep's dots (coef: p at [0, kMaxDots), q at
// [kMaxDots, 2 kMaxDots), u . u at p[m], u . w at q[m]):
//   s = ||u - V p|| = sqrt(u . u - p . p)   (u - V p is orthogonal to V)
//   h = v . w with v = (u - V p) / s, i.e. (u . w - p . q) / s
// written to coef[2 kMaxDots + {0, 1, 2}] = s, h, 1/s.  One warp, fixed order.
__global__ void k_dcgs2_coef(int m, double* __restrict__ coef) {
  const int lane = threadIdx.x & 31;
  double pp = 0.0, pq = 0.0;
  for (int i = lane; i < m; i += 32) {
    const double p = coef[i];
    pp = fma(p, p, pp);
    pq = fma(p, coef[kMaxDots + i], pq);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pp += __shfl_xor_sync(0xffffffffu, pp, o);
    pq += __shfl_xor_sync(0xffffffffu, pq, o);
  }
  if (threadIdx.x == 0) {
    const double sn = sqrt(fmax(coef[m] - pp, 0.0));
    coef[2 * kMaxDots] = sn;
    coef[2 * kMaxDots + 1] = sn > 0.0 ? (coef[kMaxDots + m] - pq) / sn : 0.0;
    coef[2 * kMaxDots + 2] = sn > 0.0 ? 1.0 / sn : 0.0;
  }
}

// The update of the same step, one more pass over rows 0..m-1 (pair arithmetic):
//   v  = (u - sum_i p_i V_i) / s         written over u (row m): final
//   w' = w - sum_i q_i V_i - h v          written to wn (row m + 1): the next pending
// vector before its normalisation; partial[blockIdx.x] = the block's sum of w'^2.
// A CTA takes tiles of kTile entries (one a thread); a tile's rows stream through
// the ring eight at a time, u and w with the first eight.
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_dcgs2_update(int64_t n, int64_t ld, int m,
                                                           const float2* __restrict__ V,
                                                           float2* u,
                                                           const float2* __restrict__ w,
                                                           float2* wn,
                                                           const double* __restrict__ coef,
                                                           double* __restrict__ partial,
                                                           int* __restrict__ err) {
  extern __shared__ __align__(128) float2 ring[];
  __shared__ Ring R;
  __shared__ float2 cp[kMaxDots], cq[kMaxDots];   // -p_i and -q_i as pairs
  __shared__ double sh[kConsumers];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    cp[i] = to_pair(-coef[i]);
    cq[i] = to_pair(-coef[kMaxDots + i]);
  }
  const float2 hneg = to_pair(-coef[2 * kMaxDots + 1]);
  const float2 inv_s = to_pair(coef[2 * kMaxDots + 2]);
  const int nch = max(1, (m + 7) / 8);
  const int64_t ntiles = (n + kTile - 1) / kTile;
  const int64_t my = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t nq = my * nch;
  ring_init(R);   // also orders the coefficient stores before their use
  float Sn = 0.f, sn = 0.f;
  if (threadIdx.x >= kTile) {
    if (threadIdx.x == kTile)
      ring_produce(R, nq, err, [&](int st, int64_t q) {
        const int64_t k0 = (blockIdx.x + (q / nch) * gridDim.x) * kTile;
        const int c = (int)(q % nch);
        const int r0 = 8 * c, rn = max(0, min(8, m - r0));
        const uint32_t bytes = piece_bytes(ld, k0);
        bar_expect(&R.full[st], bytes * (rn + (c == 0 ? 2 : 0)));
        float2* dst = ring + (size_t)st * kPieces * kTile;
        for (int r = 0; r < rn; ++r)
          bulk_load(dst + r * kTile, V + (int64_t)(r0 + r) * ld + k0, bytes, &R.full[st]);
        if (c == 0) {
          bulk_load(dst + 8 * kTile, u + k0, bytes, &R.full[st]);
          bulk_load(dst + 9 * kTile, w + k0, bytes, &R.full[st]);
        }
      });
  } else {
    // even and odd rows of a chunk in separate sums: two independent chains each
    float Sv = 0.f, sv = 0.f, Sw = 0.f, sw = 0.f, Tv = 0.f, tv = 0.f, Tw = 0.f, tw = 0.f;
    for (int64_t q = 0; q < nq; ++q) {
      if (!ring_wait(R, q, err)) break;
      const float2* sg = ring + (size_t)(q % kStages) * kPieces * kTile;
      const int c = (int)(q % nch);
      if (c == 0) {
        const float2 uk = sg[8 * kTile + threadIdx.x], wk = sg[9 * kTile + threadIdx.x];
        Sv = uk.x; sv = uk.y; Sw = wk.x; sw = wk.y;
        Tv = tv = Tw = tw = 0.f;
      }
      const int r0 = 8 * c, rn = min(8, m - r0);
#pragma unroll
      for (int r = 0; r < 8; r += 2) {
        if (r < rn) {
          const float2 v = sg[r * kTile + threadIdx.x];
          pair_fma(Sv, sv, cp[r0 + r], v.x, v.y);
          pair_fma(Sw, sw, cq[r0 + r], v.x, v.y);
        }
        if (r + 1 < rn) {
          const float2 v = sg[(r + 1) * kTile + threadIdx.x];
          pair_fma(Tv, tv, cp[r0 + r + 1], v.x, v.y);
          pair_fma(Tw, tw, cq[r0 + r + 1], v.x, v.y);
        }
      }
      ring_release(R, q);
      const int64_t k = (blockIdx.x + (q / nch) * gridDim.x) * kTile + threadIdx.x;
      if (c == nch - 1 && k < n) {
        pair_add(Sv, sv, Tv, tv);
        pair_add(Sw, sw, Tw, tw);
        const float2 a = norm_pair(Sv, sv);
        float P = 0.f, pl = 0.f;
        pair_fma(P, pl, inv_s, a.x, a.y);
        const float2 vk = norm_pair(P, pl);
        u[k] = vk;
        pair_fma(Sw, sw, hneg, vk.x, vk.y);
        const float2 wk2 = norm_pair(Sw, sw);
        wn[k] = wk2;
        pair_fma(Sn, sn, wk2, wk2.x, wk2.y);
      }
    }
  }
  __syncthreads();
  double t = (double)Sn + (double)sn;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0 && wid < kConsumers) sh[wid] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int q = 0; q < kConsumers; ++q) sum += sh[q];
    partial[blockIdx.x] = sum;
  }
}

// v *= 1 / sqrt(nrm2[0]) (0 if the norm is 0) in pair arithmetic, also written to v2 as
// FP64 values: normalises the pending vector and stages it as the preconditioner's input
__global__ void k_scale_norm(int64_t n, float2* __restrict__ v, double* __restrict__ v2,
                             const double* __restrict__ nrm2) {
  const double r = sqrt(fmax(nrm2[0], 0.0));
  const float2 f = to_pair(r > 0.0 ? 1.0 / r : 0.0);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = v[k];
    float P = 0.f, pl = 0.f;
    pair_fma(P, pl, f, a.x, a.y);
    const float2 t = norm_pair(P, pl);
    v[k] = t;
    v2[k] = from_pair(t);
  }
}

// v = pairs of a * f, v2 = a * f in FP64 (the first basis vector r / ||r||)
__global__ void k_pair_scaled(int64_t n, const double* __restrict__ a, double f,
                              float2* __restrict__ v, double* __restrict__ v2) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double t = a[k] * f;
    v[k] = to_pair(t);
    v2[k] = t;
  }
}

// b = pairs of a (the Krylov vector K z for the sweep)
__global__ void k_to_pair(int64_t n, const double* __restrict__ a, float2* __restrict__ b) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = to_pair(a[k]);
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

// x += sum_i y[i] Z_i (y staged in shared memory; the basis loads of one index go
// out eight at a time, the sum keeps the order i = 0, 1, ...)
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
  // the basis V as FP32 pairs (8 bytes an entry, the FP64 layout's size); Z in FP64
  float2* V = reinterpret_cast<float2*>(h->gm_V.p);
  double* Z = h->gm_Z;
  // basis vectors start on 64-byte boundaries
  const int64_t ld = (n + 7) / 8 * 8;
  double* w = h->kw;
  float2* wp = reinterpret_cast<float2*>(h->gm_wp.p);   // w as pairs for the sweep
  AMG_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  c.dots(b, b, S_BB);
  const double bnorm = std::sqrt(read_scalar(h, S_BB));
  if (bnorm == 0.0) { st->iterations = 0; return AMG_OK; }
  // coef (device, read back once a step): the sweep's dots with u at [0, kMaxDots),
  // with w at [kMaxDots, 2 kMaxDots), then s, h, 1/s, ||w'||^2
  constexpr int kS = 2 * kMaxDots;
  DBuf<double> coef, ydev;
  coef.alloc(kS + 8);
  ydev.alloc(kMaxDots);
  // H by columns: Hc[j * (m + 1) + i] = H(i, j); rotated in place once a column is final
  std::vector<double> Hc((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), hb(kS + 8), tmp(m + 1);
  // the sweep's kernels: kThreads threads a CTA, the ring in dynamic shared memory,
  // kCtasPerSm CTAs an SM
  int dev = 0, sms = 0;
  AMG_CUDA(cudaGetDevice(&dev));
  AMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  AMG_CUDA(cudaFuncSetAttribute(k_mdot2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kStreamSmem));
  AMG_CUDA(cudaFuncSetAttribute(k_dcgs2_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kStreamSmem));
  const int64_t ntiles = (n + kTile - 1) / kTile;
  const int ublocks = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)kCtasPerSm * sms));
  auto mdot2 = [&](int rows, const float2* u, const float2* wv) {
    const int grows = (rows + kMdotG - 1) / kMdotG;
    const int cols = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)kCtasPerSm * sms / grows, ntiles));
    k_mdot2<<<dim3(cols, grows), kThreads, kStreamSmem, s>>>(n, ld, rows, V, u, wv, h->red,
                                                          h->flag.p);
    k_mdot_final<<<(2 * rows + 7) / 8, 256, 0, s>>>(h->red, cols, rows, 2, kMaxDots, coef.p);
    h->launches += 2;
  };
  int it = 0;
  double rel = 1.0;
  bool conv = false;
  auto col = [&](int j) { return Hc.data() + (size_t)j * (m + 1); };
  // rotations 0..j-1 on column c[0..j+1], then the one that zeroes c[j+1]
  auto rotate = [&](double* cj, int j, double& ck, double& sk) {
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * cj[i] + sn[i] * cj[i + 1];
      cj[i + 1] = -sn[i] * cj[i] + cs[i] * cj[i + 1];
      cj[i] = t;
    }
    const double den = std::hypot(cj[j], cj[j + 1]);
    ck = cj[j] / den;
    sk = cj[j + 1] / den;
    cj[j] = den;
    cj[j + 1] = 0.0;
  };
  auto commit = [&](int j) {
    rotate(col(j), j, cs[j], sn[j]);
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
  };
  auto read_coef = [&](int cnt) {
    AMG_CUDA(cudaMemcpyAsync(hb.data(), coef.p, cnt * sizeof(double), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
  };
  // z_j = M u_j, the pressure projection of z_j and w = K z_j run on fixed vectors (u_j
  // staged in kr, z_j in kz) as one graph launch per step, captured once per solve: the
  // preconditioner's short coarse-level kernels then run back to back after the host's
  // synchronisation of the step before
  double* ur = h->kr;
  double* zr = h->kz;
  // the FP32 cycle's operator products in FP32 pairs for the velocity block (the
  // residual at each restart and at exit stays FP64)
  float* pf = h->L[0]->val2.p ? h->kpf.p : nullptr;
  auto step = [&]() {
    precond(h, ur, zr);
    project_pressure(h, c, zr);
    if (pf) apply_K_pair(h, zr, pf, w);
    else apply_K(h, zr, w);
  };
  cudaGraphExec_t exec = nullptr;
  struct ExecGuard {
    cudaGraphExec_t& e;
    ~ExecGuard() { if (e) cudaGraphExecDestroy(e); }
  } exec_guard{exec};
  int64_t per_step = 0;
  bool tried = !h->opt.use_graphs || h->iter_graph_failed;
  auto run_step = [&]() {
    if (!tried) {
      tried = true;
      const int64_t l0 = h->launches;
      cudaGraph_t gr = nullptr;
      bool capturing = false;
      try {
        AMG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        capturing = true;
        step();
        capturing = false;
        AMG_CUDA(cudaStreamEndCapture(s, &gr));
        AMG_CUDA(cudaGraphInstantiate(&exec, gr, 0));
        per_step = h->launches - l0;
      } catch (const Error&) {
        if (capturing) {
          cudaGraph_t junk = nullptr;
          cudaStreamEndCapture(s, &junk);
          if (junk) cudaGraphDestroy(junk);
        }
        cudaGetLastError();
        exec = nullptr;
        h->iter_graph_failed = true;   // plain launches from here on
      }
      if (gr) cudaGraphDestroy(gr);
      h->launches = l0;
    }
    if (exec) {
      AMG_CUDA(cudaGraphLaunch(exec, s));
      h->launches += per_step;
    } else {
      step();
    }
  };
  while (it < h->opt.max_iterations && !conv) {
    // r = b - K x, u_0 = r / ||r|| (its own sweep makes it exactly unit)
    apply_K(h, x, w);
    k_sub<<<gridr(n), 256, 0, s>>>(n, b, w, w);
    h->launches++;
    c.dots(w, w, S_T0);
    const double beta = std::sqrt(read_scalar(h, S_T0));
    if (beta == 0.0) { conv = true; rel = 0.0; break; }
    k_pair_scaled<<<gridr(n), 256, 0, s>>>(n, w, 1.0 / beta, V, ur);
    h->launches++;
    std::fill(Hc.begin(), Hc.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    double rho = beta;   // the norm that scaled the pending vector u_j
    int jused = 0;
    for (int j = 0; j < m; ++j) {
      float2* uj = V + (int64_t)j * ld;
      double* zj = Z + (int64_t)j * ld;
      run_step();
      launch_copy(zr, zj, n, s, h);
      k_to_pair<<<gridr(n), 256, 0, s>>>(n, w, wp);
      h->launches++;
      // one sweep: dots of rows 0..j with u_j and w, then the update of u_j to v_j and of
      // w to the next pending vector u_{j+1} (row j + 1), normalised on the device
      {
        mdot2(j + 1, uj, wp);
        k_dcgs2_coef<<<1, 32, 0, s>>>(j, coef.p);
        float2* un = V + (int64_t)(j + 1) * ld;
        k_dcgs2_update<<<ublocks, kThreads, kStreamSmem, s>>>(n, ld, j, V, uj, wp, un, coef.p,
                                                           h->red, h->flag.p);
        k_final<<<1, 256, 0, s>>>(h->red, ublocks, 1, coef.p + kS + 3);
        k_scale_norm<<<gridr(n), 256, 0, s>>>(n, un, ur, coef.p + kS + 3);
        h->launches += 4;
      }
      read_coef(kS + 8);
      // u_j = s v_j + sum_{i<j} p_i v_i, and w'_{j-1} = rho u_j: column j - 1 is final
      const double sj = hb[kS], hjj = hb[kS + 1];
      if (j == 0) {
        g[0] = rho * sj;
      } else {
        double* cp = col(j - 1);
        for (int i = 0; i < j; ++i) cp[i] += rho * hb[i];
        cp[j] = rho * sj;
        commit(j - 1);
        rel = std::fabs(g[j]) / bnorm;
      }
      // column j before the reorthogonalisation of u_{j+1}: H(j+1, j) = ||w'||
      rho = std::sqrt(std::max(hb[kS + 3], 0.0));
      double* cj = col(j);
      for (int i = 0; i < j; ++i) cj[i] = hb[kMaxDots + i];
      cj[j] = hjj;
      cj[j + 1] = rho;
      ++it;
      jused = j + 1;
      std::copy(cj, cj + j + 2, tmp.begin());
      double ck, sk;
      rotate(tmp.data(), j, ck, sk);
      const double est = std::fabs(sk * g[j]) / bnorm;
      if (est > tol && j + 1 < m && it < h->opt.max_iterations) continue;
      // stopping: reorthogonalise u_{j+1} against rows 0..j now, making column j final
      {
        const float2* un = V + (int64_t)(j + 1) * ld;
        mdot2(j + 2, un, un);
      }
      read_coef(j + 2);
      std::copy(cj, cj + j + 2, tmp.begin());
      const double gj = g[j];
      double pp = 0.0;
      for (int i = 0; i <= j; ++i) {
        cj[i] += rho * hb[i];
        pp += hb[i] * hb[i];
      }
      const double hnext = rho * std::sqrt(std::max(hb[j + 1] - pp, 0.0));
      cj[j + 1] = hnext;
      commit(j);
      rel = std::fabs(g[j + 1]) / bnorm;
      if (!std::isfinite(rel)) fail(AMG_ERR_BREAKDOWN, "non-finite residual in FGMRES");
      if (rel <= tol || j + 1 >= m || it >= h->opt.max_iterations || hnext == 0.0) {
        conv = rel <= tol;
        break;
      }
      // the estimate before the reorthogonalisation was too optimistic: go on, and let
      // the next sweep finalise column j as usual
      std::copy(tmp.begin(), tmp.begin() + j + 2, cj);
      g[j] = gj;
      g[j + 1] = 0.0;
    }
    // y = R^{-1} g (R: the rotated H, upper triangular), x += Z y
    std::vector<double> y(jused);
    for (int i = jused - 1; i >= 0; --i) {
      double t = g[i];
      for (int k = i + 1; k < jused; ++k) t -= col(k)[i] * y[k];
      y[i] = t / col(i)[i];
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
      ensure(h->gm_wp, ld);
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
