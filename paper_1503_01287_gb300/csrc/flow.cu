// The multicolour block Gauss-Seidel sweep of one level (Sec. 3.3) as a single
// launch, in dataflow order.
//
// The sweep's result is defined colour by colour: every row of colour c is
// updated from the new values of its lower-colour neighbours and the old values
// of the others.  The colour chain launches one kernel per colour; here one
// cooperative launch walks the rows in colour-major order and each row waits
// only for the neighbours whose new values it reads:
//
//   * the level's stored (colour-major) copy is cut into chunks of 32/G rows,
//     never across a colour boundary; warp w takes chunks w, w + W, w + 2W, ...
//     in increasing order (decreasing for the reverse sweep), all warps
//     resident (cooperative launch);
//   * every column index carries two bits: the neighbour has a lower colour or a
//     higher one; a forward sweep waits on the lower ones, a reverse sweep on the
//     higher ones.  A waited-on row lies in an earlier chunk, held by a resident
//     warp that reaches it after its own earlier chunks, so by induction over
//     the chunk order every wait ends;
//   * new values travel through a tagged exchange array: each 32-bit piece of a
//     node's new value is stored beside the sweep number in one 64-bit word
//     (single-copy atomic, relaxed accesses at gpu scope), so a reader that sees
//     the current sweep number in a word has that piece's new value, whatever
//     order the writer's stores reach L2 in: no fence on the path from one row
//     to the next.  The sweep number lives on the device (state[0]); the last
//     CTA to finish advances it, so captured graphs replay without host
//     arguments, and the exchange array is never cleared;
//   * the iterate itself is updated in place for the kernels after the sweep.
//     A neighbour that is not waited on (the other direction) cannot change
//     while it is read: its own row waits for this row's new value, which is
//     computed from these reads.
//
// Every wait is bounded: a thread that has polled kFlowSpins times in total
// records a timeout in the error word and waits no more (the kernel always
// ends; the host reports AMG_ERR_TIMEOUT).  With the chain's lanes per row the
// per-lane summation order is the chain kernel's, so the results are bitwise
// those of the colour chain.
#include <algorithm>
#include <cstring>
#include <vector>

#include "amg_internal.cuh"
#include "vec.cuh"

namespace amgp2 {

namespace {

constexpr unsigned kLowerBit = 0x80000000u;    // the neighbour has a lower colour
constexpr unsigned kHigherBit = 0x40000000u;   // the neighbour has a higher colour
constexpr unsigned kNodeMask = 0x3fffffffu;
constexpr unsigned kNoBlock = 0xffffffffu;
constexpr int kFlowThreads = 256;
constexpr int kFlowSpins = 1 << 20;            // polls per thread, over the whole launch

__device__ __forceinline__ unsigned flow_ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// The exchange array holds 4 (FP32) or 8 (FP64) 64-bit words a node: word c of
// FP32 is (component c, sweep number); FP64 splits component c into words 2c
// (high half) and 2c + 1 (low half).  Tag in the upper 32 bits.
template <typename T>
struct Tagged;

template <>
struct Tagged<float> {
  static constexpr int kWords = 4;
  __device__ static void put(unsigned long long* w, int i, unsigned ep, float a, float b,
                             float c) {
    const unsigned long long t = (unsigned long long)ep << 32;
    unsigned long long* p = w + 4 * (size_t)i;
    asm volatile("st.relaxed.gpu.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p),
                 "l"(t | __float_as_uint(a)), "l"(t | __float_as_uint(b)),
                 "l"(t | __float_as_uint(c)), "l"(t)
                 : "memory");
  }
  // true (and the values) once all three pieces carry the sweep number
  __device__ static bool get(const unsigned long long* w, int j, unsigned ep, float& a, float& b,
                             float& c) {
    unsigned long long w0, w1, w2, w3;
    asm volatile("ld.relaxed.gpu.global.v4.b64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(w0), "=l"(w1), "=l"(w2), "=l"(w3)
                 : "l"(w + 4 * (size_t)j)
                 : "memory");
    a = __uint_as_float((unsigned)w0);
    b = __uint_as_float((unsigned)w1);
    c = __uint_as_float((unsigned)w2);
    return (unsigned)(w0 >> 32) == ep && (unsigned)(w1 >> 32) == ep &&
           (unsigned)(w2 >> 32) == ep;
  }
};

template <>
struct Tagged<double> {
  static constexpr int kWords = 8;
  __device__ static void put(unsigned long long* w, int i, unsigned ep, double a, double b,
                             double c) {
    const unsigned long long t = (unsigned long long)ep << 32;
    unsigned long long* p = w + 8 * (size_t)i;
    const unsigned long long ua = __double_as_longlong(a), ub = __double_as_longlong(b),
                             uc = __double_as_longlong(c);
    asm volatile("st.relaxed.gpu.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p),
                 "l"(t | (ua >> 32)), "l"(t | (ua & 0xffffffffull)), "l"(t | (ub >> 32)),
                 "l"(t | (ub & 0xffffffffull))
                 : "memory");
    asm volatile("st.relaxed.gpu.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p + 4),
                 "l"(t | (uc >> 32)), "l"(t | (uc & 0xffffffffull)), "l"(t), "l"(t)
                 : "memory");
  }
  __device__ static bool get(const unsigned long long* w, int j, unsigned ep, double& a,
                             double& b, double& c) {
    unsigned long long q[6], d0, d1;
    const unsigned long long* p = w + 8 * (size_t)j;
    asm volatile("ld.relaxed.gpu.global.v4.b64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(q[0]), "=l"(q[1]), "=l"(q[2]), "=l"(q[3])
                 : "l"(p)
                 : "memory");
    asm volatile("ld.relaxed.gpu.global.v4.b64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(q[4]), "=l"(q[5]), "=l"(d0), "=l"(d1)
                 : "l"(p + 4)
                 : "memory");
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 6; ++k) ok = ok && (unsigned)(q[k] >> 32) == ep;
    a = __longlong_as_double((long long)((q[0] << 32) | (q[1] & 0xffffffffull)));
    b = __longlong_as_double((long long)((q[2] << 32) | (q[3] & 0xffffffffull)));
    c = __longlong_as_double((long long)((q[4] << 32) | (q[5] & 0xffffffffull)));
    return ok;
  }
};

// L2 prefetch of [lo, hi) rounded down to 16-byte boundaries at both ends (so it
// never reaches past the range; a hint only)
__device__ __forceinline__ void flow_prefetch_l2(const void* lo, const void* hi) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(lo) & ~uintptr_t(15);
  const uintptr_t e = reinterpret_cast<uintptr_t>(hi) & ~uintptr_t(15);
  if (e > a)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a))
                 : "memory");
}

// Counts one round of polls against the thread's budget; false once it is spent
// (recorded in the error word) or another thread has recorded an error: the
// thread then waits no more.
__device__ __forceinline__ bool flow_spin(int& spins, int* err) {
  if (++spins > kFlowSpins) {
    if (spins == kFlowSpins + 1) atomicOr(err, 4);
    spins = kFlowSpins + 1;
    return false;
  }
  if ((spins & 255) == 0 && *reinterpret_cast<volatile int*>(err)) {
    spins = kFlowSpins + 1;
    return false;
  }
  return true;
}

// Column indices of the stored copy with the colour-order bits of each block.
__global__ void k_flow_cols(int nrows, const int* __restrict__ rows,
                            const int* __restrict__ rowptr, const int* __restrict__ col,
                            const int* __restrict__ colour, unsigned* __restrict__ fcol) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nrows;
       g += gridDim.x * blockDim.x) {
    const int ci = colour[rows[g]];
    for (int k = rowptr[g]; k < rowptr[g + 1]; ++k) {
      const int j = col[k];
      const int cj = colour[j];
      fcol[k] = (unsigned)j | (cj < ci ? kLowerBit : 0u) | (cj > ci ? kHigherBit : 0u);
    }
  }
}

// Blocks prefetched per lane: the colour chain kernel's choice (the same
// per-lane summation order).
template <typename T, int G>
constexpr int flow_unroll() {
  return (sizeof(T) == 8) ? (G >= 16 ? 2 : 3) : (G >= 16 ? 3 : 4);
}

template <typename T, int G, int U>
__global__ void __launch_bounds__(kFlowThreads)
    k_gs_flow(int nchunks, const int* __restrict__ chunk, const int* __restrict__ rows,
              const int* __restrict__ rowptr, const unsigned* __restrict__ fcol,
              const T* __restrict__ val, int64_t nnzb, T* x, const T* __restrict__ b,
              const T* __restrict__ dinv, const double* __restrict__ wt,
              unsigned long long* xt, unsigned* state, int reverse, int* err) {
  const int lane = threadIdx.x & 31;
  const int sub = lane / G, gl = lane & (G - 1);
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const unsigned ep = flow_ld_relaxed(state) + 1u;
  const unsigned wbit = reverse ? kHigherBit : kLowerBit;
  const T om = wt ? (T)wt[0] : T(1);   // learned relaxation multiplier (1: plain)
  int spins = 0;
  for (int p = warp; p < nchunks; p += nwarps) {
    const int q = reverse ? nchunks - 1 - p : p;
    const int g = __ldg(chunk + q) + sub;
    const bool active = g < __ldg(chunk + q + 1);
    int i = 0, a = 0, e = 0;
    unsigned j[U];
    T v[U][9];
    T d[9];
    T b0 = T(0), b1 = T(0), b2 = T(0), xi0 = T(0), xi1 = T(0), xi2 = T(0);
#pragma unroll
    for (int u = 0; u < U; ++u) j[u] = kNoBlock;
    if (active) {
      // what no other row of the sweep writes: loaded before any wait
      i = __ldg(rows + g);
      a = __ldg(rowptr + g);
      e = __ldg(rowptr + g + 1);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = a + gl + u * G;
        if (k < e) {
          j[u] = __ldcs(fcol + k);
#pragma unroll
          for (int w = 0; w < 9; ++w) v[u][w] = __ldcs(val + w * nnzb + k);
        }
      }
      if (gl == 0) {
        ld3(b, i, b0, b1, b2);
        ld3(x, i, xi0, xi1, xi2);       // the row's own old value: only this row writes it
        const T* dp = dinv + 12 * (int64_t)i;
        ld3(dp, 0, d[0], d[1], d[2]);
        ld3(dp, 1, d[3], d[4], d[5]);
        ld3(dp, 2, d[6], d[7], d[8]);
      }
    }
    // the block values and columns of this warp's chunk two rounds ahead, into L2
    // (one contiguous range per plane), while this chunk waits and gathers
    if (lane < 10 && p + 2 * nwarps < nchunks) {
      const int pq = p + 2 * nwarps;
      const int qq = reverse ? nchunks - 1 - pq : pq;
      const int k0 = __ldg(rowptr + __ldg(chunk + qq)), k1 = __ldg(rowptr + __ldg(chunk + qq + 1));
      if (lane < 9) flow_prefetch_l2(val + lane * nnzb + k0, val + lane * nnzb + k1);
      else flow_prefetch_l2(fcol + k0, fcol + k1);
    }
    T s0 = T(0), s1 = T(0), s2 = T(0);
    if (active) {
      // neighbour values: the new ones from the exchange array, polled (all of the
      // lane's at once, the late ones again) until they carry this sweep's number;
      // the old ones from the iterate
      T xv[U][3];
      unsigned pend = 0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (j[u] == kNoBlock) continue;
        const int jj = (int)(j[u] & kNodeMask);
        if (j[u] & wbit) {
          if (!Tagged<T>::get(xt, jj, ep, xv[u][0], xv[u][1], xv[u][2])) pend |= 1u << u;
        } else {
          ld3(x, jj, xv[u][0], xv[u][1], xv[u][2]);
        }
      }
      while (pend) {
        if (!flow_spin(spins, err)) break;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if ((pend >> u & 1u) &&
              Tagged<T>::get(xt, (int)(j[u] & kNodeMask), ep, xv[u][0], xv[u][1], xv[u][2]))
            pend &= ~(1u << u);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (j[u] == kNoBlock) continue;
        const T x0 = xv[u][0], x1 = xv[u][1], x2 = xv[u][2];
        s0 = fma(v[u][0], x0, s0); s0 = fma(v[u][1], x1, s0); s0 = fma(v[u][2], x2, s0);
        s1 = fma(v[u][3], x0, s1); s1 = fma(v[u][4], x1, s1); s1 = fma(v[u][5], x2, s1);
        s2 = fma(v[u][6], x0, s2); s2 = fma(v[u][7], x1, s2); s2 = fma(v[u][8], x2, s2);
      }
      // blocks beyond the prefetched U per lane
      for (int k = a + gl + U * G; k < e; k += G) {
        const unsigned f = __ldg(fcol + k);
        const int jj = (int)(f & kNodeMask);
        T x0, x1, x2;
        if (f & wbit) {
          while (!Tagged<T>::get(xt, jj, ep, x0, x1, x2) && flow_spin(spins, err)) {
          }
        } else {
          ld3(x, jj, x0, x1, x2);
        }
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
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (active && gl == 0) {
      const T r0 = b0 - s0, r1 = b1 - s1, r2 = b2 - s2;
      const T n0 = xi0 + om * (d[0] * r0 + d[1] * r1 + d[2] * r2);
      const T n1 = xi1 + om * (d[3] * r0 + d[4] * r1 + d[5] * r2);
      const T n2 = xi2 + om * (d[6] * r0 + d[7] * r1 + d[8] * r2);
      Tagged<T>::put(xt, i, ep, n0, n1, n2);   // for the rows that wait on this one
      st3(x, i, n0, n1, n2);                    // for the kernels after the sweep
    }
  }
  // the last CTA to finish advances the sweep number for the next launch (no
  // CTA reads it after its own start, and every CTA has started by then)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(state + 1, 1u);
    if (done == gridDim.x - 1) {
      atomicExch(state + 1, 0u);
      atomicExch(state, ep);
    }
  }
}

template <typename T, int G>
const void* flow_kernel() {
  return reinterpret_cast<const void*>(k_gs_flow<T, G, flow_unroll<T, G>()>);
}

template <typename T>
const void* flow_kernel_for(int G) {
  switch (G) {
    case 4: return flow_kernel<T, 4>();
    case 8: return flow_kernel<T, 8>();
    case 16: return flow_kernel<T, 16>();
    default: return flow_kernel<T, 32>();
  }
}

// co-resident CTAs of the kernel for (T, G), 0 if cooperative launch is unavailable
template <typename T>
int flow_max_ctas(int G) {
  int dev = 0, sms = 0, coop = 0, per = 0;
  AMG_CUDA(cudaGetDevice(&dev));
  AMG_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return 0;
  AMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, flow_kernel_for<T>(G), kFlowThreads,
                                                    0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms * per;
}

}  // namespace

bool flow_prepare(amg_handle* h, Level& lv) {
  if (lv.ncolours == 0 || !lv.stored) return false;
  if (flow_max_ctas<float>(8) <= 0) return false;
  if (!lv.fcol.p) {
    cudaStream_t s = h->stream;
    lv.fcol.alloc(std::max<int64_t>(lv.nnzb, 1));
    lv.fxt.alloc(8 * (size_t)std::max(lv.n, 1));   // room for the FP64 layout
    lv.fstate.alloc(2);
    AMG_CUDA(cudaMemsetAsync(lv.fxt.p, 0, lv.fxt.bytes(), s));
    AMG_CUDA(cudaMemsetAsync(lv.fstate.p, 0, lv.fstate.bytes(), s));
    k_flow_cols<<<std::max(1, std::min(div_up(lv.n, 256), 152 * 8)), 256, 0, s>>>(
        lv.n, lv.colour_rows, lv.srowptr, lv.scol, lv.colour, lv.fcol);
    AMG_LAUNCH_CHECK();
    h->launches++;
  }
  return true;
}

void flow_set_group(amg_handle* h, Level& lv, int G) {
  const int R = 32 / G;
  std::vector<int> c;
  for (int k = 0; k < lv.ncolours; ++k)
    for (int r = lv.colour_ptr[k]; r < lv.colour_ptr[k + 1]; r += R) c.push_back(r);
  c.push_back(lv.n);
  lv.flow_nchunks = (int)c.size() - 1;
  lv.fchunk.alloc(c.size());
  AMG_CUDA(cudaMemcpyAsync(lv.fchunk.p, c.data(), c.size() * sizeof(int),
                           cudaMemcpyHostToDevice, h->stream));
  AMG_CUDA(cudaStreamSynchronize(h->stream));
  const int want = div_up(lv.flow_nchunks, kFlowThreads / 32);
  lv.flow_grid32 = std::min(want, flow_max_ctas<float>(G));
  lv.flow_grid64 = std::min(want, flow_max_ctas<double>(G));
  lv.flow = G;
}

template <typename T>
void launch_gs_flow(amg_handle* h, Level& lv, T* x, const T* b, const T* val, const T* dinv,
                    bool reverse) {
  const int grid = sizeof(T) == 4 ? lv.flow_grid32 : lv.flow_grid64;
  if (grid <= 0) fail(AMG_ERR_UNSUPPORTED, "the one-launch dataflow sweep is not available");
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kFlowThreads);
  cfg.stream = h->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const int* chunk = lv.fchunk.p;
  const int* rows = lv.colour_rows.p;
  const int* rowptr = lv.srowptr.p;
  const unsigned* fcol = lv.fcol.p;
  const double* wt = lv.wt;
  const int rev = reverse ? 1 : 0;
  switch (lv.flow) {
#define AMG_FLOW_LAUNCH(GG)                                                                   \
  AMG_CUDA(cudaLaunchKernelEx(&cfg, k_gs_flow<T, GG, flow_unroll<T, GG>()>, lv.flow_nchunks, \
                              chunk, rows, rowptr, fcol, val, lv.nnzb, x, b, dinv, wt,       \
                              lv.fxt.p, lv.fstate.p, rev, h->flag.p))
    case 4: AMG_FLOW_LAUNCH(4); break;
    case 8: AMG_FLOW_LAUNCH(8); break;
    case 16: AMG_FLOW_LAUNCH(16); break;
    default: AMG_FLOW_LAUNCH(32); break;
#undef AMG_FLOW_LAUNCH
  }
  h->launches++;
}

template void launch_gs_flow<float>(amg_handle*, Level&, float*, const float*, const float*,
                                    const float*, bool);
template void launch_gs_flow<double>(amg_handle*, Level&, double*, const double*,
                                     const double*, const double*, bool);

}  // namespace amgp2
