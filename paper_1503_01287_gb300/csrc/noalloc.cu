// amg_apply_preconditioner_noalloc: the preconditioner application of
// amg_apply_preconditioner without any device allocation inside the call.
//
// amg_apply_preconditioner stages its input and output vectors in buffers the
// handle allocates on its first call.  Some callers cannot let a library call
// allocate: applications whose framework allocator (a caching allocator, or a
// pool sized at start-up) already holds nearly all of the device memory, where
// a cudaMalloc inside the call fails or forces the framework to release memory,
// and loops with a latency budget, where cudaMalloc and cudaFree may
// synchronise the whole device.  This variant stages the two vectors in one
// file-scope static device array instead, so after amg_setup no call allocates.
#include <cstdio>
#include <mutex>

#include "amg_internal.cuh"

namespace amgp2 {

namespace {

// Two padded vectors (4 * n_nodes + n_pres entries each) of up to this many
// doubles: 2 x 10 MiB.  Every GPU that loads the library holds the array until
// the process exits.
constexpr int64_t kNoallocMaxEntries = 1310720;
constexpr int64_t kNoallocStride = kNoallocMaxEntries;   // a multiple of 32 doubles

static __device__ __align__(256) double g_noalloc_scratch[2 * kNoallocMaxEntries];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kMaxDevices] = {};

// The device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is obtained with
// cudaGetSymbolAddress, once per device, with that device current.
double* noalloc_scratch() {
  int dev = 0;
  AMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) fail(AMG_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    double* p = nullptr;
    AMG_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch));
    g_noalloc_addr[dev] = p;
  }
  return g_noalloc_addr[dev];
}

}  // namespace

void apply_preconditioner_noalloc(amg_handle* h, const double* r, double* z) {
  Level& lv = *h->L[0];
  const int64_t n4 = lv.dofs4();
  if (n4 > kNoallocMaxEntries) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "level 0 needs %lld padded entries per vector; the static scratch of "
             "amg_apply_preconditioner_noalloc holds at most %lld",
             (long long)n4, (long long)kNoallocMaxEntries);
    fail(AMG_ERR_INVALID, buf);
  }
  double* s = noalloc_scratch();
  double* sr = s;
  double* sz = s + kNoallocStride;
  // both staging vectors are fully overwritten (the cycle starts from zero), so
  // whatever an earlier call left in the array does not matter
  launch_to_padded(r, sr, lv.n, lv.np, h->stream, h);
  if (h->opt.precision == AMG_FP32) precondition_device<float>(h, sr, sz);
  else precondition_device<double>(h, sr, sz);
  launch_from_padded(sz, z, lv.n, lv.np, h->stream, h);
  AMG_LAUNCH_CHECK();
  AMG_CUDA(cudaStreamSynchronize(h->stream));
  check_wait_flag(h, "the preconditioner application");
}

}  // namespace amgp2
