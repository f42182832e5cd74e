// Allocation-free variant of the float64 mass reduction of thor_diag.
//
// Who needs it: callers that must not call cudaMalloc, either because an
// outer framework owns the whole device-memory budget (a caching allocator
// that other allocations would fragment or overrun), or because cudaMalloc
// synchronises the device and would stall work queued on other streams of a
// latency-critical loop. They own their arrays and call this entry point,
// which allocates nothing.
//
// The two-pass reduction (per-block compensated partial sums, then one
// ordered compensated sum of the partials) follows thor_diag's scheme with
// its own blocking (contiguous chunks per block), so the two agree to
// rounding; here the partials live in a file-scope device array of fixed
// size instead of the state's own scratch. Device code names that array directly; host code
// only ever passes its device address, obtained once per device with
// cudaGetSymbolAddress (the host-side symbol is a stand-in, not a device
// address).
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>

#include "../../include/thor.h"

namespace thor {
namespace {

constexpr int kThreads = 256;
constexpr size_t kChunk = 16384;           // elements summed by one block
constexpr int kMaxBlocks = 4096;           // partial sums the static array holds
constexpr int kMaxDevices = 64;

// 4096 partial sums + 1 result slot; every call overwrites the slots it uses
static __device__ __align__(256) double g_partials[kMaxBlocks + 1];

std::atomic<double*> g_dev_ptr[kMaxDevices];

__global__ void __launch_bounds__(kThreads) k_mass_partial(const double* __restrict__ rho,
                                                           const double* __restrict__ vol,
                                                           size_t n, double* part) {
  const size_t base = (size_t)blockIdx.x * kChunk;
  const size_t end = base + kChunk < n ? base + kChunk : n;
  double s = 0.0, comp = 0.0;                                 // Kahan
  for (size_t i = base + threadIdx.x; i < end; i += kThreads) {
    double y = rho[i] * vol[i] - comp;
    double t = s + y;
    comp = (t - s) - y;
    s = t;
  }
  __shared__ double sh[kThreads];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_mass_final(const double* part, int nblocks, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0, comp = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    double y = part[b] - comp;
    double t = s + y;
    comp = (t - s) - y;
    s = t;
  }
  *out = s;
}

// device address of g_partials for the current device (set up on first use)
int partials_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return THOR_ECUDA;
  double* p = g_dev_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_partials) != cudaSuccess || !addr) return THOR_ECUDA;
    p = static_cast<double*>(addr);
    g_dev_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return THOR_OK;
}

}  // namespace
}  // namespace thor

extern "C" int thor_mass_noalloc(const double* rho, const double* volume, size_t n,
                                 double* mass_out, void* stream) {
  using namespace thor;
  if (!rho || !volume || !mass_out || n == 0) return THOR_EINVAL;
  if (n > (size_t)kMaxBlocks * kChunk) return THOR_EINVAL;   // beyond the static scratch
  double* part = nullptr;
  int rc = partials_for_current_device(&part);
  if (rc) return rc;
  const int nblocks = (int)((n + kChunk - 1) / kChunk);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_mass_partial<<<nblocks, kThreads, 0, st>>>(rho, volume, n, part);
  k_mass_final<<<1, 32, 0, st>>>(part, nblocks, mass_out);
  return cudaGetLastError() == cudaSuccess ? THOR_OK : THOR_ECUDA;
}
