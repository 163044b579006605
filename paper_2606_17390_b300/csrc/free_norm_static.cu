// FP64 norm of the free entries of a residual vector, with no device allocation of any kind.
//
// This is the norm ||R_free||_2 that the global Newton iteration tests for convergence, in a
// form that needs no solver handle and takes no memory: the reduction's scratch (one partial
// sum per CTA and the CTAs' arrival counter) lives in the file-scope static device array
// below instead of a handle's workspace.  The paper has no counterpart.
//
// Who cannot allocate: a caller that holds a residual and a Dirichlet mask but no handle
// (R from another code, or from a handle it must not touch), while the device memory is
// held by a caching allocator (PyTorch's) or is full — e.g. an error path that reports the
// residual after an out-of-memory failure, or a serving loop that has pinned its memory
// budget.  cudaMalloc there could fail, or could synchronise the device behind the
// caller's back.
//
// Limits and rules:
// * n_dof <= HFE_FREE_NORM_STATIC_MAX_DOF (4,194,304 = 1,024 CTAs x 4,096 dofs); larger
//   calls are rejected with HFE_EINVAL before anything is launched.
// * The scratch is one array per device, shared by every call on that device: calls that
//   overlap (two host threads, or two streams with no ordering between them) race on it.
//   Serialise them, e.g. on one stream.
// * Only the arrival counter must be zero when a launch starts.  The module load zeroes it,
//   every call clears it again with cudaMemsetAsync on the caller's stream before its
//   launch, and the last CTA leaves it at zero.  The partial sums are written before they
//   are read and need no initial value.
// * Every call looks up the scratch's device address with cudaGetSymbolAddress, with the
//   caller's device current, and passes it to the kernel.  The address is not cached: a
//   context that is destroyed and created again (cudaDeviceReset) reloads the module, and
//   the array may then sit elsewhere.  The first call on a device (or in a new context) may
//   load the module and so may take memory once; make it before any stream capture begins.
// * An error left pending by the caller's earlier CUDA work is not consumed: the call then
//   returns HFE_ECUDA without launching anything, and the error stays for the caller.
#include <cuda_runtime.h>

#include <cstdint>

#include "hfe.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;                                          // dofs per thread
constexpr int64_t kChunk = (int64_t)kThreads * kItems;              // dofs per CTA
constexpr int kMaxCtas = (int)(HFE_FREE_NORM_STATIC_MAX_DOF / kChunk);
static_assert((int64_t)kMaxCtas * kChunk == HFE_FREE_NORM_STATIC_MAX_DOF, "limit must be whole CTAs");
constexpr int kTicketSlot = kMaxCtas;                               // counter in its own 256-byte tail
constexpr int kScratchDoubles = kMaxCtas + 32;                      // 8,448 bytes

// partial sums [0, kMaxCtas); arrival counter (an unsigned) at double slot kTicketSlot
static __device__ __align__(256) double g_norm_scratch[kScratchDoubles];

__device__ __forceinline__ double warp_total(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA in a fixed order; the result is valid in thread 0.
__device__ __forceinline__ double cta_total(double v) {
  __shared__ double w_part[kThreads / 32];
  v = warp_total(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) w_part[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = (l < kThreads / 32) ? w_part[l] : 0.0;
    v = warp_total(v);
  }
  return v;
}

// CTA b sums the squares of the free entries among dofs [b*kChunk, (b+1)*kChunk) in a fixed
// order; the last CTA to arrive adds the partials in index order and writes the square root.
// The partition does not depend on the device, so the result is reproducible bit for bit.
__global__ void __launch_bounds__(kThreads) free_norm_static_kernel(const double* __restrict__ r,
                                                                    const uint8_t* __restrict__ free_mask,
                                                                    int64_t n_dof, double* __restrict__ scratch,
                                                                    double* __restrict__ norm_out) {
  const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int64_t d = base + (int64_t)k * kThreads;
    if (d < n_dof && free_mask[d] != 0) {
      const double v = r[d];
      s += v * v;
    }
  }
  s = cta_total(s);
  __shared__ bool is_last;
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch + kTicketSlot);
  if (threadIdx.x == 0) {
    scratch[blockIdx.x] = s;
    __threadfence();
    is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double t = 0.0;
  for (unsigned k = threadIdx.x; k < gridDim.x; k += kThreads) t += __ldcg(scratch + k);
  t = cta_total(t);
  if (threadIdx.x == 0) {
    *norm_out = sqrt(t);
    *ticket = 0u;
  }
}

// True when p is device (or managed) memory of device dev.  Called only while no error is
// pending, so the error that cudaPointerGetAttributes raises for a pointer CUDA does not
// know is the only one consumed here.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" hfe_status hfe_free_norm_static(const double* r, const uint8_t* free_mask, int64_t n_dof,
                                           double* norm_out, void* cuda_stream) {
  if (norm_out == nullptr || n_dof < 0 || n_dof > HFE_FREE_NORM_STATIC_MAX_DOF) return HFE_EINVAL;
  if (n_dof > 0 && (r == nullptr || free_mask == nullptr)) return HFE_EINVAL;
  if (cudaPeekAtLastError() != cudaSuccess) return HFE_ECUDA;   // the caller's error: left pending
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return HFE_ECUDA;
  if (!on_device(norm_out, dev)) return HFE_EINVAL;
  if (n_dof > 0 && (!on_device(r, dev) || !on_device(free_mask, dev))) return HFE_EINVAL;
  // the scratch's address in the current context (looked up on every call, see the header)
  void* sym = nullptr;
  if (cudaGetSymbolAddress(&sym, g_norm_scratch) != cudaSuccess || sym == nullptr) {
    cudaGetLastError();
    return HFE_ECUDA;
  }
  double* scratch = static_cast<double*>(sym);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (n_dof == 0) {   // empty sum: the norm is +0.0 (all-zero bits)
    if (cudaMemsetAsync(norm_out, 0, sizeof(double), s) == cudaSuccess) return HFE_OK;
    cudaGetLastError();
    return HFE_ECUDA;
  }
  if (cudaMemsetAsync(scratch + kTicketSlot, 0, sizeof(unsigned), s) != cudaSuccess) {
    cudaGetLastError();
    return HFE_ECUDA;
  }
  const unsigned blocks = (unsigned)((n_dof + kChunk - 1) / kChunk);   // <= kMaxCtas by the check above
  free_norm_static_kernel<<<blocks, kThreads, 0, s>>>(r, free_mask, n_dof, scratch, norm_out);
  // no error was pending at entry, so one raised now is this launch's own
  return cudaGetLastError() == cudaSuccess ? HFE_OK : HFE_ECUDA;
}
