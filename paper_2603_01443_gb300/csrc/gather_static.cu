// cc_gather_static: the sampled-amplitude gather without any allocation.
//
// cc_gather stages the caller's host indices and the gathered amplitudes in
// the library's scratch area, which it grows with cudaMalloc on demand.  Some
// callers cannot allow that: a process whose device memory is owned by
// another allocator (a framework's caching allocator, a fixed memory budget
// set at start-up), or a latency-sensitive loop that cannot afford the
// device-wide synchronisation cudaMalloc and cudaFree may imply.  This entry
// point does the same gather through a fixed array that is part of the
// library image itself, so it never allocates device memory.
//
// The array (CC_GATHER_STATIC_MAX indices and amplitudes, 1.5 MiB) lives in
// every GPU that loads the library until the process exits.  Host code cannot
// use the array's name as a device address: every call resolves the address
// with cudaGetSymbolAddress while the caller's device is current.  The lookup
// is not cached, so a device reset that loads the library's module again (at
// a new address) cannot leave a stale pointer behind.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace {

constexpr int64_t kMax = CC_GATHER_STATIC_MAX;
constexpr size_t kIdxBytes = kMax * sizeof(int64_t);   // 512 KiB of indices
constexpr size_t kValBytes = kMax * 16;                 // 1 MiB of amplitudes (complex128 or complex64)

// Indices at [0, kIdxBytes), gathered amplitudes at [kIdxBytes, kIdxBytes + kValBytes).
// Every entry a call reads is written by that same call first, so nothing in
// the array has to start at zero.
static __device__ __align__(256) unsigned char g_gather_scratch[kIdxBytes + kValBytes];

// Device address of g_gather_scratch on the current device, looked up afresh
// on every call.
cc_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    cudaGetLastError();
    return cc::fail(CC_ECUDA, "cc_gather_static: no current CUDA device");
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_gather_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return cc::fail(CC_ECUDA, std::string("cc_gather_static: cudaGetSymbolAddress failed: ") +
                                  cudaGetErrorString(e));
  }
  *out = p;
  return CC_OK;
}

}  // namespace

extern "C" cc_status cc_gather_static(const void* psi, int64_t n_amp, int32_t precision,
                                      const int64_t* idx, int64_t n_idx, void* out, void* stream) {
  using namespace cc;
  if (!psi || !idx || !out) return fail(CC_EINVAL, "cc_gather_static: NULL argument");
  if (precision != CC_C64 && precision != CC_C128)
    return fail(CC_EINVAL, "cc_gather_static: unknown precision");
  if (n_idx < 0 || n_idx > kMax)
    return fail(CC_ERANGE, "cc_gather_static: n_idx = " + std::to_string(n_idx) +
                               " exceeds the built-in maximum of " + std::to_string(kMax) +
                               " (use cc_gather for larger samples)");
  for (int64_t i = 0; i < n_idx; ++i)
    if (idx[i] < 0 || idx[i] >= n_amp)
      return fail(CC_ERANGE, "cc_gather_static: index " + std::to_string(idx[i]) +
                                 " outside [0, n_amp)");
  if (n_idx == 0) return CC_OK;
  cc_status st = check_device();
  if (st != CC_OK) return st;
  void* base = nullptr;
  st = scratch_address(&base);
  if (st != CC_OK) return st;
  int64_t* idx_dev = static_cast<int64_t*>(base);
  void* val_dev = static_cast<unsigned char*>(base) + kIdxBytes;
  const size_t ab = precision == CC_C128 ? 16 : 8;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(idx_dev, idx, n_idx * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess)
    return fail(CC_ECUDA, std::string("cc_gather_static: copy: ") + cudaGetErrorString(e));
  st = launch_gather(psi, precision, idx_dev, n_idx, val_dev, stream);
  if (st != CC_OK) return st;
  e = cudaMemcpyAsync(out, val_dev, n_idx * ab, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess)
    return fail(CC_ECUDA, std::string("cc_gather_static: copy: ") + cudaGetErrorString(e));
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess)
    return fail(CC_ECUDA, std::string("cc_gather_static: ") + cudaGetErrorString(e));
  return CC_OK;
}
