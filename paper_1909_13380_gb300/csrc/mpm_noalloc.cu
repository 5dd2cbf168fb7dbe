// mpm_noalloc.cu -- mpm_sort_keys_static: the stable key sort with its
// scratch in a fixed device array, for callers that cannot allocate device
// memory (their own allocator holds the GPU's free memory, or they must not
// allocate once running).  It is a service of the library with no
// counterpart in the paper.
//
// The scratch lives in a file-scope __device__ array.  In host code that
// array's name is only a host-side stand-in, so every call looks up its
// device address with cudaGetSymbolAddress for the device that is current.
// The address is not cached: a context that is torn down and created again
// (cudaDeviceReset, for one) may load the module at another address, and a
// cached pointer would then be a dangling one.  The lookup is cheap once the
// module is loaded; the first call on a device loads it.  Every call shares
// the array; the sort writes each scratch word before reading it, so nothing
// has to be cleared between calls, but calls that overlap on the GPU race.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpm.h"
#include "mpm_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(22) << 20;  // 22 MiB

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

size_t keys_bytes() { return ((size_t)4 * MPM_SORT_STATIC_MAX_KEYS + 255) & ~size_t(255); }

}  // namespace

extern "C" mpm_status mpm_sort_keys_static(const uint32_t *d_keys, int32_t *d_perm, int64_t n, int32_t key_bits,
                                           void *stream) {
  if (n < 0 || n > MPM_SORT_STATIC_MAX_KEYS || key_bits < 1 || key_bits > 32 || (n > 0 && (!d_keys || !d_perm)))
    return MPM_ERR_ARG;
  if (n == 0) return MPM_OK;
  // the carve-up below must fit the fixed array for the largest n
  if (keys_bytes() + mpm::sort_scratch_bytes(MPM_SORT_STATIC_MAX_KEYS) > kScratchBytes) return MPM_ERR_STATE;
  // the array's address in the current device's context, looked up afresh
  void *base = nullptr;
  if (cudaGetSymbolAddress(&base, g_sort_scratch) != cudaSuccess || !base) return MPM_ERR_CUDA;
  uint32_t *keys_out = (uint32_t *)base;
  void *scratch = (char *)base + keys_bytes();
  cudaError_t e = mpm::sort_pairs(d_keys, nullptr, keys_out, d_perm, n, key_bits, scratch, (cudaStream_t)stream);
  return e == cudaSuccess ? MPM_OK : MPM_ERR_CUDA;
}
