// mpm_noalloc.cu -- mpm_sort_keys_static: the stable key sort with its
// scratch in a fixed device array, for callers that cannot allocate device
// memory (their own allocator holds the GPU's free memory, or they must not
// allocate once running).  It is a service of the library with no
// counterpart in the paper.
//
// The scratch lives in a file-scope __device__ array.  In host code that
// array's name is only a host-side stand-in, so its device address is looked
// up once per device with cudaGetSymbolAddress (with the device current) and
// cached.  Every call shares the array; the sort writes each scratch word
// before reading it, so nothing has to be cleared between calls, but calls
// that overlap on the GPU race.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/mpm.h"
#include "mpm_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(22) << 20;  // 22 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

size_t keys_bytes() { return ((size_t)4 * MPM_SORT_STATIC_MAX_KEYS + 255) & ~size_t(255); }

}  // namespace

extern "C" mpm_status mpm_sort_keys_static(const uint32_t *d_keys, int32_t *d_perm, int64_t n, int32_t key_bits,
                                           void *stream) {
  if (n < 0 || n > MPM_SORT_STATIC_MAX_KEYS || key_bits < 1 || key_bits > 32 || (n > 0 && (!d_keys || !d_perm)))
    return MPM_ERR_ARG;
  if (n == 0) return MPM_OK;
  // the carve-up below must fit the fixed array for the largest n
  if (keys_bytes() + mpm::sort_scratch_bytes(MPM_SORT_STATIC_MAX_KEYS) > kScratchBytes) return MPM_ERR_STATE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MPM_ERR_CUDA;
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return MPM_ERR_CUDA;
      g_addr[dev] = p;
    }
    base = g_addr[dev];
  }
  uint32_t *keys_out = (uint32_t *)base;
  void *scratch = (char *)base + keys_bytes();
  cudaError_t e = mpm::sort_pairs(d_keys, nullptr, keys_out, d_perm, n, key_bits, scratch, (cudaStream_t)stream);
  return e == cudaSuccess ? MPM_OK : MPM_ERR_CUDA;
}
