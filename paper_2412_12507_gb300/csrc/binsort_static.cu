// binsort_static.cu — bin_and_sort for callers that cannot allocate device memory.
//
// Some callers of this library have no way to hand it scratch memory: a plugin running
// inside a host application that owns every device allocation through its own pool, or a
// hard-real-time frame loop that must never enter the driver's allocator (cudaMalloc can
// block, synchronise the device or fail mid-frame).  bin_and_sort_static serves them: it
// runs the same kernels as bin_and_sort, with the scratch taken from a fixed array that
// lives in this library's device image instead of from a caller buffer.  It allocates
// nothing.
//
// The array g_bin_scratch is a file-scope __device__ variable of UT_BIN_STATIC_SCRATCH_BYTES
// bytes: every GPU that loads the library keeps it until the process exits.  In host code
// its name is only a host-side stand-in for the device symbol, never a device address, so
// every call looks the real address up with cudaGetSymbolAddress, with the calling thread's
// device current, and checks the result.  The first call on a device also loads this
// module there; make that first call before capturing any stream.  Later lookups are cheap,
// and because nothing is cached, a device reset or a re-created primary context can never
// leave a stale address behind.  All calls share the one array and it keeps the last call's
// contents; nothing in it has to start at zero (the kernels clear what they accumulate
// into), but calls whose work overlaps on the GPU race on it, so issue them on one stream
// or otherwise order them.
#include "ut3d_device.cuh"
#include "ut3d_internal.h"

namespace ut3d {
namespace {

static __device__ __align__(256) unsigned char g_bin_scratch[UT_BIN_STATIC_SCRATCH_BYTES];

// Device address of g_bin_scratch in the current context.
ut_status scratch_address(void **out) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_bin_scratch) != cudaSuccess || !p) {
    (void)cudaGetLastError();  // the failed lookup must not be reported by a later call
    return UT_ERR_CUDA;
  }
  *out = p;
  return UT_OK;
}

}  // namespace
}  // namespace ut3d

using namespace ut3d;

extern "C" ut_status bin_and_sort_static(int32_t n, const float *depth, const int16_t *rect,
                                         const uint32_t *ntiles, const ut_camera *cam, const ut_options *opt,
                                         int64_t key_capacity, uint64_t *keys, uint32_t *vals,
                                         uint32_t *tile_ranges, int64_t *k_out, ut_stream stream) {
  // bin_and_sort's own argument checks come first, so that both entry points give the same
  // status for the same arguments; only then the size limit of the fixed array
  DevCam dc;
  DevOpts dop;
  size_t need = 0;
  ut_status st = bin_check_args(n, depth, rect, ntiles, cam, opt, key_capacity, vals, tile_ranges, k_out, dc, dop,
                                &need);
  if (st != UT_OK) return st;
  if (need > (size_t)UT_BIN_STATIC_SCRATCH_BYTES) return UT_ERR_CAPACITY;
  void *ws = nullptr;
  if ((st = scratch_address(&ws)) != UT_OK) return st;
  return bin_and_sort(n, depth, rect, ntiles, cam, opt, ws, (size_t)UT_BIN_STATIC_SCRATCH_BYTES, key_capacity, keys,
                      vals, tile_ranges, k_out, stream);
}
