// ut3d_debug.cuh — the checks of a debug build (compiled with -DUT_DEBUG; a testing aid with no
// counterpart in the paper).
//
// A release build compiles every check away.  A debug build tests, at the places where a wrong
// index would write outside a buffer, that the index is in range -- key and value positions
// below the key capacity, tile ids below the number of tiles, particle indices below the scene's
// count, rectangles inside the image -- and records the first violation it sees in a per
// translation unit device record {code, a, b, c} instead of trapping; the release build's
// existing guards still skip the access.  ut_debug_read() collects the records.  The binning
// workspace additionally carries guard bytes after every sub-buffer (see binsort.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ut3d.h"

namespace ut3d {

#ifdef UT_DEBUG
namespace {
__device__ unsigned int g_ut_dbg[4];  // internal linkage: one record per translation unit

__device__ __noinline__ void dbg_record(uint32_t code, uint32_t a, uint32_t b, uint32_t c) {
  if (atomicCAS(&g_ut_dbg[0], 0u, code) == 0u) {
    g_ut_dbg[1] = a;
    g_ut_dbg[2] = b;
    g_ut_dbg[3] = c;
  }
}
}  // namespace
#define UT_DBG_CHECK(cond, code, a, b, c)                                                    \
  do {                                                                                       \
    if (!(cond)) ::ut3d::dbg_record((code), (uint32_t)(a), (uint32_t)(b), (uint32_t)(c));   \
  } while (0)
// Defines this translation unit's reader (host): copies its record out, optionally clears it.
#define UT_DBG_READER(name)                                                                   \
  ut_status name(uint32_t out[4], bool reset) {                                               \
    if (cudaMemcpyFromSymbol(out, g_ut_dbg, sizeof(unsigned int) * 4) != cudaSuccess)         \
      return UT_ERR_CUDA;                                                                     \
    const unsigned int zero[4] = {0u, 0u, 0u, 0u};                                            \
    if (reset && cudaMemcpyToSymbol(g_ut_dbg, zero, sizeof(zero)) != cudaSuccess) return UT_ERR_CUDA; \
    return UT_OK;                                                                             \
  }
#else
#define UT_DBG_CHECK(cond, code, a, b, c) \
  do {                                    \
  } while (0)
#define UT_DBG_READER(name)                      \
  ut_status name(uint32_t out[4], bool) {        \
    out[0] = out[1] = out[2] = out[3] = 0u;      \
    return UT_OK;                                \
  }
#endif

}  // namespace ut3d
