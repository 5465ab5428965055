// Index checks of the debug build (compiled with -DDSANLS_BOUNDS; build(bounds=True)
// links it as libdsanls_bounds.so).  DSANLS_IN(i, n, site) is true when
// 0 <= i < n; a failing check counts itself -- the first one also records its
// site code and index -- and the caller skips the access, so an index computed
// from the data (a column of a CSR, a row key, a scatter destination) that
// leaves its array is reported instead of read or written.  In the normal
// build the macro is the constant true and nothing below exists.  Every
// translation unit that includes this header has its own counters, read by
// its bounds_report_* function.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dsanls {
#ifdef DSANLS_BOUNDS
namespace {
__device__ unsigned long long g_bnd_count;
__device__ long long g_bnd_first[2];

__device__ __forceinline__ bool bounds_ok(long long i, long long n, int site) {
    if (i >= 0 && i < n) return true;
    if (atomicAdd(&g_bnd_count, 1ull) == 0ull) {
        g_bnd_first[0] = site;
        g_bnd_first[1] = i;
    }
    return false;
}

// (failed checks, site of the first, its index) of this translation unit; reset after reading
inline void bounds_read_tu(int reset, int64_t out[3]) {
    unsigned long long c = 0;
    long long f[2] = {0, 0};
    cudaMemcpyFromSymbol(&c, g_bnd_count, sizeof(c));
    cudaMemcpyFromSymbol(f, g_bnd_first, sizeof(f));
    out[0] = (int64_t)c;
    out[1] = f[0];
    out[2] = f[1];
    if (reset) {
        const unsigned long long z = 0;
        const long long zf[2] = {0, 0};
        cudaMemcpyToSymbol(g_bnd_count, &z, sizeof(z));
        cudaMemcpyToSymbol(g_bnd_first, zf, sizeof(zf));
    }
}
}  // namespace
#define DSANLS_IN(i, n, site) ::dsanls::bounds_ok((long long)(i), (long long)(n), (site))
#else
#define DSANLS_IN(i, n, site) true
#endif
}  // namespace dsanls
