// Device buffers of a sub-CSR built from sampled rows of a source CSR.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dsanls {

struct SubCsr {
    int64_t *off = nullptr;    // d + 1 segment offsets into the concatenated sampled rows
    int64_t *total = nullptr;  // 1: number of sampled entries
    int32_t *cnt = nullptr;    // out_rows: counts, then fill cursors
    int64_t *ptr = nullptr;    // out_rows + 1: row pointer of the sub-CSR
    int64_t *bsum = nullptr;   // ceil(out_rows / 4096) + 1: scan block sums
    int32_t *col = nullptr;    // capacity: original column index (row of the fixed factor)
    float *val = nullptr;      // capacity
    int64_t capacity = 0;      // largest possible number of sampled entries
};

void launch_exclusive_scan(const int32_t *cnt, int64_t n, int64_t *out, int64_t *bsum, cudaStream_t s);
// Builds `sub` (out_rows rows) from rows J[0..d) of the source CSR (sptr, sidx, sval),
// whose entries index rows of the output.
void launch_subcsr(const int64_t *sptr, const int32_t *sidx, const float *sval, const int32_t *J, int d,
                   int64_t out_rows, SubCsr &sub, cudaStream_t s);

}  // namespace dsanls
