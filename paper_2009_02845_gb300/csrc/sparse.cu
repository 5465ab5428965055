// Sparse M (CSR) for the sketched products with a dense sketch:
//  * warp-per-row SpMM  out[i][:] = alpha * sum_{e in row i} val_e D[col_e][:]
//    (lanes across the output columns, 16-byte loads when aligned; one FMA
//    chain per output in CSR order, deterministic).
// The subsampling sketch gathers X[:, J] into a sub-CSR instead (subcsr.cu).
#include "bounds.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace dsanls {

template <bool VEC4>
__global__ void k_spmm_rows(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                            const float *__restrict__ val, int64_t rows, const float *__restrict__ D, int64_t drows,
                            int64_t ldd, int w, float alpha, float *__restrict__ out, int64_t ldo) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < rows; i += nwarps) {
        const int64_t e0 = rowptr[i], e1 = rowptr[i + 1];
        if (VEC4) {
            for (int c0 = 0; c0 < w; c0 += 128) {
                const int c = c0 + lane * 4;
                if (c < w) {
                    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int64_t e = e0; e < e1; ++e) {
                        const float v = val[e];
                        if (!DSANLS_IN(col[e], drows, 201)) continue;
                        const float4 dv = *reinterpret_cast<const float4 *>(D + (int64_t)col[e] * ldd + c);
                        acc.x = __fmaf_rn(v, dv.x, acc.x);
                        acc.y = __fmaf_rn(v, dv.y, acc.y);
                        acc.z = __fmaf_rn(v, dv.z, acc.z);
                        acc.w = __fmaf_rn(v, dv.w, acc.w);
                    }
                    float4 r = make_float4(__fmul_rn(alpha, acc.x), __fmul_rn(alpha, acc.y), __fmul_rn(alpha, acc.z),
                                           __fmul_rn(alpha, acc.w));
                    *reinterpret_cast<float4 *>(out + i * ldo + c) = r;
                }
            }
        } else {
            for (int c0 = 0; c0 < w; c0 += 32) {
                const int c = c0 + lane;
                if (c < w) {
                    float acc = 0.0f;
                    for (int64_t e = e0; e < e1; ++e)
                        if (DSANLS_IN(col[e], drows, 202)) acc = __fmaf_rn(val[e], D[(int64_t)col[e] * ldd + c], acc);
                    out[i * ldo + c] = __fmul_rn(alpha, acc);
                }
            }
        }
    }
}

void launch_spmm_rows(const int64_t *rowptr, const int32_t *col, const float *val, int64_t rows, const float *D,
                      int64_t drows, int64_t ldd, int w, float alpha, float *out, int64_t ldo, cudaStream_t s) {
    if (rows <= 0 || w <= 0) return;
    const bool vec = (w % 4 == 0) && (ldd % 4 == 0) && (ldo % 4 == 0) && (((uintptr_t)D & 15) == 0) &&
                     (((uintptr_t)out & 15) == 0);
    int64_t blocks = ceil_div(rows, 8);
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (vec)
        k_spmm_rows<true><<<(unsigned)blocks, 256, 0, s>>>(rowptr, col, val, rows, D, drows, ldd, w, alpha, out, ldo);
    else
        k_spmm_rows<false><<<(unsigned)blocks, 256, 0, s>>>(rowptr, col, val, rows, D, drows, ldd, w, alpha, out,
                                                            ldo);
    DSANLS_LAUNCH_CHECK();
}

void bounds_report_sparse(int reset, int64_t out[3]) {
#ifdef DSANLS_BOUNDS
    bounds_read_tu(reset, out);
#else
    (void)reset;
    out[0] = out[1] = out[2] = 0;
#endif
}

}  // namespace dsanls
