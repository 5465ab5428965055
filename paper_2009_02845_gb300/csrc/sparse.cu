// Sparse M (CSR) for the sketched products (Section 3.4: a subsampling
// sketch keeps M sparse; forming A = M S costs O(|I_r| d)).
//
//  * warp-per-row SpMM  out[i][:] = alpha * sum_{e in row i} val_e D[col_e][:]
//    (lanes across the output columns, 16-byte loads when aligned; one FMA
//    chain per output in CSR order, deterministic).
//  * subsampled product: for a subsampling sketch the U-half needs, per row
//    i of M, only the entries whose column is in J (R_i = (n/d) sum over
//    those entries of M_ij V_j).  A bitmap of J marks the sampled columns; a
//    warp streams row i of the CSR, keeps the marked entries and accumulates
//    them in CSR order.  The V-half does the same on the transposed CSR with
//    a bitmap of the sampled rows J'.
#include "common.cuh"
#include "kernels.cuh"

namespace dsanls {

template <bool VEC4>
__global__ void k_spmm_rows(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                            const float *__restrict__ val, int64_t rows, const float *__restrict__ D, int64_t ldd,
                            int w, float alpha, float *__restrict__ out, int64_t ldo) {
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
                    for (int64_t e = e0; e < e1; ++e) acc = __fmaf_rn(val[e], D[(int64_t)col[e] * ldd + c], acc);
                    out[i * ldo + c] = __fmul_rn(alpha, acc);
                }
            }
        }
    }
}

void launch_spmm_rows(const int64_t *rowptr, const int32_t *col, const float *val, int64_t rows, const float *D,
                      int64_t ldd, int w, float alpha, float *out, int64_t ldo, cudaStream_t s) {
    if (rows <= 0 || w <= 0) return;
    const bool vec = (w % 4 == 0) && (ldd % 4 == 0) && (ldo % 4 == 0) && (((uintptr_t)D & 15) == 0) &&
                     (((uintptr_t)out & 15) == 0);
    int64_t blocks = ceil_div(rows, 8);
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (vec)
        k_spmm_rows<true><<<(unsigned)blocks, 256, 0, s>>>(rowptr, col, val, rows, D, ldd, w, alpha, out, ldo);
    else
        k_spmm_rows<false><<<(unsigned)blocks, 256, 0, s>>>(rowptr, col, val, rows, D, ldd, w, alpha, out, ldo);
    DSANLS_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// subsampled product of a CSR matrix against the membership bitmap of the
// sampled set (left by launch_subsample)
// ---------------------------------------------------------------------------

// One warp per row: lanes read 128 entries at a time (lane L takes entries
// base + 4L .. base + 4L + 3, four independent loads, then four independent
// bitmap tests), keep those whose column is in the sampled set, and the whole
// warp accumulates val * Y[col][:] for each kept entry in CSR order (lanes
// across the k output columns).  Deterministic: one FMA chain per output in
// CSR order.
// Sum over the sampled entries of CSR range [e0, e1) into acc (lanes across k).
DSANLS_DEV void sampled_range(const int32_t *__restrict__ col, const float *__restrict__ val, int64_t e0, int64_t e1,
                              const uint32_t *__restrict__ bits, const float *__restrict__ Y, int k, int lane,
                              float acc[4]) {
    for (int64_t base = e0; base < e1; base += 128) {
        int32_t c[4];
        unsigned nib = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t e = base + 4 * lane + j;
            c[j] = e < e1 ? col[e] : -1;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (c[j] >= 0 && ((__ldg(&bits[c[j] >> 5]) >> (c[j] & 31)) & 1u)) nib |= 1u << j;
        unsigned lanes = __ballot_sync(0xffffffffu, nib != 0);
        while (lanes) {
            const int src = __ffs(lanes) - 1;
            lanes &= lanes - 1;
            const unsigned sn = __shfl_sync(0xffffffffu, nib, src);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!((sn >> j) & 1u)) continue;
                const int32_t cj = __shfl_sync(0xffffffffu, c[j], src);
                const int64_t ej = base + 4 * src + j;
                const float vj = val[ej];
                const float *y = Y + (int64_t)cj * k;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int cc = lane + 32 * q;
                    if (cc < k) acc[q] = __fmaf_rn(vj, y[cc], acc[q]);
                }
            }
        }
    }
}

// Rows longer than LONG_ROW entries are skipped here and handled in chunks.
// The next row's bounds are loaded before the current row is processed.
__global__ void __launch_bounds__(256)
    k_sampled_spmm(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, const float *__restrict__ val,
                   int64_t rows, const uint32_t *__restrict__ bits, const float *__restrict__ Y, int k, float alpha,
                   float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t i = warp;
    int64_t e0 = 0, e1 = 0;
    if (i < rows) {
        e0 = rowptr[i];
        e1 = rowptr[i + 1];
    }
    while (i < rows) {
        const int64_t inext = i + nwarps;
        int64_t n0 = 0, n1 = 0;
        if (inext < rows) {
            n0 = rowptr[inext];
            n1 = rowptr[inext + 1];
        }
        if (e1 - e0 <= LONG_ROW) {
            float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            sampled_range(col, val, e0, e1, bits, Y, k, lane, acc);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int cc = lane + 32 * q;
                if (cc < k) out[i * k + cc] = __fmul_rn(alpha, acc[q]);
            }
        }
        i = inext;
        e0 = n0;
        e1 = n1;
    }
}

// One warp per chunk of a long row: partial[chunk][0..k)
__global__ void __launch_bounds__(256)
    k_sampled_chunks(const int64_t *__restrict__ cbeg, const int64_t *__restrict__ cend, int64_t nchunks,
                     const int32_t *__restrict__ col, const float *__restrict__ val, const uint32_t *__restrict__ bits,
                     const float *__restrict__ Y, int k, float *__restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = warp; c < nchunks; c += nwarps) {
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        sampled_range(col, val, cbeg[c], cend[c], bits, Y, k, lane, acc);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int cc = lane + 32 * q;
            if (cc < k) partial[c * k + cc] = acc[q];
        }
    }
}

// out[row] = alpha * sum of the row's chunk partials in chunk order
__global__ void k_combine_long(const int64_t *__restrict__ lrows, const int64_t *__restrict__ first, int64_t nlong,
                               const float *__restrict__ partial, int k, float alpha, float *__restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nlong * k) return;
    const int64_t l = idx / k;
    const int c = (int)(idx % k);
    float acc = 0.0f;
    for (int64_t ch = first[l]; ch < first[l + 1]; ++ch) acc += partial[ch * k + c];
    out[lrows[l] * k + c] = __fmul_rn(alpha, acc);
}

void launch_sampled_spmm(const int64_t *rowptr, const int32_t *col, const float *val, int64_t rows,
                         const uint32_t *bits, const float *Y, int k, float alpha, float *out, const LongRows &lr,
                         cudaStream_t s) {
    if (rows <= 0) return;
    int64_t blocks = ceil_div(rows, 8);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_sampled_spmm<<<(unsigned)blocks, 256, 0, s>>>(rowptr, col, val, rows, bits, Y, k, alpha, out);
    DSANLS_LAUNCH_CHECK();
    if (lr.nlong > 0) {
        int64_t cb = ceil_div(lr.nchunks, 8);
        if (cb > 152 * 16) cb = 152 * 16;
        k_sampled_chunks<<<(unsigned)cb, 256, 0, s>>>(lr.cbeg, lr.cend, lr.nchunks, col, val, bits, Y, k, lr.partial);
        DSANLS_LAUNCH_CHECK();
        k_combine_long<<<(unsigned)ceil_div(lr.nlong * k, 256), 256, 0, s>>>(lr.rows, lr.first, lr.nlong, lr.partial,
                                                                            k, alpha, out);
        DSANLS_LAUNCH_CHECK();
    }
}

}  // namespace dsanls
