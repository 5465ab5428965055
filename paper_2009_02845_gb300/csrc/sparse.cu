// Sparse M (CSR) for the sketched products (Section 3.4: a subsampling
// sketch keeps M sparse; forming A = M S costs O(|I_r| d)).
//
//  * warp-per-row SpMM  out[i][:] = alpha * sum_{e in row i} val_e D[col_e][:]
//    (lanes across the output columns, 16-byte loads when aligned; one FMA
//    chain per output in CSR order, deterministic).
//  * sub-CSR of the sampled columns: for a subsampling sketch the U-half
//    needs, per row i of M, only the entries whose column is in J.  They are
//    read from the transposed CSR (rows J of M^T), counted per row of M,
//    placed by an exclusive scan, filled, and each row sorted by column so
//    the layout (and every later sum) is independent of thread timing.
//    The V-half does the same with the roles of the two CSRs swapped.
#include "common.cuh"
#include "kernels.cuh"
#include "sparse.cuh"

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
// exclusive scan of int32 counts into int64 offsets (n + 1 entries)
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024;
constexpr int SCAN_PER = 4;
constexpr int SCAN_CHUNK = SCAN_T * SCAN_PER;

DSANLS_DEV int64_t block_exclusive_scan(int64_t v, int64_t *tmp, int64_t &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = (lane < (int)(blockDim.x >> 5)) ? tmp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        tmp[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    const int64_t warp_off = (w > 0) ? tmp[w - 1] : 0;
    total = tmp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_off + x - v;
}

__global__ void k_scan_local(const int32_t *__restrict__ cnt, int64_t n, int64_t *__restrict__ out,
                             int64_t *__restrict__ bsum) {
    __shared__ int64_t tmp[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_PER;
    int64_t v[SCAN_PER];
    int64_t s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_PER; ++q) {
        v[q] = (base + q < n) ? cnt[base + q] : 0;
        s += v[q];
    }
    int64_t total;
    int64_t off = block_exclusive_scan(s, tmp, total);
#pragma unroll
    for (int q = 0; q < SCAN_PER; ++q) {
        if (base + q < n) out[base + q] = off;
        off += v[q];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void k_scan_bsum(int64_t *__restrict__ bsum, int64_t nb) {
    __shared__ int64_t tmp[32];
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_T) {
        const int64_t b = b0 + threadIdx.x;
        const int64_t v = (b < nb) ? bsum[b] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, tmp, total);
        if (b < nb) bsum[b] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_scan_apply(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ bsum, int64_t nb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[i / SCAN_CHUNK];
    if (i == 0) out[n] = bsum[nb];
}

// bsum needs ceil(n / 4096) + 1 entries
void launch_exclusive_scan(const int32_t *cnt, int64_t n, int64_t *out, int64_t *bsum, cudaStream_t s) {
    const int64_t nb = ceil_div(n, SCAN_CHUNK);
    if (nb > 0) {
        k_scan_local<<<(unsigned)nb, SCAN_T, 0, s>>>(cnt, n, out, bsum);
        DSANLS_LAUNCH_CHECK();
    }
    k_scan_bsum<<<1, SCAN_T, 0, s>>>(bsum, nb);
    DSANLS_LAUNCH_CHECK();
    k_scan_apply<<<(unsigned)ceil_div(n + 1, 256), 256, 0, s>>>(out, n, bsum, nb);
    DSANLS_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// sub-CSR of sampled source rows
// ---------------------------------------------------------------------------
// off[p] = sum_{q<p} len(J_q) for p <= d; *total = off[d].  One CTA.
__global__ void k_sub_offsets(const int64_t *__restrict__ sptr, const int32_t *__restrict__ J, int d,
                              int64_t *__restrict__ off, int64_t *__restrict__ total) {
    __shared__ int64_t tmp[32];
    const int per = (d + SCAN_T - 1) / SCAN_T;
    const int p0 = threadIdx.x * per;
    int64_t s = 0;
    for (int q = 0; q < per; ++q) {
        const int p = p0 + q;
        if (p < d) s += sptr[J[p] + 1] - sptr[J[p]];
    }
    int64_t tot;
    int64_t o = block_exclusive_scan(s, tmp, tot);
    for (int q = 0; q < per; ++q) {
        const int p = p0 + q;
        if (p < d) {
            off[p] = o;
            o += sptr[J[p] + 1] - sptr[J[p]];
        }
    }
    if (threadIdx.x == 0) {
        off[d] = tot;
        *total = tot;
    }
}

DSANLS_DEV int find_segment(const int64_t *off, int d, int64_t e) {
    int lo = 0, hi = d;  // off[lo] <= e < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= e)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

template <bool FILL>
__global__ void k_sub_scatter(const int64_t *__restrict__ sptr, const int32_t *__restrict__ sidx,
                              const float *__restrict__ sval, const int32_t *__restrict__ J, int d,
                              const int64_t *__restrict__ off, const int64_t *__restrict__ total_dev,
                              int32_t *__restrict__ cnt, const int64_t *__restrict__ ptr, int32_t *__restrict__ ocol,
                              float *__restrict__ oval) {
    const int64_t total = *total_dev;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_segment(off, d, e);
        const int64_t q = sptr[J[p]] + (e - off[p]);
        const int32_t i = sidx[q];
        const int32_t pos = atomicAdd(&cnt[i], 1);
        if (FILL) {
            ocol[ptr[i] + pos] = J[p];
            oval[ptr[i] + pos] = sval[q];
        }
    }
}

__global__ void k_sub_sort(const int64_t *__restrict__ ptr, int64_t rows, int32_t *__restrict__ col,
                           float *__restrict__ val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const int64_t b = ptr[i], e = ptr[i + 1];
    for (int64_t x = b + 1; x < e; ++x) {
        const int32_t c = col[x];
        const float v = val[x];
        int64_t y = x - 1;
        while (y >= b && col[y] > c) {
            col[y + 1] = col[y];
            val[y + 1] = val[y];
            --y;
        }
        col[y + 1] = c;
        val[y + 1] = v;
    }
}

void launch_subcsr(const int64_t *sptr, const int32_t *sidx, const float *sval, const int32_t *J, int d,
                   int64_t out_rows, SubCsr &sub, cudaStream_t s) {
    k_sub_offsets<<<1, SCAN_T, 0, s>>>(sptr, J, d, sub.off, sub.total);
    DSANLS_LAUNCH_CHECK();
    DSANLS_CUDA(cudaMemsetAsync(sub.cnt, 0, (size_t)out_rows * sizeof(int32_t), s));
    const unsigned grid = 152 * 8;
    k_sub_scatter<false><<<grid, 256, 0, s>>>(sptr, sidx, sval, J, d, sub.off, sub.total, sub.cnt, nullptr, nullptr,
                                              nullptr);
    DSANLS_LAUNCH_CHECK();
    launch_exclusive_scan(sub.cnt, out_rows, sub.ptr, sub.bsum, s);
    DSANLS_CUDA(cudaMemsetAsync(sub.cnt, 0, (size_t)out_rows * sizeof(int32_t), s));
    k_sub_scatter<true><<<grid, 256, 0, s>>>(sptr, sidx, sval, J, d, sub.off, sub.total, sub.cnt, sub.ptr, sub.col,
                                             sub.val);
    DSANLS_LAUNCH_CHECK();
    k_sub_sort<<<(unsigned)ceil_div(out_rows, 256), 256, 0, s>>>(sub.ptr, out_rows, sub.col, sub.val);
    DSANLS_LAUNCH_CHECK();
}

}  // namespace dsanls
