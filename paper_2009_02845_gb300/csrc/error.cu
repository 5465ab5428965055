// Relative Frobenius error ||M - U V^T||_F / ||M||_F (Section 5.1).
//
// Dense M: tiled residual, 64 x 64 tile per step of a fixed-size persistent
// grid; each thread forms 4 x 4 inner products U_i . V_j in binary32
// (nonnegative terms, no cancellation), the residual and its square in FP64;
// warp-shuffle then shared-memory reduction to one FP64 partial per CTA,
// partials summed in CTA order (deterministic).
// Sparse M: the expansion ||M||^2 - 2 sum_{nnz} M_ij U_i.V_j + <U^T U, V^T V>,
// each term with FP64 accumulation.
#include "common.cuh"
#include "kernels.cuh"

namespace dsanls {

constexpr int RES_TILE = 64;
constexpr int RES_THREADS = 256;
constexpr int RES_KC = 32;  // k-chunk staged in shared memory

DSANLS_DEV double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// reduces v over the CTA; result valid in thread 0
DSANLS_DEV double cta_sum_d(double v, double *red) {
    v = warp_sum_d(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];
    __syncthreads();
    return tot;
}

__global__ void __launch_bounds__(RES_THREADS)
    k_dense_residual(const float *__restrict__ M, int64_t ld, const float *__restrict__ U,
                     const float *__restrict__ V, int64_t m, int64_t n, int k, double *__restrict__ part) {
    __shared__ __align__(16) float us[RES_KC][RES_TILE + 4];
    __shared__ __align__(16) float vs[RES_KC][RES_TILE + 4];
    __shared__ double red[RES_THREADS / 32];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t tiles_n = ceil_div(n, RES_TILE);
    const int64_t tiles = ceil_div(m, RES_TILE) * tiles_n;
    double local = 0.0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t i0 = (tile / tiles_n) * RES_TILE, j0 = (tile % tiles_n) * RES_TILE;
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
        for (int c0 = 0; c0 < k; c0 += RES_KC) {
            __syncthreads();
            for (int e = threadIdx.x; e < RES_TILE * RES_KC; e += RES_THREADS) {
                const int r = e / RES_KC, c = e % RES_KC;
                const bool okc = c0 + c < k;
                us[c][r] = (okc && i0 + r < m) ? U[(i0 + r) * k + c0 + c] : 0.0f;
                vs[c][r] = (okc && j0 + r < n) ? V[(j0 + r) * k + c0 + c] : 0.0f;
            }
            __syncthreads();
#pragma unroll 8
            for (int c = 0; c < RES_KC; ++c) {
                const float4 ua = *reinterpret_cast<const float4 *>(&us[c][ty * 4]);
                const float4 vb = *reinterpret_cast<const float4 *>(&vs[c][tx * 4]);
                const float uu[4] = {ua.x, ua.y, ua.z, ua.w};
                const float vv[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = __fmaf_rn(uu[a], vv[b], acc[a][b]);
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t i = i0 + ty * 4 + a;
            if (i >= m) continue;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int64_t j = j0 + tx * 4 + b;
                if (j < n) {
                    const double r = (double)M[i * ld + j] - (double)acc[a][b];
                    local = fma(r, r, local);
                }
            }
        }
    }
    const double tot = cta_sum_d(local, red);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_sum_parts(const double *__restrict__ part, int np, double *__restrict__ out) {
    __shared__ double red[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) v += part[i];
    const double tot = cta_sum_d(v, red);
    if (threadIdx.x == 0) *out = tot;
}

static int residual_grid(int64_t tiles, int64_t work_elems) {
    int64_t g = 152 * 8;
    if (g > tiles) g = tiles;
    if (g > work_elems) g = work_elems;
    return (int)(g < 1 ? 1 : g);
}

void launch_dense_residual(const float *M, int64_t ld, const float *U, const float *V, int64_t m, int64_t n,
                           int k, double *work, int64_t work_elems, double *out, cudaStream_t s) {
    const int64_t tiles = ceil_div(m, RES_TILE) * ceil_div(n, RES_TILE);
    const int g = residual_grid(tiles, work_elems);
    k_dense_residual<<<g, RES_THREADS, 0, s>>>(M, ld, U, V, m, n, k, work);
    DSANLS_LAUNCH_CHECK();
    k_sum_parts<<<1, 1024, 0, s>>>(work, g, out);
    DSANLS_LAUNCH_CHECK();
}

__global__ void k_sumsq(const float *__restrict__ x, int64_t len, double *__restrict__ part) {
    __shared__ double red[32];
    double v = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = (double)x[i];
        v = fma(a, a, v);
    }
    const double tot = cta_sum_d(v, red);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

void launch_sumsq(const float *x, int64_t len, double *work, int64_t work_elems, double *out, cudaStream_t s) {
    int64_t g = 152 * 8;
    if (g > work_elems) g = work_elems;
    k_sumsq<<<(unsigned)g, 256, 0, s>>>(x, len, work);
    DSANLS_LAUNCH_CHECK();
    k_sum_parts<<<1, 1024, 0, s>>>(work, (int)g, out);
    DSANLS_LAUNCH_CHECK();
}

// One warp per row of M; each lane takes one nonzero at a time and forms the
// binary32 inner product U_i . V_j; val * dot accumulated in FP64.
__global__ void k_sparse_cross(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                               const float *__restrict__ val, int64_t m, const float *__restrict__ U,
                               const float *__restrict__ V, int k, double *__restrict__ part) {
    __shared__ double red[32];
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double local = 0.0;
    for (int64_t i = warp; i < m; i += nwarps) {
        const float *u = U + i * k;
        for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
            const float *v = V + (int64_t)col[e] * k;
            float dot = 0.0f;
            for (int c = 0; c < k; ++c) dot = __fmaf_rn(u[c], v[c], dot);
            local = fma((double)val[e], (double)dot, local);
        }
    }
    const double tot = cta_sum_d(local, red);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

void launch_sparse_cross(const int64_t *rowptr, const int32_t *col, const float *val, int64_t m, const float *U,
                         const float *V, int k, double *work, int64_t work_elems, double *out, cudaStream_t s) {
    int64_t g = 152 * 8;
    if (g > work_elems) g = work_elems;
    k_sparse_cross<<<(unsigned)g, 256, 0, s>>>(rowptr, col, val, m, U, V, k, work);
    DSANLS_LAUNCH_CHECK();
    k_sum_parts<<<1, 1024, 0, s>>>(work, (int)g, out);
    DSANLS_LAUNCH_CHECK();
}

// X^T X: each CTA takes chunks of 64 rows; each thread owns (a, b) pairs of
// the upper triangle, sums the chunk in binary32 and adds it to an FP64
// accumulator; per-CTA partials are summed in CTA order.
constexpr int FG_ROWS = 64;

__global__ void k_factor_gram(const float *__restrict__ X, int64_t rows, int k, double *__restrict__ part) {
    extern __shared__ float xs[];  // FG_ROWS x (k+1)
    const int ldx = k + 1;
    const int npairs = k * (k + 1) / 2;
    constexpr int MAXP = 24;  // pairs per thread (k <= 128, 256 threads: 8256/256 < 33) -> loop below
    double acc[MAXP];
    int pa[MAXP], pb[MAXP];
#pragma unroll
    for (int q = 0; q < MAXP; ++q) {
        acc[q] = 0.0;
        const int p = threadIdx.x + q * blockDim.x;
        int a = 0, rem = p;
        if (p < npairs)
            while (rem >= k - a) {
                rem -= k - a;
                ++a;
            }
        pa[q] = a;
        pb[q] = a + rem;
    }
    const int64_t chunks = ceil_div(rows, FG_ROWS);
    for (int64_t ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
        const int64_t r0 = ch * FG_ROWS;
        const int nr = (int)min((int64_t)FG_ROWS, rows - r0);
        __syncthreads();
        for (int e = threadIdx.x; e < FG_ROWS * k; e += blockDim.x) {
            const int r = e / k, c = e % k;
            xs[r * ldx + c] = (r < nr) ? X[(r0 + r) * k + c] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < MAXP; ++q) {
            const int p = threadIdx.x + q * blockDim.x;
            if (p < npairs) {
                float sacc = 0.0f;
                for (int r = 0; r < FG_ROWS; ++r) sacc = __fmaf_rn(xs[r * ldx + pa[q]], xs[r * ldx + pb[q]], sacc);
                acc[q] += (double)sacc;
            }
        }
    }
    double *out = part + (int64_t)blockIdx.x * k * k;
#pragma unroll
    for (int q = 0; q < MAXP; ++q) {
        const int p = threadIdx.x + q * blockDim.x;
        if (p < npairs) out[pa[q] * k + pb[q]] = acc[q];
    }
}

__global__ void k_factor_gram_reduce(const double *__restrict__ part, int np, int k, double *__restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= k * k) return;
    const int a = idx / k, b = idx % k;
    const int lo = min(a, b), hi = max(a, b);
    double v = 0.0;
    for (int c = 0; c < np; ++c) v += part[(int64_t)c * k * k + lo * k + hi];
    out[idx] = v;
}

void launch_factor_gram(const float *X, int64_t rows, int k, double *work, int64_t work_elems, double *out,
                        cudaStream_t s) {
    int64_t g = 152 * 2;
    const int64_t chunks = ceil_div(rows, FG_ROWS);
    if (g > chunks) g = chunks;
    while (g > 1 && g * k * k > work_elems) g /= 2;
    if (g < 1) g = 1;
    const size_t smem = (size_t)FG_ROWS * (k + 1) * sizeof(float);
    k_factor_gram<<<(unsigned)g, 352, smem, s>>>(X, rows, k, work);
    DSANLS_LAUNCH_CHECK();
    k_factor_gram_reduce<<<(unsigned)ceil_div((int64_t)k * k, 256), 256, 0, s>>>(work, (int)g, k, out);
    DSANLS_LAUNCH_CHECK();
}

__global__ void k_sparse_combine(const double *mm, const double *cross, const double *GU, const double *GV, int k,
                                 double *out) {
    __shared__ double red[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < k * k; i += blockDim.x) v += GU[i] * GV[i];
    const double g = cta_sum_d(v, red);
    if (threadIdx.x == 0) *out = *mm - 2.0 * (*cross) + g;
}

void launch_sparse_combine(const double *mm, const double *cross, const double *GU, const double *GV, int k,
                           double *out, cudaStream_t s) {
    k_sparse_combine<<<1, 256, 0, s>>>(mm, cross, GU, GV, k, out);
    DSANLS_LAUNCH_CHECK();
}

}  // namespace dsanls
