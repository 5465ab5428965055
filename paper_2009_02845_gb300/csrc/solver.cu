// Gram matrix, step size and the NNLS subproblem update (Section 3.5).
//
//  * G = B B^T (k x k) accumulated in FP64 from the binary32 sketch product
//    B (k x d): chunks of d per CTA, products exact in FP64, chunk partials
//    summed in a fixed order (deterministic).
//  * step size of the projected gradient step: eta_t = 1/(lambda_max(G) +
//    mu_t), mu_t = alpha + beta t; lambda_max by power iteration from the
//    all-ones vector (binary32 iterations, FP64 Rayleigh quotient).
//  * fused row update, one thread per row with the row held in registers and
//    G in shared memory:
//      PGD (eq. gradient_descent):  z <- max(0, z - eta (z G - r))
//      RCD (Alg. 3, eq. entry_sol): for j: z_j <- max(0, (mu z_j + r_j -
//           sum_{l != j} G_lj z_l) / (G_jj + mu)), in place, so columns l < j
//           already hold their new values.
//    Optional clamp at sqrt(2 ||M||_F) (eq. extra_con); a NaN/Inf before the
//    projection raises a device flag that the host turns into an error.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace dsanls {

// ---------------------------------------------------------------------------
// Gram in FP64
// ---------------------------------------------------------------------------
constexpr int GRAM_THREADS = 256;
constexpr int GRAM_MAXP = 33;  // pairs per thread: k(k+1)/2 <= 8256 < 33 * 256

// Each CTA sums chunks blockIdx.x, blockIdx.x + gridDim.x, ... of the d axis
// for every pair (a <= b); each thread owns up to GRAM_MAXP pairs with FP64
// accumulators in registers.  The chunk is staged in shared memory already
// converted to FP64 (one conversion per entry, not one per product: the FP64
// pipe is the scarce unit).
__global__ void __launch_bounds__(GRAM_THREADS)
    k_gram_partial(const float *__restrict__ W, int k, int64_t d, int64_t dc, double *__restrict__ part) {
    extern __shared__ double ws[];  // k x (dc + 1), padded against bank conflicts
    const int64_t ldw = dc + 1;
    const int npairs = k * (k + 1) / 2;
    double acc[GRAM_MAXP];
    int pa[GRAM_MAXP], pb[GRAM_MAXP];
#pragma unroll
    for (int q = 0; q < GRAM_MAXP; ++q) {
        acc[q] = 0.0;
        const int p = threadIdx.x + q * GRAM_THREADS;
        int a = 0, rem = p;
        if (p < npairs)
            while (rem >= k - a) {
                rem -= k - a;
                ++a;
            }
        pa[q] = a;
        pb[q] = a + rem;
    }
    const int64_t chunks = ceil_div(d, dc);
    for (int64_t ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
        const int64_t j0 = ch * dc;
        const int64_t len = min(dc, d - j0);
        __syncthreads();
        for (int64_t e = threadIdx.x; e < (int64_t)k * dc; e += GRAM_THREADS) {
            const int a = (int)(e / dc);
            const int64_t j = e - (int64_t)a * dc;
            ws[a * ldw + j] = (j < len) ? (double)W[(int64_t)a * d + j0 + j] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < GRAM_MAXP; ++q) {
            if (threadIdx.x + q * GRAM_THREADS < npairs) {
                const double *wa = ws + (int64_t)pa[q] * ldw;
                const double *wb = ws + (int64_t)pb[q] * ldw;
                double s = acc[q];
                for (int64_t j = 0; j < len; ++j) s = fma(wa[j], wb[j], s);
                acc[q] = s;
            }
        }
    }
    double *out = part + (int64_t)blockIdx.x * k * k;
#pragma unroll
    for (int q = 0; q < GRAM_MAXP; ++q)
        if (threadIdx.x + q * GRAM_THREADS < npairs) out[pa[q] * k + pb[q]] = acc[q];
}

// 32 consecutive pairs (a <= b, row-major order of the upper triangle) per
// CTA of 256 threads: warp w sums the partials c = w, w + 8, ... of every pair
// (lane = pair; consecutive lanes read consecutive entries of a partial), then
// thread p adds the eight warp sums in warp order.  A fixed order: the result
// does not depend on scheduling.
__global__ void __launch_bounds__(256)
    k_gram_reduce(const double *__restrict__ part, int nparts, int k, double *__restrict__ G) {
    __shared__ double ws[8][33];
    const int npairs = k * (k + 1) / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = blockIdx.x * 32 + lane;
    int a = 0, b = 0;
    if (p < npairs) {
        int rem = p;
        while (rem >= k - a) {
            rem -= k - a;
            ++a;
        }
        b = a + rem;
    }
    double acc = 0.0;
    if (p < npairs)
        for (int c = warp; c < nparts; c += 8) acc += part[(int64_t)c * k * k + a * k + b];
    ws[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && p < npairs) {
        double tot = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) tot += ws[w][lane];
        G[a * k + b] = tot;
        G[b * k + a] = tot;
    }
}

void launch_gram(const float *W, int k, int64_t d, double *G64, double *work, int64_t work_elems,
                 cudaStream_t s) {
    // chunk width: about two chunks per SM, at most ~200 KB of shared memory
    int64_t dc = ceil_div(ceil_div(d, 2 * 152), 4) * 4;
    const int64_t dc_max = (200 * 1024) / (8 * (int64_t)k) - 1;
    if (dc > dc_max) dc = dc_max;
    if (dc < 1) dc = 1;
    int64_t grid = ceil_div(d, dc);
    if (grid > work_elems / ((int64_t)k * k)) grid = work_elems / ((int64_t)k * k);
    if (grid > 2 * 152) grid = 2 * 152;
    if (grid < 1) grid = 1;
    const size_t smem = (size_t)k * (dc + 1) * sizeof(double);
    k_gram_partial<<<(unsigned)grid, GRAM_THREADS, smem, s>>>(W, k, d, dc, work);
    DSANLS_LAUNCH_CHECK();
    const int64_t npairs = (int64_t)k * (k + 1) / 2;
    k_gram_reduce<<<(unsigned)ceil_div(npairs, 32), 256, 0, s>>>(work, (int)grid, k, G64);
    DSANLS_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// step size: lambda_max by power iteration, mu_t, eta_t
// ---------------------------------------------------------------------------
// One CTA of 256 threads: thread t works on row t / 2 of the power iteration
// (binary32, G in shared memory), the two threads of a row each summing one
// half of its columns; norms and the FP64 Rayleigh quotient x^T G x are
// reduced in a fixed order (warp shuffles, then the eight warp partials).
constexpr int STEP_THREADS = 256;

DSANLS_DEV float block_sum_f(float v, float *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float tot = 0.0f;
#pragma unroll
    for (int w = 0; w < STEP_THREADS / 32; ++w) tot += red[w];
    return tot;
}

DSANLS_DEV double block_sum_d(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < STEP_THREADS / 32; ++w) tot += red[w];
    return tot;
}

__global__ void __launch_bounds__(STEP_THREADS)
    k_step_size(const double *__restrict__ G64, int k, int iters, double alpha, double beta,
                const int64_t *__restrict__ t_dev, double *__restrict__ scal, float *__restrict__ Gf, int kp) {
    extern __shared__ float gs[];  // k x (k+1)
    __shared__ float x[128];
    __shared__ float redf[STEP_THREADS / 32];
    __shared__ double redd[2][STEP_THREADS / 32];
    const int tid = threadIdx.x;
    for (int e = tid; e < kp * kp; e += STEP_THREADS) {
        const int a = e / kp, b = e % kp;
        const float v = (a < k && b < k) ? (float)G64[a * k + b] : 0.0f;
        Gf[e] = v;
        if (a < k && b < k) gs[a * (k + 1) + b] = v;
    }
    const float x0 = rsqrtf((float)k);
    for (int i = tid; i < 128; i += STEP_THREADS) x[i] = (i < k) ? x0 : 0.0f;
    __syncthreads();
    const int row = tid >> 1, half = tid & 1;
    const int lh = (k + 1) / 2;
    const int l0 = half ? lh : 0, l1 = half ? k : lh;
    for (int it = 0; it < iters; ++it) {
        float a0 = 0.0f, a1 = 0.0f;
        if (row < k) {
            const float *gi = gs + row * (k + 1);
            int l = l0;
            for (; l + 1 < l1; l += 2) {
                a0 = fmaf(gi[l], x[l], a0);
                a1 = fmaf(gi[l + 1], x[l + 1], a1);
            }
            if (l < l1) a0 = fmaf(gi[l], x[l], a0);
        }
        float y = a0 + a1;
        y += __shfl_xor_sync(0xffffffffu, y, 1);  // both halves of the row
        const float nrm2 = block_sum_f(half == 0 && row < k ? y * y : 0.0f, redf);
        if (nrm2 == 0.0f) break;
        const float inv = rsqrtf(nrm2);
        if (half == 0 && row < k) x[row] = y * inv;
        __syncthreads();
    }
    // Rayleigh quotient in FP64; G is symmetric, so (G x)_i = sum_l G[l][i] x_l
    // (consecutive threads read consecutive entries of a row of G)
    double xgx = 0.0, xx = 0.0;
    if (tid < k) {
        double gx = 0.0;
        for (int l = 0; l < k; ++l) gx = fma(G64[l * k + tid], (double)x[l], gx);
        xgx = (double)x[tid] * gx;
        xx = (double)x[tid] * (double)x[tid];
    }
    xgx = block_sum_d(xgx, redd[0]);
    xx = block_sum_d(xx, redd[1]);
    if (tid == 0) {
        const double lam = xx > 0.0 ? xgx / xx : 0.0;
        const double mu = alpha + beta * (double)(*t_dev);
        scal[0] = lam;
        scal[1] = mu;
        scal[2] = 1.0 / (lam + mu);
    }
}

void launch_step_size(const double *G64, int k, int iters, double alpha, double beta, const int64_t *t_dev,
                      double *scal, float *Gf, int kp, cudaStream_t s) {
    if (k > 128) throw ArgError{"launch_step_size: k > 128"};
    const size_t smem = (size_t)k * (k + 1) * sizeof(float);
    k_step_size<<<1, STEP_THREADS, smem, s>>>(G64, k, iters, alpha, beta, t_dev, scal, Gf, kp);
    DSANLS_LAUNCH_CHECK();
}

__global__ void k_increment_t(int64_t *t, int64_t by) { *t += by; }

void launch_increment_t(int64_t *t_dev, int64_t by, cudaStream_t s) {
    k_increment_t<<<1, 1, 0, s>>>(t_dev, by);
    DSANLS_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// fused row update
// ---------------------------------------------------------------------------
constexpr int UPD_ROWS = 128;

DSANLS_DEV float project_clamp(float v, float bound, int *flag) {
    if (!(fabsf(v) <= 3.402823466e38f)) {  // NaN or Inf
        *flag = 1;
        return 0.0f;
    }
    float r = v > 0.0f ? v : 0.0f;
    if (bound > 0.0f) r = fminf(r, bound);
    return r;
}

template <int KP, int SOLVER>
__global__ void __launch_bounds__(UPD_ROWS)
    k_update(float *__restrict__ Z, const float *__restrict__ R, int64_t rows, int k, const float *__restrict__ Gf,
             const double *__restrict__ scal, float bound, int *__restrict__ flag) {
    extern __shared__ __align__(16) float sm[];
    float *gs = sm;                 // KP x KP, gs[l*KP + c] = G[l][c]
    float *zs = sm + KP * KP;       // UPD_ROWS x (k+1)
    const int ldz = k + 1;
    const int64_t r0 = (int64_t)blockIdx.x * UPD_ROWS;
    const int nr = (int)min((int64_t)UPD_ROWS, rows - r0);
    for (int e = threadIdx.x; e < KP * KP; e += blockDim.x) gs[e] = Gf[e];
    for (int e = threadIdx.x; e < nr * k; e += blockDim.x) {
        const int i = e / k, c = e % k;
        zs[i * ldz + c] = Z[(r0 + i) * k + c];
    }
    __syncthreads();
    const int i = threadIdx.x;
    if (i < nr) {
        float z[KP];
#pragma unroll
        for (int l = 0; l < KP; ++l) z[l] = (l < k) ? zs[i * ldz + l] : 0.0f;
        const float *r = R + (r0 + i) * k;
        if (SOLVER == 0) {
            const float eta = (float)scal[2];
#pragma unroll 1
            for (int c0 = 0; c0 < KP; c0 += 16) {
                float acc[16];
#pragma unroll
                for (int cc = 0; cc < 16; ++cc) acc[cc] = 0.0f;
#pragma unroll
                for (int l = 0; l < KP; ++l) {
                    const float zl = z[l];
#pragma unroll
                    for (int cc = 0; cc < 16; cc += 4) {
                        const float4 g = *reinterpret_cast<const float4 *>(&gs[l * KP + c0 + cc]);
                        acc[cc] = __fmaf_rn(zl, g.x, acc[cc]);
                        acc[cc + 1] = __fmaf_rn(zl, g.y, acc[cc + 1]);
                        acc[cc + 2] = __fmaf_rn(zl, g.z, acc[cc + 2]);
                        acc[cc + 3] = __fmaf_rn(zl, g.w, acc[cc + 3]);
                    }
                }
#pragma unroll
                for (int cc = 0; cc < 16; ++cc) {
                    const int c = c0 + cc;
                    if (c < k) {
                        const float zc = zs[i * ldz + c];  // not yet overwritten: column c belongs to this chunk
                        const float grad = __fsub_rn(acc[cc], r[c]);
                        zs[i * ldz + c] = project_clamp(__fmaf_rn(-eta, grad, zc), bound, flag);
                    }
                }
            }
        } else {
            const float mu = (float)scal[1];
#pragma unroll
            for (int j = 0; j < KP; ++j) {
                if (j < k) {
                    float tj = __fmaf_rn(mu, z[j], r[j]);
#pragma unroll
                    for (int l = 0; l < KP; ++l)
                        if (l != j) tj = __fmaf_rn(-gs[l * KP + j], z[l], tj);
                    const float den = __fadd_rn(gs[j * KP + j], mu);
                    z[j] = project_clamp(__fdiv_rn(tj, den), bound, flag);
                }
            }
#pragma unroll
            for (int l = 0; l < KP; ++l)
                if (l < k) zs[i * ldz + l] = z[l];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * k; e += blockDim.x) {
        const int ii = e / k, c = e % k;
        Z[(r0 + ii) * k + c] = zs[ii * ldz + c];
    }
}

// PGD update as a register-blocked product: a CTA owns 64 consecutive rows,
// whose Z and R entries form two contiguous ranges of 64 k floats; both are
// copied flat into shared memory with 16-byte asynchronous copies (R's copy
// overlaps the product).  Thread (ty, tx) computes rows 4ty..4ty+3 against TN
// = KP/16 columns of G: for TN >= 4 the columns tx*4 + 64 j + {0..3}, so that
// a warp's 16-byte loads of a G row are contiguous; for TN < 4 the columns
// tx*TN + {0..TN-1}.  One FMA chain per output in increasing l (the order of
// the row kernel).  The new rows are written back in place in shared memory
// and stored flat.
DSANLS_DEV void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
DSANLS_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
DSANLS_DEV void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int TN>
DSANLS_DEV int upd_col(int tx, int b) {
    if constexpr (TN >= 4)
        return (b >> 2) * 64 + tx * 4 + (b & 3);
    else
        return tx * TN + b;
}

// stage n floats from global src to shared dst with 16-byte copies (both
// 16-byte aligned); the n % 4 tail with plain loads
DSANLS_DEV void stage_flat(float *dst, const float *src, int n) {
    const int n4 = n >> 2;
    for (int e = threadIdx.x; e < n4; e += blockDim.x) cp_async16(dst + 4 * e, src + 4 * e);
    for (int e = 4 * n4 + threadIdx.x; e < n; e += blockDim.x) dst[e] = src[e];
}

template <int KP>
__global__ void __launch_bounds__(256)
    k_update_pgd_tiled(float *__restrict__ Z, const float *__restrict__ R, int64_t rows, int k,
                       const float *__restrict__ Gf, const double *__restrict__ scal, float bound, int inner,
                       int *__restrict__ flag) {
    constexpr int TN = KP / 16;
    constexpr int LDG = KP + 4;
    extern __shared__ __align__(16) float sm[];
    float *gs = sm;                // k x LDG, gs[l][c] = G[l][c] (c < KP, zero beyond k)
    float *zr = gs + k * LDG;      // 64 x k, row-major (the Z tile, then the new rows)
    float *rr = zr + 64 * k;       // 64 x k, the R tile
    // G once per CTA; the CTAs then walk the 64-row tiles
    for (int e = threadIdx.x; e < k * KP; e += 256) gs[(e / KP) * LDG + (e % KP)] = Gf[e];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const float eta = (float)scal[2];
    const float mu = (float)scal[1];
    const float *z0 = zr + (ty * 4) * k;
    const int64_t ntiles = (rows + 63) / 64;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * 64;
        const int nr = (int)min((int64_t)64, rows - r0);
        const int n = nr * k;
        stage_flat(zr, Z + r0 * k, n);
        cp_async_commit();
        stage_flat(rr, R + r0 * k, n);
        cp_async_commit();
        for (int e = n + threadIdx.x; e < 64 * k; e += 256) zr[e] = 0.0f;
        cp_async_wait<1>();  // the Z tile
        __syncthreads();
        for (int it = 0; it < inner; ++it) {
            float acc[4][TN];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < TN; ++b) acc[a][b] = 0.0f;
#pragma unroll 2
            for (int l = 0; l < k; ++l) {
                const float zv[4] = {z0[l], z0[k + l], z0[2 * k + l], z0[3 * k + l]};
                float gv[TN];
                const float *gl = gs + l * LDG;
                if constexpr (TN >= 4) {
#pragma unroll
                    for (int j = 0; j < TN / 4; ++j) {
                        const float4 g4 = *reinterpret_cast<const float4 *>(gl + j * 64 + tx * 4);
                        gv[4 * j] = g4.x;
                        gv[4 * j + 1] = g4.y;
                        gv[4 * j + 2] = g4.z;
                        gv[4 * j + 3] = g4.w;
                    }
                } else {
#pragma unroll
                    for (int b = 0; b < TN; ++b) gv[b] = gl[tx * TN + b];
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < TN; ++b) acc[a][b] = __fmaf_rn(zv[a], gv[b], acc[a][b]);
            }
            if (it == 0) {
                cp_async_wait<0>();  // the R tile
                __syncthreads();     // every thread is done reading the Z tile
                if (inner > 1) {
                    // b = r + mu u, kept in the R tile for the steps on the proximal objective
                    for (int e = threadIdx.x; e < n; e += 256) rr[e] = __fmaf_rn(mu, zr[e], rr[e]);
                    __syncthreads();
                }
            } else {
                __syncthreads();
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int i = ty * 4 + a;
                if (i >= nr) continue;
#pragma unroll
                for (int b = 0; b < TN; ++b) {
                    const int c = upd_col<TN>(tx, b);
                    if (c < k) {
                        const float x = zr[i * k + c];
                        // one step: the gradient of eq. gradient_descent (r in the tile);
                        // several: (G + mu I) x - (r + mu u) (b in the tile)
                        const float grad = inner > 1 ? __fsub_rn(__fmaf_rn(mu, x, acc[a][b]), rr[i * k + c])
                                                     : __fsub_rn(acc[a][b], rr[i * k + c]);
                        zr[i * k + c] = project_clamp(__fmaf_rn(-eta, grad, x), bound, flag);
                    }
                }
            }
            __syncthreads();  // the new rows are complete before the next product reads them
        }
        float *zo = Z + r0 * k;
        const int n4 = n >> 2;
        for (int e = threadIdx.x; e < n4; e += 256)
            reinterpret_cast<float4 *>(zo)[e] = reinterpret_cast<const float4 *>(zr)[e];
        for (int e = 4 * n4 + threadIdx.x; e < n; e += 256) zo[e] = zr[e];
        __syncthreads();  // the tile has left shared memory before the next one is staged
    }
}

template <int KP>
static void update_kp(int solver, float *Z, const float *R, int64_t rows, int k, const float *Gf,
                      const double *scal, float bound, int inner, int *flag, cudaStream_t s) {
    if (solver == 0) {
        const size_t smem_t = ((size_t)k * (KP + 4) + 2 * 64 * (size_t)k) * sizeof(float);
        // persistent: as many CTAs as fit on the GPU at once (G is staged once per CTA)
        int per_sm = 1, sms = 152, dev = 0;
        DSANLS_CUDA(cudaGetDevice(&dev));
        DSANLS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        DSANLS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update_pgd_tiled<KP>, 256, smem_t));
        const int64_t grid = std::min<int64_t>(ceil_div(rows, 64), (int64_t)std::max(1, per_sm) * sms);
        k_update_pgd_tiled<KP><<<(unsigned)grid, 256, smem_t, s>>>(Z, R, rows, k, Gf, scal, bound, inner, flag);
        DSANLS_LAUNCH_CHECK();
        return;
    }
    const size_t smem = (size_t)(KP * KP + UPD_ROWS * (k + 1)) * sizeof(float);
    const unsigned grid = (unsigned)ceil_div(rows, UPD_ROWS);
    k_update<KP, 1><<<grid, UPD_ROWS, smem, s>>>(Z, R, rows, k, Gf, scal, bound, flag);
    DSANLS_LAUNCH_CHECK();
}

void prime_solver_attributes(int max_smem) {
    allow_max_dynamic_smem(k_gram_partial, max_smem);
    allow_max_dynamic_smem(k_step_size, max_smem);
    allow_max_dynamic_smem(k_update_pgd_tiled<16>, max_smem);
    allow_max_dynamic_smem(k_update_pgd_tiled<32>, max_smem);
    allow_max_dynamic_smem(k_update_pgd_tiled<64>, max_smem);
    allow_max_dynamic_smem(k_update_pgd_tiled<128>, max_smem);
    allow_max_dynamic_smem(k_update<16, 0>, max_smem);
    allow_max_dynamic_smem(k_update<16, 1>, max_smem);
    allow_max_dynamic_smem(k_update<32, 0>, max_smem);
    allow_max_dynamic_smem(k_update<32, 1>, max_smem);
    allow_max_dynamic_smem(k_update<64, 0>, max_smem);
    allow_max_dynamic_smem(k_update<64, 1>, max_smem);
    allow_max_dynamic_smem(k_update<128, 0>, max_smem);
    allow_max_dynamic_smem(k_update<128, 1>, max_smem);
}

void launch_update(int solver, float *Z, const float *R, int64_t rows, int k, const float *Gf, int kp,
                   const double *scal, float bound, int inner, int *flag, cudaStream_t s) {
    if (rows <= 0) return;
    if (inner < 1 || (inner > 1 && solver != 0)) throw ArgError{"launch_update: inner steps need PGD"};
    if (kp <= 16)
        update_kp<16>(solver, Z, R, rows, k, Gf, scal, bound, inner, flag, s);
    else if (kp <= 32)
        update_kp<32>(solver, Z, R, rows, k, Gf, scal, bound, inner, flag, s);
    else if (kp <= 64)
        update_kp<64>(solver, Z, R, rows, k, Gf, scal, bound, inner, flag, s);
    else
        update_kp<128>(solver, Z, R, rows, k, Gf, scal, bound, inner, flag, s);
}

}  // namespace dsanls
