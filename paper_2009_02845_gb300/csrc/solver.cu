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
#include "tc_gemm.cuh"

namespace dsanls {

// ---------------------------------------------------------------------------
// Gram in FP64
// ---------------------------------------------------------------------------
// Each CTA sums chunks blockIdx.x, blockIdx.x + gridDim.x, ... of dc columns
// of the d axis.  A chunk is staged in shared memory already converted to FP64
// (one conversion per entry, not one per product: the FP64 pipe is the scarce
// unit), column by column (ws[j][a], rows padded to 4 * ceil(k/4) + 2 doubles).
// Thread p owns the 4 x 4 tile (bi, bj), bi <= bj, of the p-th block of the
// upper triangle (row-major): 16 independent FP64 accumulators fed by two
// 32-byte loads per column, so the FP64 pipe, not latency, bounds the kernel.
// Every pair a <= b is summed over the CTA's columns in increasing order.
constexpr int GRAM_TILE = 4;
constexpr int GRAM_MAX_THREADS = 544;  // 528 tiles at k = 128, rounded up to warps

__global__ void __launch_bounds__(GRAM_MAX_THREADS)
    k_gram_partial(const float *__restrict__ W, int k, int64_t d, int dc, double *__restrict__ part) {
    extern __shared__ __align__(16) double ws[];
    const int kb = (k + GRAM_TILE - 1) / GRAM_TILE;
    const int ldw = GRAM_TILE * kb + 2;  // 16-byte rows; the +2 staggers the banks of successive columns
    const int nb = kb * (kb + 1) / 2;
    const int p = threadIdx.x;
    int bi = 0, rem = p;
    if (p < nb)
        while (rem >= kb - bi) {
            rem -= kb - bi;
            ++bi;
        }
    const int bj = bi + rem;
    double acc[GRAM_TILE][GRAM_TILE];
#pragma unroll
    for (int r = 0; r < GRAM_TILE; ++r)
#pragma unroll
        for (int c = 0; c < GRAM_TILE; ++c) acc[r][c] = 0.0;
    const int64_t chunks = ceil_div(d, (int64_t)dc);
    const int rows_p = GRAM_TILE * kb;
    for (int64_t ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
        const int64_t j0 = ch * dc;
        const int len = (int)min((int64_t)dc, d - j0);
        __syncthreads();  // the previous chunk has been consumed
        for (int e = threadIdx.x; e < rows_p * dc; e += blockDim.x) {
            const int a = e / dc, j = e - a * dc;  // consecutive threads read consecutive columns of a row
            ws[j * ldw + a] = (a < k && j < len) ? (double)W[(int64_t)a * d + j0 + j] : 0.0;
        }
        __syncthreads();
        if (p < nb) {
            const double *wa = ws + GRAM_TILE * bi;
            const double *wb = ws + GRAM_TILE * bj;
            for (int j = 0; j < len; ++j) {
                const double2 a01 = *reinterpret_cast<const double2 *>(wa + j * ldw);
                const double2 a23 = *reinterpret_cast<const double2 *>(wa + j * ldw + 2);
                const double2 b01 = *reinterpret_cast<const double2 *>(wb + j * ldw);
                const double2 b23 = *reinterpret_cast<const double2 *>(wb + j * ldw + 2);
                const double av[GRAM_TILE] = {a01.x, a01.y, a23.x, a23.y};
                const double bv[GRAM_TILE] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
                for (int r = 0; r < GRAM_TILE; ++r)
#pragma unroll
                    for (int c = 0; c < GRAM_TILE; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
            }
        }
    }
    if (p < nb) {
        double *out = part + (int64_t)blockIdx.x * k * k;
#pragma unroll
        for (int r = 0; r < GRAM_TILE; ++r)
#pragma unroll
            for (int c = 0; c < GRAM_TILE; ++c) {
                const int a = GRAM_TILE * bi + r, b = GRAM_TILE * bj + c;
                if (a < k && b < k && a <= b) out[a * k + b] = acc[r][c];
            }
    }
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
    if (k < 1 || k > 128) throw ArgError{"launch_gram: k must be in [1, 128]"};
    const int kb = (k + GRAM_TILE - 1) / GRAM_TILE;
    const int nb = kb * (kb + 1) / 2;
    const int threads = (int)ceil_div(nb, 32) * 32;
    const int ldw = GRAM_TILE * kb + 2;
    // chunk width: about two chunks per SM, a multiple of 4, at most ~96 KB of
    // shared memory (two CTAs per SM)
    int64_t dc = ceil_div(ceil_div(d, 2 * 152), 4) * 4;
    const int64_t dc_max = std::max<int64_t>(4, (96 * 1024) / (8 * (int64_t)ldw));
    if (dc > dc_max) dc = dc_max;
    if (dc < 4) dc = 4;
    int64_t grid = ceil_div(d, dc);
    if (grid > work_elems / ((int64_t)k * k)) grid = work_elems / ((int64_t)k * k);
    if (grid > 2 * 152) grid = 2 * 152;
    if (grid < 1) grid = 1;
    const size_t smem = (size_t)dc * ldw * sizeof(double);
    k_gram_partial<<<(unsigned)grid, threads, smem, s>>>(W, k, d, (int)dc, work);
    DSANLS_LAUNCH_CHECK();
    const int64_t npairs = (int64_t)k * (k + 1) / 2;
    k_gram_reduce<<<(unsigned)ceil_div(npairs, 32), 256, 0, s>>>(work, (int)grid, k, G64);
    DSANLS_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// step size: lambda_max by power iteration, mu_t, eta_t
// ---------------------------------------------------------------------------
// One CTA of 256 threads.  G is staged once in shared memory in FP64 (all
// loads in flight together), written out as the padded kp x kp binary32 copy
// the update reads, and held in registers for the power iteration: thread
// (a, b), a = 2 warp + lane / 16, b = lane % 16, keeps the T x T tile of rows
// aT.. and columns bT.. (16T >= k, zero padded).  One iteration: a T x T
// product with its slice of x, a butterfly over the 16 lanes of the row block
// (every lane ends with the same row sums), the squared norm from the warp's
// two row blocks, and one block barrier: the normalisation is applied lazily
// (each iteration writes the unnormalised y = G x and the warp partials of
// |y|^2 to the other of two buffers; the next one scales its product by 1/|y|,
// the sum of the partials taken in warp order in every thread).  The FP64
// Rayleigh quotient x^T G x / x^T x reads the FP64 copy (G symmetric:
// consecutive threads read consecutive entries of a row) and is reduced in a
// fixed order over the CTA.
constexpr int STEP_THREADS = 256;

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

template <int T>
__global__ void __launch_bounds__(STEP_THREADS)
    k_step_size(const double *__restrict__ G64, int k, int iters, double alpha, double beta,
                const int64_t *__restrict__ t_dev, double *__restrict__ scal, float *__restrict__ Gf, int kp) {
    extern __shared__ __align__(16) double gd[];  // k x k FP64
    __shared__ float xb[2][16 * T];
    __shared__ float red[2][STEP_THREADS / 32];
    __shared__ double redd[2][STEP_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < k * k; e += STEP_THREADS) gd[e] = G64[e];
    // x_0 = 1/sqrt(k): buffer 0 holds the all-ones vector and |.|^2 = k
    for (int i = tid; i < 16 * T; i += STEP_THREADS) xb[0][i] = (i < k) ? 1.0f : 0.0f;
    if (tid < STEP_THREADS / 32) red[0][tid] = tid == 0 ? (float)k : 0.0f;
    __syncthreads();
    for (int e = tid; e < kp * kp; e += STEP_THREADS) {
        const int a = e / kp, b = e % kp;
        Gf[e] = (a < k && b < k) ? (float)gd[a * k + b] : 0.0f;
    }
    const int ab = 2 * warp + (lane >> 4), bb = lane & 15;
    float g[T][T];
#pragma unroll
    for (int r = 0; r < T; ++r)
#pragma unroll
        for (int c = 0; c < T; ++c) {
            const int i = ab * T + r, j = bb * T + c;
            g[r][c] = (i < k && j < k) ? (float)gd[i * k + j] : 0.0f;
        }
    int cur = 0;
    for (int it = 0; it < iters; ++it) {
        float tot = 0.0f;
#pragma unroll
        for (int w = 0; w < STEP_THREADS / 32; ++w) tot += red[cur][w];
        if (tot == 0.0f) break;  // G x = 0 (the same decision in every thread)
        const float inv = rsqrtf(tot);
        float xv[T], p[T];
#pragma unroll
        for (int c = 0; c < T; ++c) xv[c] = xb[cur][bb * T + c];
#pragma unroll
        for (int r = 0; r < T; ++r) {
            float acc = 0.0f;
#pragma unroll
            for (int c = 0; c < T; ++c) acc = fmaf(g[r][c], xv[c], acc);
            p[r] = acc;
        }
#pragma unroll
        for (int o = 1; o < 16; o <<= 1)
#pragma unroll
            for (int r = 0; r < T; ++r) p[r] += __shfl_xor_sync(0xffffffffu, p[r], o);
        float sq = 0.0f;
#pragma unroll
        for (int r = 0; r < T; ++r) {
            p[r] *= inv;
            sq = fmaf(p[r], p[r], sq);
        }
        sq += __shfl_xor_sync(0xffffffffu, sq, 16);  // the warp's two row blocks
        const int nxt = cur ^ 1;
#pragma unroll
        for (int r = 0; r < T; ++r)
            if (r == bb) xb[nxt][ab * T + r] = p[r];
        if (lane == 0) red[nxt][warp] = sq;
        __syncthreads();
        cur = nxt;
    }
    float tot = 0.0f;
#pragma unroll
    for (int w = 0; w < STEP_THREADS / 32; ++w) tot += red[cur][w];
    const float inv = tot > 0.0f ? rsqrtf(tot) : 0.0f;
    // Rayleigh quotient in FP64: thread t takes row i = t % k, column segment t / k
    const int nseg = STEP_THREADS / k;  // >= 2 for k <= 128
    const int i = tid % k, seg = tid / k;
    const int seglen = (k + nseg - 1) / nseg;
    double xgx = 0.0, xx = 0.0;
    if (seg < nseg) {
        const int c0 = seg * seglen, c1 = min(k, c0 + seglen);
        double gx = 0.0;
        for (int l = c0; l < c1; ++l) gx = fma(gd[l * k + i], (double)(xb[cur][l] * inv), gx);
        const double xi = (double)(xb[cur][i] * inv);
        xgx = xi * gx;
        if (seg == 0) xx = xi * xi;
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
    if (k < 1 || k > 128) throw ArgError{"launch_step_size: k must be in [1, 128]"};
    const size_t smem = (size_t)k * k * sizeof(double);
    if (k <= 16)
        k_step_size<1><<<1, STEP_THREADS, smem, s>>>(G64, k, iters, alpha, beta, t_dev, scal, Gf, kp);
    else if (k <= 32)
        k_step_size<2><<<1, STEP_THREADS, smem, s>>>(G64, k, iters, alpha, beta, t_dev, scal, Gf, kp);
    else if (k <= 64)
        k_step_size<4><<<1, STEP_THREADS, smem, s>>>(G64, k, iters, alpha, beta, t_dev, scal, Gf, kp);
    else
        k_step_size<8><<<1, STEP_THREADS, smem, s>>>(G64, k, iters, alpha, beta, t_dev, scal, Gf, kp);
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
    allow_max_dynamic_smem(k_step_size<1>, max_smem);
    allow_max_dynamic_smem(k_step_size<2>, max_smem);
    allow_max_dynamic_smem(k_step_size<4>, max_smem);
    allow_max_dynamic_smem(k_step_size<8>, max_smem);
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
    if (solver == 0 && inner == 1 && update_tc_supported(k)) {
        // one projected-gradient step with Z G on tensor cores (split bf16, binary32 accuracy)
        launch_update_tc(Z, R, rows, k, Gf, kp, scal, bound, flag, s);
        return;
    }
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
