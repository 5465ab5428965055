// Learned warm start for the proximal row subproblem of a half-step:
//     f(x) = 1/2 x^T (G + mu I) x - (r + mu u)^T x,  x >= 0     (eq. reg_sub)
// A small MLP maps the normalised (G, b = r + mu u) to a starting point, a
// few projected-gradient steps on f correct it, and the plain projected
// gradient step of eq. gradient_descent is kept whenever its objective is
// lower (fallback).
//
// Network (k <= 32, hidden h <= 256), parameters theta in this order:
//   W1g (h x k*k), W1b (h x k), b1 (h), W2 (h x h), b2 (h), W3 (k x h), b3 (k)
//   h1 = GELU(W1g vec(Gn) + W1b bn + b1), h2 = GELU(W2 h1 + b2),
//   y  = ReLU(W3 h2 + b3)
//   Gn = (G + mu I) / s, s = tr(G + mu I) / k; bn = b / beta, beta = ||b|| / sqrt(k)
// The weights used by the forward and backward passes are the fp32 master
// weights rounded to bf16 (bf16 weights, fp32 accumulation); Adam updates the
// fp32 masters.  All matrix products go through the CUDA-core GEMM of
// gemm_simt.cu (deterministic); GELU is the exact x Phi(x) (normcdff).
// Rows are grouped by subproblem: rows group_off[g] .. group_off[g+1]-1 share
// G_g and mu_g.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "mlp.cuh"

namespace dsanls {

namespace {

DSANLS_DEV float gelu_f(float x) { return x * normcdff(x); }
DSANLS_DEV float gelu_grad_f(float x) { return normcdff(x) + x * 0.3989422804014327f * __expf(-0.5f * x * x); }

DSANLS_DEV float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void k_round_bf16(const float *__restrict__ in, int64_t n, float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = round_bf16(in[i]);
}

// per group: s_g and Gn_g
__global__ void k_norm_groups(const float *__restrict__ G, const float *__restrict__ mu, int k, int ngroups,
                              float *__restrict__ Gn, float *__restrict__ s_out) {
    const int g = blockIdx.x;
    if (g >= ngroups) return;
    __shared__ float s_sh;
    const float *Gg = G + (int64_t)g * k * k;
    if (threadIdx.x == 0) {
        float tr = 0.0f;
        for (int i = 0; i < k; ++i) tr += Gg[i * k + i];
        s_sh = (tr + k * mu[g]) / k;
        s_out[g] = s_sh;
    }
    __syncthreads();
    const float inv = 1.0f / s_sh;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int i = e / k, j = e % k;
        Gn[(int64_t)g * k * k + e] = (Gg[e] + (i == j ? mu[g] : 0.0f)) * inv;
    }
}

// per row: beta and bn; the row's group is found from group_off
DSANLS_DEV int group_of(const int64_t *off, int ngroups, int64_t r) {
    int lo = 0, hi = ngroups;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= r)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__global__ void k_norm_rows(const float *__restrict__ b, int64_t rows, int k, float *__restrict__ bn,
                            float *__restrict__ beta) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float ss = 0.0f;
    for (int j = 0; j < k; ++j) ss = fmaf(b[r * k + j], b[r * k + j], ss);
    float bt = sqrtf(ss / k);
    if (!(bt > 0.0f)) bt = 1.0f;
    beta[r] = bt;
    const float inv = 1.0f / bt;
    for (int j = 0; j < k; ++j) bn[r * k + j] = b[r * k + j] * inv;
}

// z1 += zg[group] + b1 (in place), h1 = GELU(z1)
__global__ void k_layer1_finish(float *__restrict__ z1, float *__restrict__ h1, const float *__restrict__ zg,
                                const float *__restrict__ b1, const int64_t *__restrict__ off, int ngroups,
                                int64_t rows, int h) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * h) return;
    const int64_t r = idx / h;
    const int j = (int)(idx % h);
    const int g = group_of(off, ngroups, r);
    const float z = z1[idx] + zg[(int64_t)g * h + j] + b1[j];
    z1[idx] = z;
    h1[idx] = gelu_f(z);
}

// z += bias (per column), act = GELU(z) or ReLU(z)
__global__ void k_bias_act(float *__restrict__ z, float *__restrict__ act, const float *__restrict__ bias,
                           int64_t rows, int cols, int relu) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const float v = z[idx] + bias[idx % cols];
    z[idx] = v;
    act[idx] = relu ? fmaxf(v, 0.0f) : gelu_f(v);
}

// e = o - y* where y* > 0, max(o, 0) where y* = 0 (o before the ReLU);
// do = e / N; per-row loss 1/2 ||e||^2.  Equal to the squared error of the
// ReLU output except where o < 0 < y*, where it keeps a gradient.  ys and
// dout may be the same array (each element is read before it is written).
__global__ void k_out_grad(const float *__restrict__ o, const float *ys, int64_t rows, int k, float invN, float *dout,
                           double *__restrict__ rowloss) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    double l = 0.0;
    for (int j = 0; j < k; ++j) {
        const float oj = o[r * k + j], t = ys[r * k + j];
        const float e = t > 0.0f ? oj - t : fmaxf(oj, 0.0f);
        l += 0.5 * (double)e * (double)e;
        dout[r * k + j] = e * invN;
    }
    rowloss[r] = l;
}

// dz = dh * GELU'(z)
__global__ void k_gelu_back(const float *__restrict__ z, float *__restrict__ dh, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dh[i] *= gelu_grad_f(z[i]);
}

// out[g * cols + j] = sum over rows off[g] <= r < off[g+1] of X[r * cols + j] (row order)
__global__ void k_segment_colsum(const float *__restrict__ X, const int64_t *__restrict__ off, int nseg, int cols,
                                 float *__restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nseg * cols) return;
    const int g = (int)(idx / cols), j = (int)(idx % cols);
    float acc = 0.0f;
    for (int64_t r = off[g]; r < off[g + 1]; ++r) acc += X[r * cols + j];
    out[idx] = acc;
}

__global__ void k_sum_doubles(const double *__restrict__ x, int64_t n, double scale, double *__restrict__ out) {
    __shared__ double red[256];
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v += x[i];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] * scale;
}

__global__ void k_adam(float *__restrict__ theta, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, int64_t n, float lr, float b1, float b2, float c1, float c2,
                       float eps) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_g_to_float(const double *__restrict__ G64, int k, const double *__restrict__ scal,
                             float *__restrict__ gf, float *__restrict__ mu, int64_t *__restrict__ off, int64_t rows) {
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) gf[e] = (float)G64[e];
    if (threadIdx.x == 0) {
        mu[0] = (float)scal[1];
        off[0] = 0;
        off[1] = rows;
    }
}

__global__ void k_rhs_b(const float *__restrict__ R, const float *__restrict__ Z, const double *__restrict__ scal,
                        int64_t n, float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __fmaf_rn((float)scal[1], Z[i], R[i]);
}

unsigned nblk(int64_t n) { return (unsigned)ceil_div(n, 256); }

GemmArgs gemm(int64_t M, int64_t N, int64_t K, const float *A, int64_t lda, bool ak, const float *B, int64_t ldb,
              bool bk, float *C, int64_t ldc) {
    GemmArgs g{};
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda; g.a_kcontig = ak;
    g.B = B; g.ldb = ldb; g.b_kcontig = bk;
    g.C = C; g.ldc = ldc; g.alpha = 1.0f; g.splits = 1;
    return g;
}

}  // namespace

int64_t mlp_param_count(int k, int h) { return (int64_t)h * k * k + (int64_t)h * k + h + (int64_t)h * h + h + (int64_t)k * h + k; }

MlpOffsets mlp_offsets(int k, int h) {
    MlpOffsets o;
    o.W1g = 0;
    o.W1b = o.W1g + (int64_t)h * k * k;
    o.b1 = o.W1b + (int64_t)h * k;
    o.W2 = o.b1 + h;
    o.b2 = o.W2 + (int64_t)h * h;
    o.W3 = o.b2 + h;
    o.b3 = o.W3 + (int64_t)k * h;
    o.total = o.b3 + k;
    return o;
}

void mlp_alloc(MlpState &st, int k, int h, int64_t max_rows, int max_groups) {
    st.k = k;
    st.h = h;
    st.max_rows = max_rows;
    st.max_groups = max_groups;
    const int64_t P = mlp_param_count(k, h);
    auto al = [](auto *&p, int64_t n) {
        if (cudaMalloc((void **)&p, (size_t)std::max<int64_t>(n, 1) * sizeof(*p)) != cudaSuccess) {
            cudaGetLastError();
            throw std::bad_alloc();
        }
    };
    al(st.theta, P); al(st.wq, P); al(st.grad, P); al(st.m, P); al(st.v, P);
    al(st.Gn, (int64_t)max_groups * k * k); al(st.s, max_groups); al(st.zg, (int64_t)max_groups * h);
    al(st.dzg, (int64_t)max_groups * h);
    al(st.bn, max_rows * k); al(st.beta, max_rows);
    al(st.z1, max_rows * h); al(st.h1, max_rows * h); al(st.z2, max_rows * h); al(st.h2, max_rows * h);
    al(st.o, max_rows * k); al(st.y, max_rows * k); al(st.dout, max_rows * k); al(st.rowloss, max_rows);
    al(st.loss, 1); al(st.all_off, 2);
    al(st.gf1, (int64_t)k * k); al(st.mu1, 1); al(st.off1, 2);
    DSANLS_CUDA(cudaMemset(st.m, 0, P * sizeof(float)));
    DSANLS_CUDA(cudaMemset(st.v, 0, P * sizeof(float)));
    const int64_t zero_n[2] = {0, 0};
    DSANLS_CUDA(cudaMemcpy(st.all_off, zero_n, sizeof zero_n, cudaMemcpyHostToDevice));
}

void mlp_free(MlpState &st) {
    for (void *p : {(void *)st.theta, (void *)st.wq, (void *)st.grad, (void *)st.m, (void *)st.v, (void *)st.Gn,
                    (void *)st.s, (void *)st.zg, (void *)st.dzg, (void *)st.bn, (void *)st.beta, (void *)st.z1,
                    (void *)st.h1, (void *)st.z2, (void *)st.h2, (void *)st.o, (void *)st.y, (void *)st.dout,
                    (void *)st.rowloss, (void *)st.loss, (void *)st.all_off, (void *)st.gf1, (void *)st.mu1,
                    (void *)st.off1})
        if (p) cudaFree(p);
    st = MlpState{};
}

void mlp_quantise(MlpState &st, cudaStream_t s) {
    const int64_t P = mlp_param_count(st.k, st.h);
    k_round_bf16<<<nblk(P), 256, 0, s>>>(st.theta, P, st.wq);
    DSANLS_LAUNCH_CHECK();
}

// Forward pass: y (rows x k, normalised output) in st.y; o, z1, h1, z2, h2 kept.
void mlp_forward(MlpState &st, const float *G, const float *mu, const int64_t *off, int ngroups, const float *b,
                 int64_t rows, cudaStream_t s) {
    const int k = st.k, h = st.h;
    const MlpOffsets O = mlp_offsets(k, h);
    const float *W = st.wq;
    k_norm_groups<<<ngroups, 128, 0, s>>>(G, mu, k, ngroups, st.Gn, st.s);
    DSANLS_LAUNCH_CHECK();
    launch_sgemm(gemm(ngroups, h, (int64_t)k * k, st.Gn, (int64_t)k * k, true, W + O.W1g, (int64_t)k * k, true, st.zg,
                      h),
                 s);
    k_norm_rows<<<nblk(rows), 256, 0, s>>>(b, rows, k, st.bn, st.beta);
    DSANLS_LAUNCH_CHECK();
    launch_sgemm(gemm(rows, h, k, st.bn, k, true, W + O.W1b, k, true, st.z1, h), s);
    k_layer1_finish<<<nblk(rows * h), 256, 0, s>>>(st.z1, st.h1, st.zg, W + O.b1, off, ngroups, rows, h);
    DSANLS_LAUNCH_CHECK();
    launch_sgemm(gemm(rows, h, h, st.h1, h, true, W + O.W2, h, true, st.z2, h), s);
    k_bias_act<<<nblk(rows * h), 256, 0, s>>>(st.z2, st.h2, W + O.b2, rows, h, 0);
    DSANLS_LAUNCH_CHECK();
    launch_sgemm(gemm(rows, k, h, st.h2, h, true, W + O.W3, h, true, st.o, k), s);
    k_bias_act<<<nblk(rows * k), 256, 0, s>>>(st.o, st.y, W + O.b3, rows, k, 1);
    DSANLS_LAUNCH_CHECK();
}

// Loss and gradient (into st.grad) of the one-sided squared error (k_out_grad) after mlp_forward.
void mlp_backward(MlpState &st, const int64_t *off, int ngroups, const float *ystar, int64_t rows, cudaStream_t s) {
    const int k = st.k, h = st.h;
    const MlpOffsets O = mlp_offsets(k, h);
    const float *W = st.wq;
    float *dG = st.grad;
    k_out_grad<<<nblk(rows), 256, 0, s>>>(st.o, ystar, rows, k, 1.0f / (float)rows, st.dout, st.rowloss);
    DSANLS_LAUNCH_CHECK();
    k_sum_doubles<<<1, 256, 0, s>>>(st.rowloss, rows, 1.0 / (double)rows, st.loss);  // mean over rows
    DSANLS_LAUNCH_CHECK();
    // dW3 = do^T h2, db3 = colsum(do)
    launch_sgemm(gemm(k, h, rows, st.dout, k, false, st.h2, h, false, dG + O.W3, h), s);
    const int64_t hostoff[2] = {0, rows};
    DSANLS_CUDA(cudaMemcpyAsync(st.all_off, hostoff, sizeof hostoff, cudaMemcpyHostToDevice, s));
    k_segment_colsum<<<nblk(k), 256, 0, s>>>(st.dout, st.all_off, 1, k, dG + O.b3);
    DSANLS_LAUNCH_CHECK();
    // dh2 = do W3 -> dz2 (in h2's buffer)
    launch_sgemm(gemm(rows, h, k, st.dout, k, true, W + O.W3, h, false, st.h2, h), s);
    k_gelu_back<<<nblk(rows * h), 256, 0, s>>>(st.z2, st.h2, rows * h);
    DSANLS_LAUNCH_CHECK();
    // dW2 = dz2^T h1, db2
    launch_sgemm(gemm(h, h, rows, st.h2, h, false, st.h1, h, false, dG + O.W2, h), s);
    k_segment_colsum<<<nblk(h), 256, 0, s>>>(st.h2, st.all_off, 1, h, dG + O.b2);
    DSANLS_LAUNCH_CHECK();
    // dh1 = dz2 W2 -> dz1 (in h1's buffer)
    launch_sgemm(gemm(rows, h, h, st.h2, h, true, W + O.W2, h, false, st.h1, h), s);
    k_gelu_back<<<nblk(rows * h), 256, 0, s>>>(st.z1, st.h1, rows * h);
    DSANLS_LAUNCH_CHECK();
    // dW1b = dz1^T bn, db1, per-group dzg and dW1g = dzg^T Gn
    launch_sgemm(gemm(h, k, rows, st.h1, h, false, st.bn, k, false, dG + O.W1b, k), s);
    k_segment_colsum<<<nblk(h), 256, 0, s>>>(st.h1, st.all_off, 1, h, dG + O.b1);
    DSANLS_LAUNCH_CHECK();
    k_segment_colsum<<<nblk((int64_t)ngroups * h), 256, 0, s>>>(st.h1, off, ngroups, h, st.dzg);
    DSANLS_LAUNCH_CHECK();
    launch_sgemm(gemm(h, (int64_t)k * k, ngroups, st.dzg, h, false, st.Gn, (int64_t)k * k, false, dG + O.W1g,
                      (int64_t)k * k),
                 s);
}

void mlp_adam(MlpState &st, float lr, cudaStream_t s) {
    const int64_t P = mlp_param_count(st.k, st.h);
    st.adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)st.adam_t), c2 = 1.0f - std::pow(b2, (float)st.adam_t);
    k_adam<<<nblk(P), 256, 0, s>>>(st.theta, st.m, st.v, st.grad, P, lr, b1, b2, c1, c2, 1e-8f);
    DSANLS_LAUNCH_CHECK();
    mlp_quantise(st, s);
}

__global__ void k_init_segment(float *__restrict__ theta, int64_t off, int64_t n, float a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) theta[off + i] = a * (2.0f * theta[off + i] - 1.0f);
}

void mlp_init(MlpState &st, uint64_t seed, cudaStream_t s) {
    const int k = st.k, h = st.h;
    const MlpOffsets O = mlp_offsets(k, h);
    launch_uniform_field(seed, 0x20, 0, O.total, 1, st.theta, s);
    struct Seg {
        int64_t off, n;
        float fan_in;
    };
    const Seg segs[7] = {{O.W1g, (int64_t)h * k * k, (float)(k * k + k)}, {O.W1b, (int64_t)h * k, (float)(k * k + k)},
                         {O.b1, h, 0.0f}, {O.W2, (int64_t)h * h, (float)h}, {O.b2, h, 0.0f},
                         {O.W3, (int64_t)k * h, (float)h}, {O.b3, k, 0.0f}};
    for (const Seg &g : segs) {
        const float a = g.fan_in > 0.0f ? std::sqrt(3.0f / g.fan_in) : 0.0f;
        k_init_segment<<<nblk(g.n), 256, 0, s>>>(st.theta, g.off, g.n, a);
        DSANLS_LAUNCH_CHECK();
    }
    mlp_quantise(st, s);
}

__global__ void k_targets(const float *__restrict__ xstar, const float *__restrict__ s_g,
                          const float *__restrict__ beta, const int64_t *__restrict__ off, int ngroups, int64_t rows,
                          int k, float *__restrict__ ys) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * k) return;
    const int64_t r = idx / k;
    ys[idx] = xstar[idx] * s_g[group_of(off, ngroups, r)] / beta[r];
}

__global__ void k_unscale(const float *__restrict__ y, const float *__restrict__ s_g, const float *__restrict__ beta,
                          const int64_t *__restrict__ off, int ngroups, int64_t rows, int k, float *__restrict__ x) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * k) return;
    const int64_t r = idx / k;
    x[idx] = y[idx] * beta[r] / s_g[group_of(off, ngroups, r)];
}

void mlp_targets(MlpState &st, const int64_t *off, int ngroups, const float *xstar, int64_t rows, cudaStream_t s) {
    k_targets<<<nblk(rows * st.k), 256, 0, s>>>(xstar, st.s, st.beta, off, ngroups, rows, st.k, st.dout);
    DSANLS_LAUNCH_CHECK();
}

void mlp_unscale(MlpState &st, const int64_t *off, int ngroups, int64_t rows, float *x_out, cudaStream_t s) {
    k_unscale<<<nblk(rows * st.k), 256, 0, s>>>(st.y, st.s, st.beta, off, ngroups, rows, st.k, x_out);
    DSANLS_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// learned update of one half-step (k <= 32): one warp per row, lane c owns
// column c of the row; (x G)_c = sum_l x_l G[l][c] with x_l broadcast from
// lane l (an FMA chain in increasing l)
// ---------------------------------------------------------------------------
constexpr int LF_THREADS = 256;

DSANLS_DEV float row_times_g(float x, float init, const float (*gs)[33], int lane) {
    float acc = init;
#pragma unroll
    for (int l = 0; l < 32; ++l) acc = __fmaf_rn(__shfl_sync(0xffffffffu, x, l), gs[l][lane], acc);
    return acc;
}

DSANLS_DEV float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(LF_THREADS)
    k_learned_finish(float *__restrict__ Z, const float *__restrict__ R, const float *__restrict__ y,
                     const float *__restrict__ beta, const float *__restrict__ s_g, const float *__restrict__ Gf,
                     int kp, const double *__restrict__ scal, int64_t rows, int k, int pg_iters, int plain_iters,
                     unsigned long long *__restrict__ kept, int *__restrict__ flag) {
    __shared__ float gs[32][33];
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int a = e / 32, c = e % 32;
        gs[a][c] = (a < k && c < k) ? Gf[a * kp + c] : 0.0f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const bool on = lane < k;
    const float mu = (float)scal[1], eta = (float)scal[2];
    const float inv_s = 1.0f / s_g[0];
    unsigned long long nkept = 0;
    const int64_t nwarps = (int64_t)gridDim.x * (LF_THREADS / 32);
    for (int64_t r = (int64_t)blockIdx.x * (LF_THREADS / 32) + (threadIdx.x >> 5); r < rows; r += nwarps) {
        const float u = on ? Z[r * k + lane] : 0.0f;
        const float rc = on ? R[r * k + lane] : 0.0f;
        const float bb = __fmaf_rn(mu, u, rc);
        float x = on ? y[r * k + lane] * (beta[r] * inv_s) : 0.0f;
        // the plain path's update from u: one step of eq. gradient_descent, or
        // plain_iters steps on f from u
        float xp;
        if (plain_iters <= 1) {
            const float v = __fmaf_rn(-eta, row_times_g(u, 0.0f, gs, lane) - rc, u);
            xp = (on && v > 0.0f) ? v : 0.0f;
        } else {
            xp = u;
            for (int it = 0; it < plain_iters; ++it) {
                const float v = __fmaf_rn(-eta, row_times_g(xp, mu * xp, gs, lane) - bb, xp);
                xp = (on && v > 0.0f) ? v : 0.0f;
            }
        }
        // correction: pg_iters projected-gradient steps on f from the network's point
        for (int it = 0; it < pg_iters; ++it) {
            const float v = __fmaf_rn(-eta, row_times_g(x, mu * x, gs, lane) - bb, x);
            x = (on && v > 0.0f) ? v : 0.0f;
        }
        // objectives f(x) = 1/2 x^T (G + mu I) x - b^T x
        const float fx = warp_sum(x * (0.5f * row_times_g(x, mu * x, gs, lane) - bb));
        const float fp = warp_sum(xp * (0.5f * row_times_g(xp, mu * xp, gs, lane) - bb));
        const bool use_mlp = fx <= fp;
        nkept += use_mlp ? 1 : 0;
        float v = use_mlp ? x : xp;
        if (!(fabsf(v) <= 3.402823466e38f)) {
            *flag = 1;
            v = 0.0f;
        }
        if (on) Z[r * k + lane] = v;
    }
    if (lane == 0 && nkept) atomicAdd(kept, nkept);
}

void mlp_learned_update(MlpState &st, float *Z, const float *R, int64_t rows, const double *G64, const float *Gf,
                        int kp, const double *scal, int pg_iters, int plain_iters, unsigned long long *kept, int *flag,
                        cudaStream_t s) {
    const int k = st.k;
    // one group: G (fp32) and mu from the half-step
    k_g_to_float<<<1, 256, 0, s>>>(G64, k, scal, st.gf1, st.mu1, st.off1, rows);
    DSANLS_LAUNCH_CHECK();
    // b = R + mu Z into st.dout (rows x k) for the network input
    k_rhs_b<<<nblk(rows * k), 256, 0, s>>>(R, Z, scal, rows * k, st.dout);
    DSANLS_LAUNCH_CHECK();
    mlp_forward(st, st.gf1, st.mu1, st.off1, 1, st.dout, rows, s);
    const int64_t blocks = std::min<int64_t>(ceil_div(rows, LF_THREADS / 32), 152 * 8);
    k_learned_finish<<<(unsigned)blocks, LF_THREADS, 0, s>>>(Z, R, st.y, st.beta, st.s, Gf, kp, scal, rows, k,
                                                            pg_iters, plain_iters, kept, flag);
    DSANLS_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// harvesting training triples: exact proximal minimiser by FISTA (Beck and
// Teboulle 2009), one warp per row as above
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(LF_THREADS)
    k_harvest(const float *__restrict__ Z, const float *__restrict__ R, const float *__restrict__ Gf, int kp,
              const double *__restrict__ scal, int64_t rows, int k, int iters, float *__restrict__ b_out,
              float *__restrict__ x_out) {
    __shared__ float gs[32][33];
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int a = e / 32, c = e % 32;
        gs[a][c] = (a < k && c < k) ? Gf[a * kp + c] : 0.0f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const bool on = lane < k;
    const float mu = (float)scal[1];
    const float step = (float)(1.0 / (scal[0] * 1.0001 + scal[1]));  // 1 / (lambda_max(G) + mu)
    const int64_t nwarps = (int64_t)gridDim.x * (LF_THREADS / 32);
    for (int64_t r = (int64_t)blockIdx.x * (LF_THREADS / 32) + (threadIdx.x >> 5); r < rows; r += nwarps) {
        const float u = on ? Z[r * k + lane] : 0.0f;
        const float bb = on ? __fmaf_rn(mu, u, R[r * k + lane]) : 0.0f;
        if (on) b_out[r * k + lane] = bb;
        float x = u, yv = u, tk = 1.0f;
        for (int it = 0; it < iters; ++it) {
            const float v = yv - step * (row_times_g(yv, mu * yv, gs, lane) - bb);
            const float nx = (on && v > 0.0f) ? v : 0.0f;
            const float tn = 0.5f * (1.0f + sqrtf(1.0f + 4.0f * tk * tk));
            const float w = (tk - 1.0f) / tn;
            yv = nx + w * (nx - x);
            x = nx;
            tk = tn;
        }
        if (on) x_out[r * k + lane] = x;
    }
}

void mlp_harvest(const float *Z, const float *R, const float *Gf, int kp, const double *scal, int64_t rows, int k,
                 int iters, float *b_out, float *x_out, cudaStream_t s) {
    const int64_t blocks = std::min<int64_t>(ceil_div(rows, LF_THREADS / 32), 152 * 8);
    k_harvest<<<(unsigned)blocks, LF_THREADS, 0, s>>>(Z, R, Gf, kp, scal, rows, k, iters, b_out, x_out);
    DSANLS_LAUNCH_CHECK();
}

}  // namespace dsanls
