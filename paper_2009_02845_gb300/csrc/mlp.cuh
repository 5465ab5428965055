// Learned warm start: network state and launchers (see mlp.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dsanls {

struct MlpOffsets {
    int64_t W1g, W1b, b1, W2, b2, W3, b3, total;
};

struct MlpState {
    int k = 0, h = 0;
    int64_t max_rows = 0;
    int max_groups = 0;
    int64_t adam_t = 0;
    float *theta = nullptr;  // fp32 master parameters
    float *wq = nullptr;     // the same rounded to bf16 (used by every pass)
    float *grad = nullptr, *m = nullptr, *v = nullptr;
    float *Gn = nullptr, *s = nullptr, *zg = nullptr, *dzg = nullptr;
    float *bn = nullptr, *beta = nullptr;
    float *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr;
    float *o = nullptr, *y = nullptr, *dout = nullptr;
    double *rowloss = nullptr, *loss = nullptr;
    int64_t *all_off = nullptr;
    float *gf1 = nullptr, *mu1 = nullptr;  // single-group input of the learned update
    int64_t *off1 = nullptr;
};

int64_t mlp_param_count(int k, int h);
MlpOffsets mlp_offsets(int k, int h);
void mlp_alloc(MlpState &st, int k, int h, int64_t max_rows, int max_groups);
void mlp_free(MlpState &st);
void mlp_quantise(MlpState &st, cudaStream_t s);
void mlp_forward(MlpState &st, const float *G, const float *mu, const int64_t *off, int ngroups, const float *b,
                 int64_t rows, cudaStream_t s);
void mlp_backward(MlpState &st, const int64_t *off, int ngroups, const float *ystar, int64_t rows, cudaStream_t s);
void mlp_adam(MlpState &st, float lr, cudaStream_t s);
// Learned form of a half-step's update of Z (rows x k, k <= 32) from R, G (FP64 and
// padded fp32 Gf with row stride kp) and scal = {lambda, mu, eta}; counts kept rows.
void mlp_learned_update(MlpState &st, float *Z, const float *R, int64_t rows, const double *G64, const float *Gf,
                        int kp, const double *scal, int pg_iters, int plain_iters, unsigned long long *kept, int *flag,
                        cudaStream_t s);
// b = R + mu Z and the exact proximal minimiser x* (FISTA, `iters` steps) per row.
void mlp_harvest(const float *Z, const float *R, const float *Gf, int kp, const double *scal, int64_t rows, int k,
                 int iters, float *b_out, float *x_out, cudaStream_t s);
// theta ~ U(-sqrt(3/fan_in), sqrt(3/fan_in)) from Philox stream 0x20 keyed by seed; biases 0.
void mlp_init(MlpState &st, uint64_t seed, cudaStream_t s);
// y* = x* s_g / beta_r (targets of the normalised problem) into st.dout after mlp_forward.
void mlp_targets(MlpState &st, const int64_t *off, int ngroups, const float *xstar, int64_t rows, cudaStream_t s);
// x0 = y beta_r / s_g (the warm start in the original scale) after mlp_forward.
void mlp_unscale(MlpState &st, const int64_t *off, int ngroups, int64_t rows, float *x_out, cudaStream_t s);

}  // namespace dsanls

// The opaque handle behind dsanls_mlp_t.
struct dsanls_mlp_ctx {
    dsanls::MlpState st;
    int device = 0;
    cudaStream_t own_stream = nullptr;
};
