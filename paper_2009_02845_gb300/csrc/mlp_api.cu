// C ABI of the learned warm start's network: creation, parameters,
// prediction and one training step (forward, backward, Adam).
#include <cuda_runtime.h>

#include <new>
#include <string>

#include "../../include/dsanls.h"
#include "common.cuh"
#include "kernels.cuh"
#include "mlp.cuh"

using namespace dsanls;

namespace {

template <typename F>
int mguard(F &&body) {
    try {
        return body();
    } catch (const CudaError &e) {
        record_handleless_error(std::string("CUDA error: ") + cudaGetErrorString(e.err) + " (" + e.where + ")");
        cudaGetLastError();
        return DSANLS_ECUDA;
    } catch (const ArgError &e) {
        record_handleless_error(e.what);
        return DSANLS_EINVAL;
    } catch (const std::bad_alloc &) {
        record_handleless_error("out of memory");
        return DSANLS_ENOMEM;
    } catch (...) {
        record_handleless_error("unexpected internal error");
        return DSANLS_ECUDA;
    }
}

int check_batch(const dsanls_mlp_ctx *m, const float *G, const float *mu, const int64_t *off, int32_t ngroups,
                const float *b, int64_t rows) {
    if (!G || !mu || !off || !b || ngroups < 1 || ngroups > m->st.max_groups || rows < 1 || rows > m->st.max_rows) {
        record_handleless_error("bad pointers, ngroups (1..max_groups) or rows (1..max_rows)");
        return DSANLS_EINVAL;
    }
    return DSANLS_OK;
}

}  // namespace

extern "C" {

int dsanls_mlp_create(int32_t k, int32_t hidden, int64_t max_rows, int32_t max_groups, uint64_t seed,
                      dsanls_mlp_t *out) {
    if (!out) return DSANLS_EINVAL;
    *out = nullptr;
    if (k < 1 || k > 32 || hidden < 1 || hidden > 256 || max_rows < 1 || max_groups < 1) {
        record_handleless_error("need 1 <= k <= 32, 1 <= hidden <= 256, max_rows >= 1, max_groups >= 1");
        return DSANLS_EINVAL;
    }
    dsanls_mlp_ctx *m = nullptr;
    try {
        m = new dsanls_mlp_ctx();
    } catch (...) {
        return DSANLS_ENOMEM;
    }
    const int rc = mguard([&]() {
        DSANLS_CUDA(cudaGetDevice(&m->device));
        DSANLS_CUDA(cudaStreamCreateWithFlags(&m->own_stream, cudaStreamNonBlocking));
        prime_kernel_attributes();
        mlp_alloc(m->st, k, hidden, max_rows, max_groups);
        mlp_init(m->st, seed, m->own_stream);
        DSANLS_CUDA(cudaStreamSynchronize(m->own_stream));
        return DSANLS_OK;
    });
    if (rc != DSANLS_OK) {
        dsanls_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return DSANLS_OK;
}

int dsanls_mlp_param_count(dsanls_mlp_t m, int64_t *count) {
    if (!m || !count) return DSANLS_EINVAL;
    *count = mlp_param_count(m->st.k, m->st.h);
    return DSANLS_OK;
}

int dsanls_mlp_get_params(dsanls_mlp_t m, float *theta) {
    if (!m || !theta) return DSANLS_EINVAL;
    return mguard([&]() {
        DSANLS_CUDA(cudaDeviceSynchronize());
        DSANLS_CUDA(cudaMemcpy(theta, m->st.theta, mlp_param_count(m->st.k, m->st.h) * sizeof(float),
                               cudaMemcpyDeviceToHost));
        return DSANLS_OK;
    });
}

int dsanls_mlp_set_params(dsanls_mlp_t m, const float *theta) {
    if (!m || !theta) return DSANLS_EINVAL;
    return mguard([&]() {
        DSANLS_CUDA(cudaDeviceSynchronize());
        DSANLS_CUDA(cudaMemcpy(m->st.theta, theta, mlp_param_count(m->st.k, m->st.h) * sizeof(float),
                               cudaMemcpyHostToDevice));
        mlp_quantise(m->st, m->own_stream);
        DSANLS_CUDA(cudaStreamSynchronize(m->own_stream));
        return DSANLS_OK;
    });
}

int dsanls_mlp_predict(dsanls_mlp_t m, const float *G, const float *mu, const int64_t *group_off, int32_t ngroups,
                       const float *b, int64_t rows, float *x_out, void *stream) {
    if (!m || !x_out) return DSANLS_EINVAL;
    if (int rc = check_batch(m, G, mu, group_off, ngroups, b, rows)) return rc;
    return mguard([&]() {
        cudaStream_t s = (cudaStream_t)stream;
        mlp_forward(m->st, G, mu, group_off, ngroups, b, rows, s);
        mlp_unscale(m->st, group_off, ngroups, rows, x_out, s);
        return DSANLS_OK;
    });
}

int dsanls_mlp_train_step(dsanls_mlp_t m, const float *G, const float *mu, const int64_t *group_off, int32_t ngroups,
                          const float *b, const float *xstar, int64_t rows, float lr, double *loss, float *grad,
                          void *stream) {
    if (!m || !xstar) return DSANLS_EINVAL;
    if (int rc = check_batch(m, G, mu, group_off, ngroups, b, rows)) return rc;
    if (!(lr >= 0.0f)) {
        record_handleless_error("lr must be >= 0");
        return DSANLS_EINVAL;
    }
    return mguard([&]() {
        cudaStream_t s = (cudaStream_t)stream;
        mlp_forward(m->st, G, mu, group_off, ngroups, b, rows, s);
        mlp_targets(m->st, group_off, ngroups, xstar, rows, s);
        mlp_backward(m->st, group_off, ngroups, m->st.dout, rows, s);
        if (grad)
            DSANLS_CUDA(cudaMemcpyAsync(grad, m->st.grad, mlp_param_count(m->st.k, m->st.h) * sizeof(float),
                                        cudaMemcpyDeviceToHost, s));
        if (loss) DSANLS_CUDA(cudaMemcpyAsync(loss, m->st.loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        if (lr > 0.0f) mlp_adam(m->st, lr, s);
        DSANLS_CUDA(cudaStreamSynchronize(s));
        return DSANLS_OK;
    });
}

void dsanls_mlp_destroy(dsanls_mlp_t m) {
    if (!m) return;
    cudaDeviceSynchronize();
    mlp_free(m->st);
    if (m->own_stream) cudaStreamDestroy(m->own_stream);
    delete m;
}

}  // extern "C"
