// Batched sketched ANLS: instance table and launch plumbing.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace dsanls {

// One dense instance; offsets are element offsets into the batch's packed
// arrays (data: M then M^T; factors: U and V; S, B, R scratch; G doubles).
struct BatchInst {
    int64_t m, n;
    int32_t k, d, dv, pad;
    uint64_t seed;
    float scale[2];  // 1/sqrt(d) and 1/sqrt(d') rounded to binary32
    int64_t offM, offU, offV, offS, offB, offR, offG;
};

struct BatchDev {
    int count = 0;
    BatchInst *inst = nullptr;
    float *data = nullptr, *factors = nullptr, *S = nullptr, *B = nullptr, *R = nullptr;
    float *P = nullptr;  // reassociated order: P_i = S_i B_i^T (K_i x k_i, at the offsets of R)
    __nv_bfloat16 *data_b = nullptr;  // bf16 form: bf16 copy of data
    int bf16 = 0;
    double *G = nullptr;
    int2 *bitems[2] = {nullptr, nullptr}, *aritems[2] = {nullptr, nullptr}, *uitems[2] = {nullptr, nullptr};
    int nb[2] = {0, 0}, nar[2] = {0, 0}, nu[2] = {0, 0};
    int2 *pitems[2] = {nullptr, nullptr};  // (instance, 64-row tile of K_i)
    int np[2] = {0, 0};
    int64_t *sketch_prefix[2] = {nullptr, nullptr};
    int *counters = nullptr;  // 12 work-queue counters (6 per side)
    int64_t *t_dev = nullptr;
    int *flag = nullptr;
    int solver = 0, power_iters = 32;
    int order = 0;  // 0: R = (X S) B^T; 1: R = X (S B^T)
    double alpha = 1.0, beta = 1.0;
};

// Launch geometry picked by the autotuner.
struct BatchLaunch {
    int persistent_blocks = 152 * 4;
    int sketch_blocks = 152 * 8;
};

void batch_build_items(const std::vector<BatchInst> &h, int side, std::vector<int2> &bitems,
                       std::vector<int2> &aritems, std::vector<int2> &uitems, std::vector<int2> &pitems,
                       std::vector<int64_t> &sketch_prefix);
// Events ev[0..5] (optional) are recorded around the five phases:
// sketch, B, AR, gram, update.
void batch_half_step(const BatchDev &g, int side, const BatchLaunch &cfg, cudaStream_t s, cudaEvent_t *ev = nullptr);
void batch_init_factors(const BatchInst *inst, int count, float *factors, cudaStream_t s);

}  // namespace dsanls
