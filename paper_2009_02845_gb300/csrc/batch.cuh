// Batched sketched ANLS: instance table and launch plumbing.
#pragma once

#include <cuda.h>
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
    // tensor-core form: padded bf16 copy of M_i and M_i^T (rows padded to multiples
    // of 8 elements) and the padded bf16 S_i^T, element offsets (multiples of 8)
    int64_t offMp, offSt, offYt;  // offYt: padded bf16 Y_i^T (k_i x pad8(K_i)) of the half-step
    int64_t offSt1;  // S_i^T of the V-half (offSt: of the U-half), so both can be drawn ahead
};

// element offset of the padded bf16 S_i^T of a half-step
__host__ __device__ inline int64_t st_off(const BatchInst &b, int side) { return side == 0 ? b.offSt : b.offSt1; }

struct BatchDev {
    int count = 0;
    BatchInst *inst = nullptr;
    float *data = nullptr, *factors = nullptr, *S = nullptr, *B = nullptr, *R = nullptr;
    float *P = nullptr;  // reassociated order: P_i = S_i B_i^T (K_i x k_i, at the offsets of R)
    __nv_bfloat16 *data_b = nullptr;  // bf16 form: bf16 copy of data
    int bf16 = 0;
    // bf16 paper order on tensor cores: padded bf16 data and S^T, (instance,
    // 128-row tile) items, prefix of the S^T sketch threads
    int tc = 0;
    __nv_bfloat16 *data_p = nullptr, *St = nullptr, *Yt = nullptr;
    int2 *tcitems[2] = {nullptr, nullptr}, *tcbitems[2] = {nullptr, nullptr};  // R items, B items (S^T row tiles)
    int2 *tcitems2[2] = {nullptr, nullptr};  // R items of two row tiles (instance, 256-row pair)
    int ntc[2] = {0, 0}, ntcb[2] = {0, 0}, ntc2[2] = {0, 0};
    // TMA tensor maps of the tensor-core products, 3 per (side, instance) at
    // (side * count + i) * 3: X_i (128-row boxes), S_i^T (64-row boxes), Y_i^T (32-row boxes)
    CUtensorMap *tmaps = nullptr;
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

// Tile of the tensor-core product of one half-step (picked per side: the sketch
// widths of the two halves differ).
struct TcTile {
    int nc = 128;    // sketch columns per chunk of the tensor-core product (64 to 256)
    int stages = 4;  // ring stages
    int rt = 1;      // 128-row tiles per work item (1 or 2)
    int mode = 1;    // 0: cp.async ring (all threads); 1: TMA ring; 2: TMA ring, epilogue off the copy path
    int ctas = 304;  // persistent CTAs
};

// Launch geometry picked by the autotuner.
struct BatchLaunch {
    int persistent_blocks = 152 * 4;
    int sketch_blocks = 152 * 8;
    TcTile tc[2];         // U-half, V-half
    int tc_b_ctas = 304;  // persistent CTAs of B = Y^T S on tensor cores
};

void batch_build_items(const std::vector<BatchInst> &h, int side, std::vector<int2> &bitems,
                       std::vector<int2> &aritems, std::vector<int2> &uitems, std::vector<int2> &pitems,
                       std::vector<int64_t> &sketch_prefix);
// Streams and events of the forked iteration: the Gram and step size of each
// half-step run on `gram` beside the right-hand side, and (tensor-core form) the
// V-half sketch S_1^T is drawn on `sketch` while the U-half runs.  The main
// path runs on a stream of higher priority than both, so the product's
// persistent CTAs are placed first and the side work fills what they leave.
struct BatchFork {
    cudaStream_t gram = nullptr, sketch = nullptr;
    cudaEvent_t b_done[2] = {nullptr, nullptr}, g_done[2] = {nullptr, nullptr}, s_done = nullptr;
    bool sketch_ahead = false;  // S_1^T was drawn on `sketch`; the V-half waits for s_done
};

// Events ev[0..5] (optional) are recorded around the five phases:
// sketch, B, AR, gram, update.  With `fork` (and no ev) the Gram runs on
// fork->gram, joined before the update.
void batch_half_step(const BatchDev &g, int side, const BatchLaunch &cfg, cudaStream_t s, cudaEvent_t *ev = nullptr,
                     const BatchFork *fork = nullptr);
void batch_init_factors(const BatchInst *inst, int count, float *factors, cudaStream_t s);
// (instance, 128-row tile) items of the tensor-core products, largest first: of
// R_i (rows of X_i), of R_i in pairs of tiles (instance, 256-row pair) and of B_i
// (rows of S_i^T, d_i of them).
void batch_build_tc_items(const std::vector<BatchInst> &h, int side, std::vector<int2> &tcitems,
                          std::vector<int2> &tcitems2, std::vector<int2> &tcbitems);
// batch_tc.cu
size_t batch_tc_smem(int nc, int stages, int rt);
// mode 0: all-thread cp.async ring; 1: TMA ring fed by one thread; 2: TMA ring
// with the chunk epilogue overlapped (warp-specialised, rt = 1)
bool batch_tc_tile_built(int nc, int stages, int rt, int mode);
size_t batch_tc_smem_mode(int nc, int stages, int rt, int mode);
void batch_prime_tc(int max_smem);
int batch_tc_ctas_per_sm(int nc, int stages, int rt, int mode);
int batch_tc_b_ctas_per_sm();
void launch_batch_ar_tc(const BatchDev &g, int side, int nc, int stages, int rt, int tma, int ctas, int *counter,
                        cudaStream_t s);
// the tensor maps of g.tmaps (host copy), from the padded buffers of g
void batch_tc_encode_maps(const std::vector<BatchInst> &h, const BatchDev &g, std::vector<CUtensorMap> &maps);
void launch_batch_sketch_t(const BatchDev &g, int side, cudaStream_t s);
// B_i = Y_i^T S_i on tensor cores (padded bf16 Y_i^T first); counter: a cleared queue counter
void launch_batch_b_tc(const BatchDev &g, int side, int tma, int ctas, int *counter, cudaStream_t s);
void launch_batch_pad_bf16(const BatchDev &g, cudaStream_t s);

}  // namespace dsanls
