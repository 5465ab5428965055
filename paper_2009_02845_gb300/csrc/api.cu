// C ABI of libdsanls: handle state, buffer management and the orchestration
// of one outer iteration of sketched ANLS (Alg. 1 with the sketched
// subproblems of Section 3.2; the per-node body of Alg. 2 on one GPU).
//
// Per half-step (side 0: U against M and V; side 1: V against M^T and U):
//   sketch (Gaussian field / Feistel subsample / identity)  -> S or J
//   B = Y^T S                       (eq. def_A_B, "B^t = V^T S^t")
//   R = (X S) B^T                   (gradient term A B^T, eq. gradient_descent)
//   G = B B^T in FP64, eta_t        (eq. gradient_descent / reg_sub)
//   fused NNLS update of Z          (PGD step or Alg. 3 sweep)
// The iteration index t lives in device memory so that one captured CUDA
// graph replays every iteration unchanged.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/dsanls.h"
#include "common.cuh"
#include "kernels.cuh"
#include "mlp.cuh"
#include "tc_gemm.cuh"

using namespace dsanls;

namespace {

// Allocation-failure test switch (dsanls_debug_fail_alloc_after): when >= 0,
// the number of handle allocations that still succeed; the next one fails as
// if the device were out of memory.
std::atomic<int64_t> g_alloc_budget{-1};

template <typename T>
void dalloc(T *&p, int64_t count) {
    if (p) {
        cudaFree(p);
        p = nullptr;
    }
    if (count <= 0) return;
    for (int64_t b = g_alloc_budget.load(); b >= 0; b = g_alloc_budget.load()) {
        if (b == 0) throw std::bad_alloc();
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) break;
    }
    cudaError_t e = cudaMalloc((void **)&p, (size_t)count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        throw std::bad_alloc();
    }
}

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// Gaussian, Rademacher, count and SRHT sketches are dense matrices drawn from the field
bool dense_kind(int kind) {
    return kind == DSANLS_SKETCH_GAUSSIAN || kind == DSANLS_SKETCH_RADEMACHER || kind == DSANLS_SKETCH_COUNT ||
           kind == DSANLS_SKETCH_SRHT;
}

// generator of a dense sketch kind (DRAW_* of the field kernels)
int draw_kind(int kind) {
    switch (kind) {
        case DSANLS_SKETCH_RADEMACHER: return DRAW_RADEMACHER;
        case DSANLS_SKETCH_COUNT: return DRAW_COUNT;
        case DSANLS_SKETCH_SRHT: return DRAW_SRHT;
        default: return DRAW_GAUSS;
    }
}

// order of the Walsh-Hadamard matrix of an SRHT over K rows: the least power of two >= K
int64_t srht_pad(int64_t K) {
    int64_t p = 1;
    while (p < K) p <<= 1;
    return p;
}

int kp_bucket(int k) { return k <= 16 ? 16 : (k <= 32 ? 32 : (k <= 64 ? 64 : 128)); }

constexpr int MAX_SPLITS = 32;
constexpr int64_t WORK_ELEMS = 320ll * 128 * 128;

}  // namespace

struct dsanls_ctx {
    int device = 0;
    int64_t m = 0, n = 0;
    int k = 0, d = 0;
    int sketch = 0;
    uint64_t seed = 0;
    dsanls_options opt{};
    int64_t t_host = 0;
    cudaStream_t own_stream = nullptr;
    // the Gram and the step size depend only on B, the right-hand side R only on B
    // and the data: they run as a parallel branch (forked after B, joined before
    // the update) on this higher-priority stream
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    // data
    bool has_dense = false, has_sparse = false;
    bool sumsq_dirty = false;  // ||M||^2 of new dense data not computed yet (done when needed)
    float *M = nullptr, *MT = nullptr;
    __nv_bfloat16 *Mb = nullptr, *MTb = nullptr;
    // FP32 form on tensor cores: three-way bf16 splits of M and M^T
    __nv_bfloat16 *M3[3] = {nullptr, nullptr, nullptr}, *MT3[3] = {nullptr, nullptr, nullptr};
    int64_t nnz = 0;
    int64_t *rp = nullptr, *trp = nullptr;
    int32_t *ci = nullptr, *tci = nullptr;
    float *cv = nullptr, *tcv = nullptr;
    std::vector<int64_t> h_rp, h_trp;  // host copies of the row pointers (validation)

    // factors
    float *U = nullptr, *V = nullptr;
    // bf16-factor form (sparse data, subsampling sketch, BF16): the bf16 U16 and
    // V16 are the factors; U and V are refreshed from them when read
    __nv_bfloat16 *U16 = nullptr, *V16 = nullptr;

    // workspaces (sized by prepare())
    int64_t cfg_key[7] = {-1, -1, -1, -1, -1, -1, -1};
    float *S = nullptr;
    __nv_bfloat16 *Sb = nullptr;
    int32_t *J = nullptr;
    float *A = nullptr;
    float *W = nullptr;
    float *Wpart = nullptr;
    float *R = nullptr;
    float *Rpart = nullptr;
    __nv_bfloat16 *Ytb = nullptr;  // bf16 Y^T (k x K) for the tensor-core B = Y^T S
    uint8_t *Mq = nullptr, *MTq = nullptr, *Sq = nullptr;  // fp8 E4M3 forms (FP8 precision)
    float *qscale[2] = {nullptr, nullptr};                  // per 128-row block scales of M, M^T
    float *Bpart = nullptr;        // split-K slices of that product
    // reassociated order: P = S B^T (K x k fp32, FP32 form); bf16 S (K x d), bf16 B,
    // bf16 P^T (k x K) and the split-K partials of P^T and of R (BF16 form)
    float *P = nullptr;
    __nv_bfloat16 *Sn = nullptr, *Bb = nullptr, *Ptb = nullptr;
    float *Ppart = nullptr, *Rpart2 = nullptr;
    // fp8 reassociated order: P^T in fp32, its E4M3 codes and one scale per row of P^T
    float *Ptf = nullptr, *pscale = nullptr;
    uint8_t *Pq = nullptr;
    // FP32 form on tensor cores: split parts of S^T (paper order) or of P^T
    // (reassociated order) and the split-K partials of their products
    __nv_bfloat16 *St3[3] = {nullptr, nullptr, nullptr}, *Pt3[3] = {nullptr, nullptr, nullptr};
    float *Spart = nullptr;
    double *G64[2] = {nullptr, nullptr};
    double *scal[2] = {nullptr, nullptr};
    float *Gf = nullptr;
    double *work = nullptr;
    int64_t *t_dev = nullptr;
    int *flag = nullptr;
    double *dscal = nullptr;  // [0] ||M||^2, [1] residual^2, [2] cross, [3..] Gram of U, Gram of V
    uint32_t *bits = nullptr;  // membership bitmap of the sampled set (sparse subsampling)
    SubCsr sub[2];             // sub-CSR of X[:, J] per side (sparse data, subsampling sketch)
    dsanls_mlp_ctx *mlp = nullptr;          // learned warm start (borrowed), or none
    int pg_iters = 0;
    unsigned long long *kept = nullptr;     // rows whose learned point was kept
    float bound = 0.0f;

    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
    uint64_t graph_launches = 0;  // kernels per captured outer iteration
    std::string err;

    cudaStream_t stream() const { return opt.stream ? (cudaStream_t)opt.stream : own_stream; }
};

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

thread_local std::string g_last_error;

template <typename F>
int guarded(dsanls_ctx *h, F &&body) {
    std::string &err = h ? h->err : g_last_error;
    try {
        return body();
    } catch (const CudaError &e) {
        err = std::string("CUDA error: ") + cudaGetErrorString(e.err) + " (" + e.where + ")";
        cudaGetLastError();
        return DSANLS_ECUDA;
    } catch (const ArgError &e) {
        err = e.what;
        return DSANLS_EINVAL;
    } catch (const std::bad_alloc &) {
        err = "out of memory";
        return DSANLS_ENOMEM;
    } catch (...) {
        err = "unexpected internal error";
        return DSANLS_ECUDA;
    }
}

int fail(dsanls_ctx *h, int code, const std::string &msg) {
    if (h) h->err = msg;
    return code;
}

void check_sketch(int kind, int64_t K, int64_t dd, const char *what) {
    if (dd < 1) throw ArgError{std::string(what) + " must be >= 1"};
    if (kind == DSANLS_SKETCH_SUBSAMPLE && dd > K)
        throw ArgError{std::string(what) + ": subsampling needs sketch size <= dimension"};
    if (kind == DSANLS_SKETCH_SRHT && dd > srht_pad(K))
        throw ArgError{std::string(what) + ": the SRHT needs sketch size <= the dimension rounded up to a power of two"};
    if (kind == DSANLS_SKETCH_IDENTITY && dd != K)
        throw ArgError{std::string(what) + ": the identity sketch needs sketch size == dimension"};
    if (dd > (1 << 30)) throw ArgError{std::string(what) + " too large"};
}

void invalidate_graph(dsanls_ctx *h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_valid = false;
}

int d_v_of(const dsanls_ctx *h) { return h->opt.d_v > 0 ? h->opt.d_v : h->d; }

// BF16 with a subsampling sketch on sparse data: the factors are stored in bf16
bool bf16_factors(const dsanls_ctx *h) {
    return h->has_sparse && h->sketch == DSANLS_SKETCH_SUBSAMPLE && h->opt.precision == DSANLS_PREC_BF16;
}

// binary32 U and V from the bf16 factors (before anything reads U or V)
void factors_to_f32(dsanls_ctx *h, cudaStream_t s) {
    if (!h->U16) return;
    launch_cast_f32(h->U16, h->m * h->k, h->U, s);
    launch_cast_f32(h->V16, h->n * h->k, h->V, s);
}

// The FP32 form of a dense-sketch product runs on tensor cores from three-way
// bf16 splits when the rows of both orientations of M are 16-byte multiples
// (TMA), else on CUDA cores.
bool fp32_split(const dsanls_ctx *h) {
    return h->has_dense && h->opt.precision == DSANLS_PREC_FP32 && h->m % 8 == 0 && h->n % 8 == 0;
}

// Sum of the d largest row lengths of a CSR row pointer (the most entries a
// sampled set of d of its rows can hold).
int64_t top_sum(const std::vector<int64_t> &ptr, int64_t d) {
    std::vector<int64_t> len(ptr.size() > 0 ? ptr.size() - 1 : 0);
    for (size_t i = 0; i < len.size(); ++i) len[i] = ptr[i + 1] - ptr[i];
    d = std::min<int64_t>(d, (int64_t)len.size());
    std::nth_element(len.begin(), len.begin() + d, len.end(), std::greater<int64_t>());
    int64_t s = 0;
    for (int64_t i = 0; i < d; ++i) s += len[i];
    return s;
}

// (Re)allocate the per-configuration workspaces.
void prepare(dsanls_ctx *h) {
    const int dv = d_v_of(h);
    const int64_t key[7] = {h->sketch, h->d, dv, h->opt.precision, h->has_dense ? 1 : 0, h->has_sparse ? 1 : 0,
                            h->opt.order};
    if (std::equal(key, key + 7, h->cfg_key)) return;
    invalidate_graph(h);
    const int64_t m = h->m, n = h->n, k = h->k;
    const int64_t dmax = std::max<int64_t>(h->d, dv);
    const bool gauss = dense_kind(h->sketch);  // Gaussian or Rademacher: dense S
    const bool ident = h->sketch == DSANLS_SKETCH_IDENTITY;
    const bool fp8 = h->opt.precision == DSANLS_PREC_FP8;
    const bool bf16 = h->opt.precision == DSANLS_PREC_BF16 || fp8;  // fp8 keeps bf16 S^T for B = Y^T S
    const bool reas = gauss && h->opt.order == DSANLS_ORDER_REASSOCIATED;
    // identity sketch in bf16: R = X Y on the streaming tensor-core product
    const bool ident_tc = ident && h->opt.precision == DSANLS_PREC_BF16 && h->has_dense;
    const int64_t kmax = std::max(m, n);
    dalloc(h->S, (gauss && !bf16) ? std::max(n * h->d, m * dv) : 0);
    dalloc(h->Sb, (gauss && bf16) ? std::max(n * h->d, m * dv) : 0);
    const bool srht = h->sketch == DSANLS_SKETCH_SRHT;
    dalloc(h->J, (h->sketch == DSANLS_SKETCH_SUBSAMPLE || srht) ? dmax : 0);
    dalloc(h->A, (gauss && !bf16 && !reas) ? std::max(m * h->d, n * dv) : 0);
    dalloc(h->P, (reas && !bf16) ? kmax * k : 0);
    dalloc(h->Sn, (reas && bf16) ? std::max(n * h->d, m * dv) : 0);
    dalloc(h->Bb, (reas && bf16) ? k * dmax : 0);
    dalloc(h->Ptb, (reas && bf16) ? k * kmax : 0);
    dalloc(h->Ppart, (reas && bf16) ? std::max(tc_gemm_bf16out_part_elems(k, h->d, n),
                                               tc_gemm_bf16out_part_elems(k, dv, m)) : 0);
    dalloc(h->Rpart2, ((reas && bf16) || ident_tc)
                          ? std::max({tc_skinny_part_elems(m, n, k), tc_skinny_part_elems(n, m, k),
                                      fp8 ? tc_skinny_fp8_part_elems(m, n, k) : 0,
                                      fp8 ? tc_skinny_fp8_part_elems(n, m, k) : 0})
                          : 0);
    dalloc(h->Ptf, (reas && fp8) ? k * kmax : 0);
    dalloc(h->Pq, (reas && fp8) ? k * kmax : 0);
    dalloc(h->pscale, (reas && fp8) ? 2 * k : 0);  // scales, then the row maxima (scratch)
    const bool split = gauss && fp32_split(h);
    for (int a = 0; a < 3; ++a) {
        dalloc(h->St3[a], (split && !reas) ? std::max(n * h->d, m * dv) : 0);
        dalloc(h->Pt3[a], (split && reas) ? k * kmax : 0);
    }
    dalloc(h->Spart, split ? std::max({tc_split3_part_elems(m, n, h->d), tc_split3_part_elems(n, m, dv),
                                       tc_skinny_split3_part_elems(m, n, k), tc_skinny_split3_part_elems(n, m, k),
                                       (int64_t)1})
                           : 0);
    dalloc(h->W, k * (ident ? std::max(m, n) : dmax));
    dalloc(h->Wpart, (gauss && !bf16) ? (int64_t)MAX_SPLITS * k * dmax : 0);
    dalloc(h->Ytb, ((gauss && bf16) || ident_tc) ? k * std::max(m, n) : 0);
    dalloc(h->Bpart, (gauss && bf16) ? tc_gemm_part_elems(k, dmax) : 0);
    dalloc(h->R, std::max(m, n) * k);
    dalloc(h->Rpart, (gauss && bf16 && !reas) ? tc_rpart_elems(std::max(m, n), dmax, k) : 0);
    dalloc(h->Sq, (gauss && fp8 && !reas) ? std::max(n * h->d, m * dv) : 0);
    dalloc(h->bits, h->sketch == DSANLS_SKETCH_SUBSAMPLE ? ceil_div(std::max(m, n), 32) + 1
                    : (srht ? ceil_div(srht_pad(std::max(m, n)), 32) + 1 : 0));
    if (bf16_factors(h)) {
        if (!h->U16) {  // the factors enter the bf16 form rounded to bf16
            dalloc(h->U16, m * k);
            dalloc(h->V16, n * k);
            launch_copy_cast_bf16(h->U, m * k, h->U16, h->stream());
            launch_copy_cast_bf16(h->V, n * k, h->V16, h->stream());
        }
    } else if (h->U16) {  // leaving the bf16 form: the binary32 factors take over
        factors_to_f32(h, h->stream());
        dfree(h->U16);
        dfree(h->V16);
    }
    if (h->sketch == DSANLS_SKETCH_SUBSAMPLE && h->has_sparse) {
        // U-half: columns of M (rows of M^T), V-half: rows of M; room for the
        // longest possible sampled set of each side
        h->sub[0].reserve(m, h->d, top_sum(h->h_trp, h->d), h->stream());
        h->sub[1].reserve(n, dv, top_sum(h->h_rp, dv), h->stream());
    } else {
        h->sub[0].release();
        h->sub[1].release();
    }
    std::copy(key, key + 7, h->cfg_key);
}

// ---------------------------------------------------------------------------
// one half-step
// ---------------------------------------------------------------------------
// Optional CUDA events at the phase boundaries of a half-step (profiling).
struct PhaseEvents {
    cudaEvent_t ev[DSANLS_NPHASES + 1];
};

inline void mark(PhaseEvents *pe, int i, cudaStream_t s) {
    if (pe) DSANLS_CUDA(cudaEventRecord(pe->ev[i], s));
}

void half_step(dsanls_ctx *h, int side, cudaStream_t s, PhaseEvents *pe = nullptr, bool update = true) {
    const int64_t rows = side == 0 ? h->m : h->n;
    const int64_t K = side == 0 ? h->n : h->m;
    const int dd = side == 0 ? h->d : d_v_of(h);
    const int k = h->k;
    float *Z = side == 0 ? h->U : h->V;
    const float *Y = side == 0 ? h->V : h->U;
    // data views: X = rows x K (M or M^T), XT = K x rows
    const float *X = side == 0 ? h->M : h->MT;
    const float *XT = side == 0 ? h->MT : h->M;
    const int64_t *xp = side == 0 ? h->rp : h->trp;
    const int32_t *xc = side == 0 ? h->ci : h->tci;
    const float *xv = side == 0 ? h->cv : h->tcv;
    const bool dense = h->has_dense;
    int64_t gram_d = dd;
    const int kp = kp_bucket(k);
    bool fuse_sub = false;  // sparse subsampled data: short rows' R formed in the update
    float fuse_c2 = 0.0f;
    // after B: the Gram and the step size on the aux stream, in parallel with R
    // (profiling keeps every phase in order on one stream)
    bool forked = false;
    auto start_gram = [&]() {
        if (pe) return;
        DSANLS_CUDA(cudaEventRecord(h->ev_fork, s));
        DSANLS_CUDA(cudaStreamWaitEvent(h->aux_stream, h->ev_fork, 0));
        launch_gram(h->W, k, gram_d, h->G64[side], h->work, WORK_ELEMS, h->aux_stream);
        launch_step_size(h->G64[side], k, h->opt.power_iters, h->opt.alpha, h->opt.beta, h->t_dev, h->scal[side],
                         h->Gf, kp, h->aux_stream);
        DSANLS_CUDA(cudaEventRecord(h->ev_join, h->aux_stream));
        forked = true;
    };

    mark(pe, DSANLS_PHASE_SKETCH, s);
    if (dense_kind(h->sketch)) {
        const int rade = draw_kind(h->sketch);
        // Gaussian / Rademacher entries carry 1/sqrt(dd); count sketch entries are +-1
        const float scale = h->sketch == DSANLS_SKETCH_COUNT ? 1.0f : (float)(1.0 / std::sqrt((double)dd));
        const bool fp8 = dense && h->opt.precision == DSANLS_PREC_FP8;
        const bool tc = dense && (h->opt.precision == DSANLS_PREC_BF16 || fp8);
        const bool reas = h->opt.order == DSANLS_ORDER_REASSOCIATED;
        const __nv_bfloat16 *Xb = side == 0 ? h->Mb : h->MTb;
        // S drawn inside the GEMMs (BF16, paper order, Gaussian): no pre-pass
        const bool regen = tc && !fp8 && !reas && h->sketch == DSANLS_SKETCH_GAUSSIAN && h->opt.regen_sketch;
        // SRHT: the sampled Hadamard columns J (dd of srht_pad(K), side 0x40 | side)
        const int32_t *hcols = nullptr;
        if (h->sketch == DSANLS_SKETCH_SRHT) {
            launch_subsample(h->seed, 0x40u | (uint32_t)side, 0, h->t_dev, srht_pad(K), dd, h->J, h->bits, s);
            hcols = h->J;
        }
        // S (K x dd), N(0, 1/dd) entries of the field, stream `side`: fp32 S for the
        // CUDA-core form, bf16 S^T (K-major operand) for the tensor-core forms, and
        // for the fp8 form also fp8 S^T of the unit-variance draws; the reassociated
        // bf16 form also keeps bf16 S (d-major operand of P^T = B S^T)
        if (regen)
            ;
        else if (tc && reas)
            launch_gaussian_pair(h->seed, (uint32_t)side, h->t_dev, K, dd, scale, h->Sb, h->Sn, rade, hcols, 0, s);
        else if (fp8)
            launch_gaussian_dual(h->seed, (uint32_t)side, h->t_dev, K, dd, scale, h->Sb, h->Sq, rade, hcols, s);
        else if (tc)
            launch_gaussian_field<__nv_bfloat16>(h->seed, (uint32_t)side, 0, h->t_dev, K, dd, scale, true, h->Sb, rade,
                                                 hcols, s);
        else
            launch_gaussian_field<float>(h->seed, (uint32_t)side, 0, h->t_dev, K, dd, scale, false, h->S, rade,
                                         hcols, s);
        mark(pe, DSANLS_PHASE_B, s);
        if (regen) {
            launch_transpose_bf16(Y, K, k, h->Ytb, s);
            launch_tc_gemm_regen(h->Ytb, k, K, dd, h->seed, (uint32_t)side, h->t_dev, scale, h->Bpart, h->W, h->flag,
                                 s);
        } else if (tc) {
            // B = Y^T S (k x dd) on tensor cores from bf16 Y^T and S^T, split-K
            launch_transpose_bf16(Y, K, k, h->Ytb, s);
            launch_tc_gemm(h->Ytb, h->Sb, k, K, dd, h->Bpart, h->W, h->flag, s);
        } else {
            // B = Y^T S  (k x dd), split over K, partials summed in order
            const int64_t tiles = ceil_div(k, 128) * ceil_div(dd, 128);
            int splits = (int)std::min<int64_t>(MAX_SPLITS, std::max<int64_t>(1, (2 * 152) / std::max<int64_t>(1, tiles)));
            splits = (int)std::min<int64_t>(splits, std::max<int64_t>(1, K / 256));
            GemmArgs g{};
            g.M = k; g.N = dd; g.K = K;
            g.A = Y; g.lda = k; g.ga = nullptr; g.a_kcontig = false;
            g.B = h->S; g.ldb = dd; g.gb = nullptr; g.b_kcontig = false;
            g.C = h->Wpart; g.ldc = dd; g.alpha = 1.0f; g.splits = splits; g.c_split_stride = (int64_t)k * dd;
            launch_sgemm(g, s);
            launch_split_reduce(h->Wpart, (int64_t)k * dd, splits, k, dd, dd, h->W, dd, s);
        }
        mark(pe, DSANLS_PHASE_PRODUCT, s);
        start_gram();
        if (reas) {
            // P = S B^T (K x k), then R = X P: 2 K dd k + 2 rows K k flops
            if (fp8) {
                // P^T in fp32, then one E4M3 scale per row of P^T
                launch_copy_cast_bf16(h->W, (int64_t)k * dd, h->Bb, s);
                launch_tc_gemm(h->Bb, h->Sn, k, dd, K, h->Ppart, h->Ptf, h->flag, s);
                launch_quant_rows(h->Ptf, k, K, h->pscale, h->Pq, reinterpret_cast<unsigned int *>(h->pscale + k), s);
            } else if (tc) {
                launch_copy_cast_bf16(h->W, (int64_t)k * dd, h->Bb, s);
                launch_tc_gemm_bf16out(h->Bb, h->Sn, k, dd, K, h->Ppart, h->Ptb, h->flag, s);
            } else {
                GemmArgs g{};
                g.M = K; g.N = k; g.K = dd;
                g.A = h->S; g.lda = dd; g.a_kcontig = true;
                g.B = h->W; g.ldb = dd; g.b_kcontig = true;
                g.C = h->P; g.ldc = k; g.alpha = 1.0f; g.splits = 1;
                launch_sgemm(g, s);
            }
            mark(pe, DSANLS_PHASE_RHS, s);
            if (fp8) {
                launch_tc_skinny_fp8(side == 0 ? h->Mq : h->MTq, h->qscale[side], h->Pq, h->pscale, rows, K, k,
                                     h->Rpart2, h->R, h->flag, s);
            } else if (tc) {
                launch_tc_skinny(Xb, h->Ptb, rows, K, k, h->Rpart2, h->R, h->flag, s);
            } else if (dense && fp32_split(h)) {
                // R = X P at binary32 accuracy on tensor cores (six bf16 products of the splits)
                launch_split3_transpose(h->P, K, k, h->Pt3, s);
                launch_tc_skinny_split3(side == 0 ? h->M3 : h->MT3, h->Pt3, rows, K, k, h->Spart, h->R, h->flag, s);
            } else if (dense) {
                GemmArgs g{};
                g.M = rows; g.N = k; g.K = K;
                g.A = X; g.lda = K; g.a_kcontig = true;
                g.B = h->P; g.ldb = k; g.b_kcontig = false;
                g.C = h->R; g.ldc = k; g.alpha = 1.0f; g.splits = 1;
                launch_sgemm(g, s);
            } else {
                launch_spmm_rows(xp, xc, xv, rows, h->P, K, k, k, 1.0f, h->R, k, s);
            }
        } else if (tc) {
            // R = (X S) B^T on tcgen05, X and S in bf16, A never stored
            if (fp8) {
                launch_tc_sketch_rhs_fp8(side == 0 ? h->Mq : h->MTq, h->qscale[side], h->Sq, scale, h->W, rows, K, dd,
                                         k, h->Rpart, h->R, h->flag, s);
            } else if (regen) {
                launch_tc_sketch_rhs_regen(Xb, h->W, rows, K, dd, k, h->seed, (uint32_t)side, h->t_dev, scale, h->Rpart,
                                           h->R, h->flag, s);
            } else {
                launch_tc_sketch_rhs(Xb, h->Sb, h->W, rows, K, dd, k, h->Rpart, h->R, h->flag, s);
            }
            mark(pe, DSANLS_PHASE_RHS, s);
        } else {
            if (dense && fp32_split(h)) {
                // A = X S at binary32 accuracy on tensor cores (six bf16 products of the splits)
                launch_split3_transpose(h->S, K, dd, h->St3, s);
                launch_tc_gemm_split3(side == 0 ? h->M3 : h->MT3, h->St3, rows, K, dd, h->Spart, h->A, h->flag, s);
            } else if (dense) {
                GemmArgs g{};
                g.M = rows; g.N = dd; g.K = K;
                g.A = X; g.lda = K; g.a_kcontig = true;
                g.B = h->S; g.ldb = dd; g.b_kcontig = false;
                g.C = h->A; g.ldc = dd; g.alpha = 1.0f; g.splits = 1;
                launch_sgemm(g, s);
            } else {
                launch_spmm_rows(xp, xc, xv, rows, h->S, K, dd, dd, 1.0f, h->A, dd, s);
            }
            mark(pe, DSANLS_PHASE_RHS, s);
            GemmArgs g{};
            g.M = rows; g.N = k; g.K = dd;
            g.A = h->A; g.lda = dd; g.a_kcontig = true;
            g.B = h->W; g.ldb = dd; g.b_kcontig = true;
            g.C = h->R; g.ldc = k; g.alpha = 1.0f; g.splits = 1;
            launch_sgemm(g, s);
        }
    } else if (h->sketch == DSANLS_SKETCH_SUBSAMPLE) {
        const float c = (float)std::sqrt((double)K / (double)dd);
        const float c2 = c * c;
        // sparse data with one PGD step on tensor cores: the right-hand side of the
        // short sub-CSR rows is formed inside the update (R is neither written nor read)
        fuse_sub = !dense && update && !h->mlp && h->opt.solver == DSANLS_SOLVER_PGD && h->opt.inner_iters == 1 &&
                   update_tc_supported(k);
        fuse_c2 = c2;
        launch_subsample(h->seed, (uint32_t)side, 0, h->t_dev, K, dd, h->J, h->bits, s);
        mark(pe, DSANLS_PHASE_B, s);
        const __nv_bfloat16 *Y16 = side == 0 ? h->V16 : h->U16;
        if (h->U16)
            launch_gather_w(Y16, k, h->J, dd, c, h->W, s);
        else
            launch_gather_w(Y, k, h->J, dd, c, h->W, s);
        mark(pe, DSANLS_PHASE_PRODUCT, s);
        start_gram();
        if (dense) {
            GemmArgs g{};
            g.M = rows; g.N = k; g.K = dd;
            g.A = XT; g.lda = rows; g.ga = h->J; g.a_kcontig = false;
            g.B = Y; g.ldb = k; g.gb = h->J; g.b_kcontig = false;
            g.C = h->R; g.ldc = k; g.alpha = c2; g.splits = 1;
            mark(pe, DSANLS_PHASE_RHS, s);
            launch_sgemm(g, s);
        } else {
            // X[:, J] gathered from the rows J of the CSR of X^T, then
            // R = c^2 X[:, J] Y[J, :] row by row
            mark(pe, DSANLS_PHASE_RHS, s);
            const int64_t *ytp = side == 0 ? h->trp : h->rp;
            const int32_t *ytc = side == 0 ? h->tci : h->ci;
            const float *ytv = side == 0 ? h->tcv : h->cv;
            launch_subcsr_build(ytp, ytc, ytv, h->J, dd, h->sub[side], s);
            if (fuse_sub) {  // short rows: formed inside the row update
                if (h->U16)
                    launch_subcsr_long_rows(h->sub[side], Y16, K, k, c2, h->R, s);
                else
                    launch_subcsr_long_rows(h->sub[side], Y, K, k, c2, h->R, s);
            } else if (h->U16) {
                launch_subcsr_rows(h->sub[side], Y16, K, k, c2, h->R, s);
            } else {
                launch_subcsr_rows(h->sub[side], Y, K, k, c2, h->R, s);
            }
        }
    } else {  // identity
        mark(pe, DSANLS_PHASE_B, s);
        launch_transpose(Y, k, K, k, h->W, K, s);
        gram_d = K;
        mark(pe, DSANLS_PHASE_PRODUCT, s);
        start_gram();
        mark(pe, DSANLS_PHASE_RHS, s);
        if (dense && h->opt.precision == DSANLS_PREC_BF16) {
            // R = X Y on the streaming tensor-core product from bf16 X and bf16 Y^T
            launch_transpose_bf16(Y, K, k, h->Ytb, s);
            launch_tc_skinny(side == 0 ? h->Mb : h->MTb, h->Ytb, rows, K, k, h->Rpart2, h->R, h->flag, s);
        } else if (dense) {
            GemmArgs g{};
            g.M = rows; g.N = k; g.K = K;
            g.A = X; g.lda = K; g.a_kcontig = true;
            g.B = Y; g.ldb = k; g.b_kcontig = false;
            g.C = h->R; g.ldc = k; g.alpha = 1.0f; g.splits = 1;
            launch_sgemm(g, s);
        } else {
            launch_spmm_rows(xp, xc, xv, rows, Y, K, k, k, 1.0f, h->R, k, s);
        }
    }
    if (forked) {
        DSANLS_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
    } else {
        mark(pe, DSANLS_PHASE_GRAM, s);
        launch_gram(h->W, k, gram_d, h->G64[side], h->work, WORK_ELEMS, s);
        mark(pe, DSANLS_PHASE_STEP_SIZE, s);
        launch_step_size(h->G64[side], k, h->opt.power_iters, h->opt.alpha, h->opt.beta, h->t_dev, h->scal[side],
                         h->Gf, kp, s);
    }
    mark(pe, DSANLS_PHASE_UPDATE, s);
    if (!update) return;
    if (h->mlp)
        mlp_learned_update(h->mlp->st, Z, h->R, rows, h->G64[side], h->Gf, kp, h->scal[side], h->pg_iters,
                           h->opt.inner_iters, h->kept,
                           h->flag, s);
    else if (fuse_sub && h->U16)
        launch_update_tc_subcsr(side == 0 ? h->U16 : h->V16, h->R, h->sub[side], side == 0 ? h->V16 : h->U16, K,
                                fuse_c2, rows, k, h->Gf, kp, h->scal[side], h->bound, h->flag, s);
    else if (fuse_sub)
        launch_update_tc_subcsr(Z, h->R, h->sub[side], Y, K, fuse_c2, rows, k, h->Gf, kp, h->scal[side], h->bound,
                                h->flag, s);
    else if (h->U16)  // bf16 factors: one PGD step on tensor cores (checked at set_options)
        launch_update_tc(side == 0 ? h->U16 : h->V16, h->R, rows, k, h->Gf, kp, h->scal[side], h->bound, h->flag, s);
    else
        launch_update(h->opt.solver, Z, h->R, rows, k, h->Gf, kp, h->scal[side], h->bound, h->opt.inner_iters, h->flag,
                      s);
    mark(pe, DSANLS_NPHASES, s);
}

void outer_iteration(dsanls_ctx *h, cudaStream_t s) {
    half_step(h, 0, s);
    half_step(h, 1, s);
    launch_increment_t(h->t_dev, 1, s);
}

int check_ready(dsanls_ctx *h) {
    if (!h->has_dense && !h->has_sparse) return fail(h, DSANLS_ESTATE, "no data: call dsanls_set_dense or dsanls_set_csr first");
    return DSANLS_OK;
}

int pending_status(dsanls_ctx *h) {
    DSANLS_CUDA(cudaStreamSynchronize(h->stream()));
    int flag = 0;
    DSANLS_CUDA(cudaMemcpy(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        DSANLS_CUDA(cudaMemset(h->flag, 0, sizeof(int)));
        if (flag & 2) return fail(h, DSANLS_ETIMEOUT, "a bounded device wait gave up (tensor-core pipeline)");
        return fail(h, DSANLS_ENUMERIC, "an update produced NaN or Inf");
    }
    return DSANLS_OK;
}

// bf16 (BF16 form) or fp8 with per-128-row-block scales (FP8 form) copies of M and M^T.
void make_reduced_copies(dsanls_ctx *h) {
    if (!h->has_dense) return;
    cudaStream_t s = h->stream();
    if (h->opt.precision == DSANLS_PREC_BF16 && !h->Mb) {
        dalloc(h->Mb, h->m * h->n);
        dalloc(h->MTb, h->m * h->n);
        launch_copy_cast_bf16(h->M, h->m * h->n, h->Mb, s);
        launch_copy_cast_bf16(h->MT, h->m * h->n, h->MTb, s);
    }
    if (fp32_split(h) && !h->M3[0]) {
        for (int a = 0; a < 3; ++a) {
            dalloc(h->M3[a], h->m * h->n);
            dalloc(h->MT3[a], h->m * h->n);
        }
        launch_split3(h->M, h->m * h->n, h->M3, s);
        launch_split3(h->MT, h->m * h->n, h->MT3, s);
    }
    if (h->opt.precision == DSANLS_PREC_FP8 && !h->Mq) {
        dalloc(h->Mq, h->m * h->n);
        dalloc(h->MTq, h->m * h->n);
        dalloc(h->qscale[0], ceil_div(h->m, 128));
        dalloc(h->qscale[1], ceil_div(h->n, 128));
        launch_quant_rowblocks(h->M, h->m, h->n, h->qscale[0], h->Mq, s);
        launch_quant_rowblocks(h->MT, h->n, h->m, h->qscale[1], h->MTq, s);
    }
}

void copy_in(void *dst, const void *src, size_t bytes, int on_device, cudaStream_t s) {
    DSANLS_CUDA(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}

// ||M||^2 into dscal[0] when the dense data changed since it was last computed
void ensure_sumsq(dsanls_ctx *h) {
    if (!h->sumsq_dirty || !h->has_dense) return;
    launch_sumsq(h->M, h->m * h->n, h->work, WORK_ELEMS, h->dscal + 0, h->stream());
    h->sumsq_dirty = false;
}

void set_bound(dsanls_ctx *h) {
    h->bound = 0.0f;
    if (h->opt.bound_clamp && (h->has_dense || h->has_sparse)) {
        ensure_sumsq(h);
        double mm = 0.0;
        DSANLS_CUDA(cudaStreamSynchronize(h->stream()));
        DSANLS_CUDA(cudaMemcpy(&mm, h->dscal + 0, sizeof(double), cudaMemcpyDeviceToHost));
        h->bound = (float)std::sqrt(2.0 * std::sqrt(mm));
    }
}

}  // namespace

namespace dsanls {
void record_handleless_error(const std::string &msg) { g_last_error = msg; }

static std::atomic<uint64_t> g_launches{0};
uint64_t launch_count() { return g_launches.load(); }
void add_launches(uint64_t n) { g_launches.fetch_add(n); }

// cudaFuncSetAttribute applies to the current device only, so the kernels'
// shared-memory limits are raised once per device, with that device current;
// the mutex orders callers on different host threads.
void prime_kernel_attributes() {
    constexpr int kMaxPrimedDevices = 64;
    static std::mutex mu;
    static bool done[kMaxPrimedDevices] = {};
    int dev = 0, max_smem = 0;
    DSANLS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxPrimedDevices) throw ArgError{"device ordinal out of range"};
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return;
    DSANLS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    prime_rng_attributes(max_smem);
    prime_solver_attributes(max_smem);
    prime_tc_attributes(max_smem);
    batch_prime_tc(max_smem);
    done[dev] = true;
}
}  // namespace dsanls

// ---------------------------------------------------------------------------
// exported API
// ---------------------------------------------------------------------------
extern "C" {

int dsanls_default_options(dsanls_options *opt) {
    if (!opt) return DSANLS_EINVAL;
    std::memset(opt, 0, sizeof(*opt));
    opt->solver = DSANLS_SOLVER_PGD;
    opt->precision = DSANLS_PREC_FP32;
    opt->d_v = 0;
    opt->power_iters = 32;
    opt->alpha = 1.0;
    opt->beta = 1.0;
    opt->t = 0;
    opt->bound_clamp = 0;
    opt->use_graph = 0;
    opt->order = DSANLS_ORDER_PAPER;
    opt->inner_iters = 1;
    opt->stream = nullptr;
    opt->regen_sketch = 0;
    return DSANLS_OK;
}

int dsanls_create(int64_t m, int64_t n, int32_t k, int32_t d, int32_t sketch_kind, uint64_t seed, dsanls_t *out) {
    if (!out) return DSANLS_EINVAL;
    *out = nullptr;
    if (m < 1 || n < 1 || k < 1 || k > 128 || d < 1) return DSANLS_EINVAL;
    if (m > (1ll << 31) - 1 || n > (1ll << 31) - 1) return DSANLS_EINVAL;
    if (sketch_kind < DSANLS_SKETCH_GAUSSIAN || sketch_kind > DSANLS_SKETCH_SRHT) return DSANLS_EINVAL;
    if (sketch_kind == DSANLS_SKETCH_SUBSAMPLE && d > n) return DSANLS_EINVAL;
    if (sketch_kind == DSANLS_SKETCH_SRHT && d > srht_pad(n)) return DSANLS_EINVAL;
    if (sketch_kind == DSANLS_SKETCH_IDENTITY && d != n) return DSANLS_EINVAL;
    dsanls_ctx *h = nullptr;
    try {
        h = new dsanls_ctx();
    } catch (...) {
        return DSANLS_ENOMEM;
    }
    h->m = m; h->n = n; h->k = k; h->d = d; h->sketch = sketch_kind; h->seed = seed;
    dsanls_default_options(&h->opt);
    if (sketch_kind == DSANLS_SKETCH_IDENTITY) h->opt.d_v = (int32_t)m;
    const int rc = guarded(h, [&]() {
        DSANLS_CUDA(cudaGetDevice(&h->device));
        DSANLS_CUDA(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
        int prio_least = 0, prio_greatest = 0;
        DSANLS_CUDA(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
        DSANLS_CUDA(cudaStreamCreateWithPriority(&h->aux_stream, cudaStreamNonBlocking, prio_greatest));
        DSANLS_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        DSANLS_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        prime_kernel_attributes();
        cudaStream_t s = h->stream();
        dalloc(h->U, m * k);
        dalloc(h->V, n * k);
        for (int side = 0; side < 2; ++side) {
            dalloc(h->G64[side], (int64_t)k * k);
            dalloc(h->scal[side], 4);
            DSANLS_CUDA(cudaMemsetAsync(h->G64[side], 0, sizeof(double) * k * k, s));
            DSANLS_CUDA(cudaMemsetAsync(h->scal[side], 0, sizeof(double) * 4, s));
        }
        dalloc(h->Gf, 128 * 128);
        dalloc(h->work, WORK_ELEMS);
        dalloc(h->t_dev, 1);
        dalloc(h->flag, 1);
        dalloc(h->dscal, 3 + 2 * 128 * 128);
        DSANLS_CUDA(cudaMemsetAsync(h->t_dev, 0, sizeof(int64_t), s));
        DSANLS_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
        DSANLS_CUDA(cudaMemsetAsync(h->dscal, 0, sizeof(double) * 3, s));
        launch_uniform_field(seed, DSANLS_STREAM_INIT_U, 0, m, k, h->U, s);
        launch_uniform_field(seed, DSANLS_STREAM_INIT_V, 0, n, k, h->V, s);
        DSANLS_CUDA(cudaStreamSynchronize(s));
        return DSANLS_OK;
    });
    if (rc != DSANLS_OK) {
        g_last_error = h->err;
        dsanls_destroy(h);
        return rc;
    }
    *out = h;
    return DSANLS_OK;
}

int dsanls_get_options(dsanls_t h, dsanls_options *opt) {
    if (!h || !opt) return DSANLS_EINVAL;
    *opt = h->opt;
    opt->t = h->t_host;
    return DSANLS_OK;
}

int dsanls_set_options(dsanls_t h, const dsanls_options *opt) {
    if (!h) return DSANLS_EINVAL;
    if (!opt) return fail(h, DSANLS_EINVAL, "options pointer is NULL");
    DeviceGuard dg(h->device);
    return guarded(h, [&]() {
        if (opt->solver != DSANLS_SOLVER_PGD && opt->solver != DSANLS_SOLVER_RCD) throw ArgError{"unknown solver"};
        if (opt->precision < DSANLS_PREC_FP32 || opt->precision > DSANLS_PREC_FP8) throw ArgError{"unknown precision"};
        if (opt->precision == DSANLS_PREC_FP8 &&
            (h->has_sparse || !dense_kind(h->sketch) || h->m % 16 || h->n % 16 ||
             h->d % 8 || (opt->d_v > 0 ? opt->d_v : h->d) % 8))
            throw ArgError{"FP8 precision needs dense data, a Gaussian sketch, m and n multiples of 16, d and d_v of 8"};
        if (opt->precision == DSANLS_PREC_BF16 && h->sketch == DSANLS_SKETCH_SUBSAMPLE) {
            // the bf16-factor form of sparse data
            if (h->has_dense) throw ArgError{"BF16 with a subsampling sketch is the bf16-factor form of sparse data"};
            if (opt->solver != DSANLS_SOLVER_PGD || opt->inner_iters != 1 || !update_tc_supported(h->k) ||
                h->mlp || opt->bound_clamp)
                throw ArgError{"bf16 factors need one PGD step per half, 32 < k <= 128, no network and no bound"};
        } else if (opt->precision == DSANLS_PREC_BF16 && (h->has_sparse || !tc_supported(h->k))) {
            throw ArgError{"BF16 precision needs dense data and a Gaussian or identity sketch, or sparse data and a "
                           "subsampling sketch (bf16 factors)"};
        }
        if (opt->precision == DSANLS_PREC_BF16 && h->sketch != DSANLS_SKETCH_SUBSAMPLE) {
            const int dv = opt->d_v > 0 ? opt->d_v : h->d;
            if (h->m % 8 || h->n % 8 || h->d % 8 || dv % 8)
                throw ArgError{"BF16 precision needs m, n, d and d_v multiples of 8 (16-byte TMA rows)"};
        }
        if (opt->order != DSANLS_ORDER_PAPER && opt->order != DSANLS_ORDER_REASSOCIATED) throw ArgError{"unknown order"};
        if (opt->order == DSANLS_ORDER_REASSOCIATED && !dense_kind(h->sketch))
            throw ArgError{"the reassociated order needs a dense sketch (Gaussian, Rademacher, count or SRHT)"};
        if (opt->power_iters < 0 || opt->power_iters > 10000) throw ArgError{"power_iters out of range"};
        if (opt->inner_iters < 1 || opt->inner_iters > 256) throw ArgError{"inner_iters must be in 1..256"};
        if (opt->regen_sketch != 0 && opt->regen_sketch != 1) throw ArgError{"regen_sketch must be 0 or 1"};
        if (opt->inner_iters > 1 && opt->solver != DSANLS_SOLVER_PGD)
            throw ArgError{"inner_iters > 1 needs the PGD solver"};
        if (!(opt->alpha >= 0.0) || !(opt->beta >= 0.0) || !std::isfinite(opt->alpha) || !std::isfinite(opt->beta))
            throw ArgError{"alpha and beta must be finite and >= 0"};
        if (opt->t < 0) throw ArgError{"t must be >= 0"};
        const int dv = opt->d_v > 0 ? opt->d_v : h->d;
        check_sketch(h->sketch, h->m, dv, "d_v");
        const bool cfg_change = (opt->precision != h->opt.precision) || (dv != d_v_of(h)) ||
                                (opt->stream != h->opt.stream) || (opt->solver != h->opt.solver) ||
                                (opt->power_iters != h->opt.power_iters) || (opt->alpha != h->opt.alpha) ||
                                (opt->beta != h->opt.beta) || (opt->bound_clamp != h->opt.bound_clamp) ||
                                (opt->use_graph != h->opt.use_graph) || (opt->order != h->opt.order) ||
                                (opt->inner_iters != h->opt.inner_iters) || (opt->regen_sketch != h->opt.regen_sketch);
        // finish work queued on the old stream before switching
        DSANLS_CUDA(cudaStreamSynchronize(h->stream()));
        h->opt = *opt;
        if (cfg_change) invalidate_graph(h);
        make_reduced_copies(h);
        if (opt->t != h->t_host) {
            h->t_host = opt->t;
            DSANLS_CUDA(cudaMemcpyAsync(h->t_dev, &h->t_host, sizeof(int64_t), cudaMemcpyHostToDevice, h->stream()));
        }
        set_bound(h);
        DSANLS_CUDA(cudaStreamSynchronize(h->stream()));
        return DSANLS_OK;
    });
}

int dsanls_set_dense(dsanls_t h, const float *M, int64_t ld, int32_t on_device) {
    if (!h) return DSANLS_EINVAL;
    if (!M || ld < h->n) return fail(h, DSANLS_EINVAL, "M is NULL or ld < n");
    if (h->opt.precision == DSANLS_PREC_BF16 && h->sketch == DSANLS_SKETCH_SUBSAMPLE)
        return fail(h, DSANLS_EINVAL, "BF16 with a subsampling sketch is the bf16-factor form of sparse data");
    DeviceGuard dg(h->device);
    return guarded(h, [&]() {
        cudaStream_t s = h->stream();
        if (h->has_sparse) {
            dfree(h->rp); dfree(h->ci); dfree(h->cv); dfree(h->trp); dfree(h->tci); dfree(h->tcv);
            h->has_sparse = false;
        }
        // new values in the buffers of earlier dense data keep the captured graph valid
        const bool refresh = h->has_dense && h->M && h->MT;
        if (!h->M) dalloc(h->M, h->m * h->n);
        if (!h->MT) dalloc(h->MT, h->m * h->n);
        const bool bf16 = h->opt.precision == DSANLS_PREC_BF16, fp8 = h->opt.precision == DSANLS_PREC_FP8;
        const bool cast_b = refresh && bf16 && h->Mb;
        if (on_device) {
            DSANLS_CUDA(cudaMemcpy2DAsync(h->M, h->n * sizeof(float), M, ld * sizeof(float), h->n * sizeof(float),
                                          h->m, cudaMemcpyDeviceToDevice, s));
            launch_transpose(h->M, h->n, h->m, h->n, h->MT, h->m, s);
            if (cast_b) launch_copy_cast_bf16(h->M, h->m * h->n, h->Mb, s);
        } else {
            // host data: copied in chunks of rows (about 256 MB); the transpose (and bf16
            // copy) of a chunk runs on the second stream while the next chunk is copied
            const int64_t ch = std::max<int64_t>(1024, ((int64_t)256 << 20) / (h->n * (int64_t)sizeof(float)));
            for (int64_t r0 = 0; r0 < h->m; r0 += ch) {
                const int64_t rc = std::min(ch, h->m - r0);
                DSANLS_CUDA(cudaMemcpy2DAsync(h->M + r0 * h->n, h->n * sizeof(float), M + r0 * ld, ld * sizeof(float),
                                              h->n * sizeof(float), rc, cudaMemcpyHostToDevice, s));
                DSANLS_CUDA(cudaEventRecord(h->ev_fork, s));
                DSANLS_CUDA(cudaStreamWaitEvent(h->aux_stream, h->ev_fork, 0));
                launch_transpose(h->M + r0 * h->n, h->n, rc, h->n, h->MT + r0, h->m, h->aux_stream);
                if (cast_b) launch_copy_cast_bf16(h->M + r0 * h->n, rc * h->n, h->Mb + r0 * h->n, h->aux_stream);
            }
            DSANLS_CUDA(cudaEventRecord(h->ev_join, h->aux_stream));
            DSANLS_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
        }
        h->sumsq_dirty = true;  // ||M||^2 is computed when a relative error or the bound needs it
        h->has_dense = true;
        if (cast_b) {
            launch_copy_cast_bf16(h->MT, h->m * h->n, h->MTb, s);
        } else {
            dfree(h->Mb);
            dfree(h->MTb);
        }
        const bool split = fp32_split(h);
        if (refresh && split && h->M3[0]) {
            launch_split3(h->M, h->m * h->n, h->M3, s);
            launch_split3(h->MT, h->m * h->n, h->MT3, s);
        } else {
            for (int a = 0; a < 3; ++a) {
                dfree(h->M3[a]);
                dfree(h->MT3[a]);
            }
        }
        if (refresh && fp8 && h->Mq) {
            launch_quant_rowblocks(h->M, h->m, h->n, h->qscale[0], h->Mq, s);
            launch_quant_rowblocks(h->MT, h->n, h->m, h->qscale[1], h->MTq, s);
        } else {
            dfree(h->Mq);
            dfree(h->MTq);
        }
        const bool had_copies = (bf16 && h->Mb) || (fp8 && h->Mq) || (!bf16 && !fp8 && (!split || h->M3[0]));
        make_reduced_copies(h);
        // a graph holds the buffer pointers and, with the clamp, the bound by value
        if (!refresh || !had_copies || h->opt.bound_clamp) {
            invalidate_graph(h);
            std::fill(h->cfg_key, h->cfg_key + 6, -1);
        }
        set_bound(h);
        DSANLS_CUDA(cudaStreamSynchronize(s));
        return DSANLS_OK;
    });
}

int dsanls_set_csr(dsanls_t h, const int64_t *rowptr, const int32_t *col, const float *val, int64_t nnz,
                   const int64_t *t_rowptr, const int32_t *t_col, const float *t_val, int32_t on_device) {
    if (!h) return DSANLS_EINVAL;
    if (!rowptr || nnz < 0 || (nnz > 0 && (!col || !val))) return fail(h, DSANLS_EINVAL, "bad CSR pointers");
    if (t_rowptr && (nnz > 0 && (!t_col || !t_val))) return fail(h, DSANLS_EINVAL, "bad transposed CSR pointers");
    if (!t_rowptr && on_device) return fail(h, DSANLS_EINVAL, "device CSR input needs the transposed CSR too");
    if (h->opt.precision == DSANLS_PREC_BF16 && h->sketch != DSANLS_SKETCH_SUBSAMPLE)
        return fail(h, DSANLS_EINVAL, "BF16 precision needs dense data (or a subsampling sketch: bf16 factors)");
    DeviceGuard dg(h->device);
    return guarded(h, [&]() {
        cudaStream_t s = h->stream();
        const int64_t m = h->m, n = h->n;
        // host copies of the row pointers (validation and capacity planning)
        h->h_rp.assign(m + 1, 0);
        h->h_trp.assign(n + 1, 0);
        std::vector<int32_t> hcol, htcol;
        std::vector<float> hval, htval;
        if (on_device) {
            DSANLS_CUDA(cudaMemcpy(h->h_rp.data(), rowptr, (m + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
            DSANLS_CUDA(cudaMemcpy(h->h_trp.data(), t_rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
        } else {
            std::memcpy(h->h_rp.data(), rowptr, (m + 1) * sizeof(int64_t));
        }
        if (h->h_rp[0] != 0 || h->h_rp[m] != nnz) throw ArgError{"rowptr[0] must be 0 and rowptr[m] == nnz"};
        for (int64_t i = 0; i < m; ++i)
            if (h->h_rp[i + 1] < h->h_rp[i]) throw ArgError{"rowptr must be nondecreasing"};
        const int32_t *tc_src = t_col;
        const float *tv_src = t_val;
        if (!on_device) {
            for (int64_t e = 0; e < nnz; ++e)
                if (col[e] < 0 || col[e] >= n) throw ArgError{"column index out of range"};
            if (t_rowptr) {
                std::memcpy(h->h_trp.data(), t_rowptr, (n + 1) * sizeof(int64_t));
                if (h->h_trp[0] != 0 || h->h_trp[n] != nnz) throw ArgError{"t_rowptr[0] must be 0 and t_rowptr[n] == nnz"};
                for (int64_t j = 0; j < n; ++j)
                    if (h->h_trp[j + 1] < h->h_trp[j]) throw ArgError{"t_rowptr must be nondecreasing"};
                for (int64_t e = 0; e < nnz; ++e)
                    if (t_col[e] < 0 || t_col[e] >= m) throw ArgError{"transposed column index out of range"};
            } else {
                // counting-sort transpose; rows come out in increasing order within each column
                for (int64_t e = 0; e < nnz; ++e) h->h_trp[col[e] + 1]++;
                for (int64_t j = 0; j < n; ++j) h->h_trp[j + 1] += h->h_trp[j];
                htcol.resize(nnz);
                htval.resize(nnz);
                std::vector<int64_t> cur(h->h_trp.begin(), h->h_trp.end() - 1);
                for (int64_t i = 0; i < m; ++i)
                    for (int64_t e = h->h_rp[i]; e < h->h_rp[i + 1]; ++e) {
                        const int64_t pos = cur[col[e]]++;
                        htcol[pos] = (int32_t)i;
                        htval[pos] = val[e];
                    }
                tc_src = htcol.data();
                tv_src = htval.data();
            }
        } else if (h->h_trp[0] != 0 || h->h_trp[n] != nnz) {
            throw ArgError{"t_rowptr[0] must be 0 and t_rowptr[n] == nnz"};
        }
        if (h->has_dense) {
            dfree(h->M); dfree(h->MT); dfree(h->Mb); dfree(h->MTb); dfree(h->Mq); dfree(h->MTq);
            for (int a = 0; a < 3; ++a) {
                dfree(h->M3[a]);
                dfree(h->MT3[a]);
            }
            h->has_dense = false;
        }
        dalloc(h->rp, m + 1);
        dalloc(h->trp, n + 1);
        dalloc(h->ci, std::max<int64_t>(nnz, 1));
        dalloc(h->cv, std::max<int64_t>(nnz, 1));
        dalloc(h->tci, std::max<int64_t>(nnz, 1));
        dalloc(h->tcv, std::max<int64_t>(nnz, 1));
        DSANLS_CUDA(cudaMemcpyAsync(h->rp, h->h_rp.data(), (m + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        DSANLS_CUDA(cudaMemcpyAsync(h->trp, h->h_trp.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        if (nnz > 0) {
            copy_in(h->ci, col, nnz * sizeof(int32_t), on_device, s);
            copy_in(h->cv, val, nnz * sizeof(float), on_device, s);
            copy_in(h->tci, tc_src, nnz * sizeof(int32_t), on_device, s);
            copy_in(h->tcv, tv_src, nnz * sizeof(float), on_device, s);
        }
        h->nnz = nnz;
        launch_sumsq(h->cv, nnz, h->work, WORK_ELEMS, h->dscal + 0, s);
        h->has_sparse = true;
        invalidate_graph(h);
        std::fill(h->cfg_key, h->cfg_key + 6, -1);
        set_bound(h);
        DSANLS_CUDA(cudaStreamSynchronize(s));  // host staging buffers go out of scope
        return DSANLS_OK;
    });
}

int dsanls_set_factors(dsanls_t h, const float *U, const float *V, int32_t on_device) {
    if (!h) return DSANLS_EINVAL;
    DeviceGuard dg(h->device);
    return guarded(h, [&]() {
        cudaStream_t s = h->stream();
        if (h->U16 && (!U || !V)) factors_to_f32(h, s);  // the factor not given keeps its bf16 value
        if (U) copy_in(h->U, U, (size_t)h->m * h->k * sizeof(float), on_device, s);
        if (V) copy_in(h->V, V, (size_t)h->n * h->k * sizeof(float), on_device, s);
        if (h->U16) {  // the bf16 factors take the new values, rounded
            launch_copy_cast_bf16(h->U, h->m * h->k, h->U16, s);
            launch_copy_cast_bf16(h->V, h->n * h->k, h->V16, s);
        }
        DSANLS_CUDA(cudaStreamSynchronize(s));
        return DSANLS_OK;
    });
}

int dsanls_step(dsanls_t h, int32_t outer_iters) {
    if (!h) return DSANLS_EINVAL;
    if (outer_iters < 0) return fail(h, DSANLS_EINVAL, "outer_iters < 0");
    if (int rc = check_ready(h)) return rc;
    DeviceGuard dg(h->device);
    return guarded(h, [&]() {
        cudaStream_t s = h->stream();
        prepare(h);
        if (h->opt.use_graph) {
            if (!h->graph_valid) {
                cudaGraph_t g = nullptr;
                const uint64_t before = launch_count();
                DSANLS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                try {
                    outer_iteration(h, s);
                } catch (...) {
                    cudaGraph_t dummy = nullptr;
                    cudaStreamEndCapture(s, &dummy);
                    if (dummy) cudaGraphDestroy(dummy);
                    throw;
                }
                DSANLS_CUDA(cudaStreamEndCapture(s, &g));
                h->graph_launches = launch_count() - before;
                add_launches(0 - h->graph_launches);  // captured, not run
                cudaError_t e = cudaGraphInstantiate(&h->graph, g, 0);
                cudaGraphDestroy(g);
                DSANLS_CUDA(e);
                h->graph_valid = true;
            }
            for (int it = 0; it < outer_iters; ++it) DSANLS_CUDA(cudaGraphLaunch(h->graph, s));
            add_launches(h->graph_launches * (uint64_t)outer_iters);
        } else {
            for (int it = 0; it < outer_iters; ++it) outer_iteration(h, s);
        }
        h->t_host += outer_iters;
        return DSANLS_OK;
    });
}

int dsanls_half_step(dsanls_t h, int32_t side) {
    if (!h) return DSANLS_EINVAL;
    if (side != 0 && side != 1) return fail(h, DSANLS_EINVAL, "side must be 0 or 1");
    if (int rc = check_ready(h)) return rc;
    DeviceGuard dg(h->device);
    return guarded(h, [&]() {
        prepare(h);
        half_step(h, side, h->stream());
        return DSANLS_OK;
    });
}

int dsanls_rel_error(dsanls_t h, double *out) {
    if (!h) return DSANLS_EINVAL;
    if (!out) return fail(h, DSANLS_EINVAL, "out is NULL");
    if (int rc = check_ready(h)) return rc;
    DeviceGuard dg(h->device);
    return guarded(h, [&]() {
        cudaStream_t s = h->stream();
        factors_to_f32(h, s);
        if (h->has_dense) {
            ensure_sumsq(h);
            launch_dense_residual(h->M, h->n, h->U, h->V, h->m, h->n, h->k, h->work, WORK_ELEMS, h->dscal + 1, s);
        } else {
            double *GU = h->dscal + 3, *GV = h->dscal + 3 + 128 * 128;
            launch_sparse_cross(h->rp, h->ci, h->cv, h->m, h->U, h->V, h->k, h->work, WORK_ELEMS, h->dscal + 2, s);
            launch_factor_gram(h->U, h->m, h->k, h->work, WORK_ELEMS, GU, s);
            launch_factor_gram(h->V, h->n, h->k, h->work, WORK_ELEMS, GV, s);
            launch_sparse_combine(h->dscal + 0, h->dscal + 2, GU, GV, h->k, h->dscal + 1, s);
        }
        if (int rc = pending_status(h)) return rc;
        double v[2];
        DSANLS_CUDA(cudaMemcpy(v, h->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost));
        *out = v[0] > 0.0 ? std::sqrt(std::max(v[1], 0.0) / v[0]) : 0.0;
        return DSANLS_OK;
    });
}

int dsanls_get_factors(dsanls_t h, float *U, float *V, int32_t on_device) {
    if (!h) return DSANLS_EINVAL;
    DeviceGuard dg(h->device);
    return guarded(h, [&]() {
        factors_to_f32(h, h->stream());
        if (int rc = pending_status(h)) return rc;
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (U) DSANLS_CUDA(cudaMemcpyAsync(U, h->U, (size_t)h->m * h->k * sizeof(float), kind, h->stream()));
        if (V) DSANLS_CUDA(cudaMemcpyAsync(V, h->V, (size_t)h->n * h->k * sizeof(float), kind, h->stream()));
        DSANLS_CUDA(cudaStreamSynchronize(h->stream()));
        return DSANLS_OK;
    });
}

int dsanls_get_gram(dsanls_t h, int32_t side, double *G, double *eta) {
    if (!h) return DSANLS_EINVAL;
    if (side != 0 && side != 1) return fail(h, DSANLS_EINVAL, "side must be 0 or 1");
    DeviceGuard dg(h->device);
    return guarded(h, [&]() {
        if (int rc = pending_status(h)) return rc;
        if (G) DSANLS_CUDA(cudaMemcpy(G, h->G64[side], (size_t)h->k * h->k * sizeof(double), cudaMemcpyDeviceToHost));
        if (eta) DSANLS_CUDA(cudaMemcpy(eta, h->scal[side] + 2, sizeof(double), cudaMemcpyDeviceToHost));
        return DSANLS_OK;
    });
}

int dsanls_sync(dsanls_t h) {
    if (!h) return DSANLS_EINVAL;
    DeviceGuard dg(h->device);
    return guarded(h, [&]() { return pending_status(h); });
}

int dsanls_profile_half_step(dsanls_t h, int32_t side, int32_t reps, double *ms) {
    if (!h) return DSANLS_EINVAL;
    if ((side != 0 && side != 1) || reps < 1 || !ms) return fail(h, DSANLS_EINVAL, "bad side, reps or output");
    if (int rc = check_ready(h)) return rc;
    DeviceGuard dg(h->device);
    PhaseEvents pe;
    int created = 0;
    const int rc = guarded(h, [&]() {
        prepare(h);
        for (; created <= DSANLS_NPHASES; ++created) DSANLS_CUDA(cudaEventCreate(&pe.ev[created]));
        cudaStream_t s = h->stream();
        for (int i = 0; i < DSANLS_NPHASES; ++i) ms[i] = 0.0;
        for (int r = 0; r < reps; ++r) {
            half_step(h, side, s, &pe);
            DSANLS_CUDA(cudaEventSynchronize(pe.ev[DSANLS_NPHASES]));
            for (int i = 0; i < DSANLS_NPHASES; ++i) {
                float t = 0.0f;
                DSANLS_CUDA(cudaEventElapsedTime(&t, pe.ev[i], pe.ev[i + 1]));
                ms[i] += t / reps;
            }
        }
        return pending_status(h);
    });
    for (int i = 0; i < created; ++i) cudaEventDestroy(pe.ev[i]);
    return rc;
}

int dsanls_set_mlp(dsanls_t h, dsanls_mlp_t m, int32_t pg_iters) {
    if (!h) return DSANLS_EINVAL;
    if (pg_iters < 0 || pg_iters > 1000) return fail(h, DSANLS_EINVAL, "pg_iters must be in [0, 1000]");
    if (m && (m->st.k != h->k || h->k > 32 || m->st.max_rows < std::max(h->m, h->n)))
        return fail(h, DSANLS_EINVAL, "the network's k must equal the handle's (<= 32) and max_rows >= max(m, n)");
    if (m && h->opt.bound_clamp) return fail(h, DSANLS_EINVAL, "the learned form has no bound clamp");
    if (m && h->opt.precision == DSANLS_PREC_BF16 && h->sketch == DSANLS_SKETCH_SUBSAMPLE)
        return fail(h, DSANLS_EINVAL, "the learned form has no bf16 factors");
    DeviceGuard dg(h->device);
    return guarded(h, [&]() {
        DSANLS_CUDA(cudaStreamSynchronize(h->stream()));
        if (!h->kept) {
            dalloc(h->kept, 1);
            DSANLS_CUDA(cudaMemset(h->kept, 0, sizeof(unsigned long long)));
        }
        h->mlp = m;
        h->pg_iters = pg_iters;
        invalidate_graph(h);
        return DSANLS_OK;
    });
}

int dsanls_mlp_kept(dsanls_t h, int64_t *kept) {
    if (!h || !kept) return DSANLS_EINVAL;
    DeviceGuard dg(h->device);
    return guarded(h, [&]() {
        unsigned long long v = 0;
        DSANLS_CUDA(cudaStreamSynchronize(h->stream()));
        if (h->kept) DSANLS_CUDA(cudaMemcpy(&v, h->kept, sizeof v, cudaMemcpyDeviceToHost));
        *kept = (int64_t)v;
        return DSANLS_OK;
    });
}

int dsanls_harvest(dsanls_t h, int32_t side, int32_t iters, float *G, float *mu, float *b, float *xstar) {
    if (!h) return DSANLS_EINVAL;
    if ((side != 0 && side != 1) || iters < 1 || !G || !mu || !b || !xstar)
        return fail(h, DSANLS_EINVAL, "bad side, iters or output pointers");
    if (h->k > 32) return fail(h, DSANLS_EINVAL, "harvesting supports k <= 32");
    if (int rc = check_ready(h)) return rc;
    DeviceGuard dg(h->device);
    return guarded(h, [&]() {
        cudaStream_t s = h->stream();
        prepare(h);
        half_step(h, side, s, nullptr, false);
        const int64_t rows = side == 0 ? h->m : h->n;
        const float *Z = side == 0 ? h->U : h->V;
        mlp_harvest(Z, h->R, h->Gf, kp_bucket(h->k), h->scal[side], rows, h->k, iters, b, xstar, s);
        std::vector<double> g((size_t)h->k * h->k + 1);
        DSANLS_CUDA(cudaMemcpyAsync(g.data(), h->G64[side], (size_t)h->k * h->k * sizeof(double), cudaMemcpyDeviceToHost, s));
        DSANLS_CUDA(cudaMemcpyAsync(g.data() + (size_t)h->k * h->k, h->scal[side] + 1, sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
        DSANLS_CUDA(cudaStreamSynchronize(s));
        std::vector<float> gf(g.begin(), g.end());
        DSANLS_CUDA(cudaMemcpyAsync(G, gf.data(), (size_t)h->k * h->k * sizeof(float), cudaMemcpyHostToDevice, s));
        DSANLS_CUDA(cudaMemcpyAsync(mu, gf.data() + (size_t)h->k * h->k, sizeof(float), cudaMemcpyHostToDevice, s));
        DSANLS_CUDA(cudaStreamSynchronize(s));
        return DSANLS_OK;
    });
}

int dsanls_debug_fail_alloc_after(int64_t n) {
    g_alloc_budget.store(n < 0 ? -1 : n);
    return DSANLS_OK;
}

int dsanls_debug_tc_wait(uint64_t wait_ns, int32_t starve) {
    if (starve != 0 && starve != 1) return DSANLS_EINVAL;
    if (starve && wait_ns == 0) {
        record_handleless_error("dsanls_debug_tc_wait: a starved producer needs a short wait limit");
        return DSANLS_EINVAL;
    }
    return guarded(nullptr, [&]() {
        set_tc_wait_debug(wait_ns, starve);
        return DSANLS_OK;
    });
}

int dsanls_debug_bounds_report(int32_t reset, int64_t *out) {
    if (!out) return DSANLS_EINVAL;
    return guarded(nullptr, [&]() {
        int64_t a[3], b[3], c[3];
        bounds_report_subcsr(reset, a);
        bounds_report_sparse(reset, b);
        bounds_report_tc(reset, c);
        out[0] = a[0] + b[0] + c[0];
        out[1] = a[0] ? a[1] : (b[0] ? b[1] : c[1]);
        out[2] = a[0] ? a[2] : (b[0] ? b[2] : c[2]);
#ifdef DSANLS_BOUNDS
        return 1;
#else
        return 0;
#endif
    });
}

int dsanls_kernel_launches(uint64_t *out) {
    if (!out) return DSANLS_EINVAL;
    *out = launch_count();
    return DSANLS_OK;
}

const char *dsanls_last_error(dsanls_t h) {
    if (!h) return g_last_error.c_str();
    return h->err.c_str();
}

void dsanls_destroy(dsanls_t h) {
    if (!h) return;
    {
        DeviceGuard dg(h->device);
        if (h->own_stream) cudaStreamSynchronize(h->own_stream);
        if (h->opt.stream) cudaStreamSynchronize((cudaStream_t)h->opt.stream);
        invalidate_graph(h);
        dfree(h->M); dfree(h->MT); dfree(h->Mb); dfree(h->MTb);
        dfree(h->rp); dfree(h->trp); dfree(h->ci); dfree(h->tci); dfree(h->cv); dfree(h->tcv);
        dfree(h->U); dfree(h->V); dfree(h->U16); dfree(h->V16);
        dfree(h->S); dfree(h->Sb); dfree(h->J); dfree(h->A); dfree(h->W); dfree(h->Wpart); dfree(h->R);
        dfree(h->Rpart); dfree(h->Ytb); dfree(h->Bpart);
        dfree(h->P); dfree(h->Sn); dfree(h->Bb); dfree(h->Ptb); dfree(h->Ppart); dfree(h->Rpart2);
        dfree(h->Ptf); dfree(h->Pq); dfree(h->pscale); dfree(h->Spart);
        for (int a = 0; a < 3; ++a) {
            dfree(h->M3[a]); dfree(h->MT3[a]); dfree(h->St3[a]); dfree(h->Pt3[a]);
        }
        dfree(h->Mq); dfree(h->MTq); dfree(h->Sq); dfree(h->qscale[0]); dfree(h->qscale[1]);
        for (int side = 0; side < 2; ++side) {
            dfree(h->G64[side]);
            dfree(h->scal[side]);
        }
        dfree(h->Gf); dfree(h->work); dfree(h->t_dev); dfree(h->flag); dfree(h->dscal);
        dfree(h->bits); dfree(h->kept);
        h->sub[0].release();
        h->sub[1].release();
        if (h->aux_stream) {
            cudaStreamSynchronize(h->aux_stream);
            cudaStreamDestroy(h->aux_stream);
        }
        if (h->ev_fork) cudaEventDestroy(h->ev_fork);
        if (h->ev_join) cudaEventDestroy(h->ev_join);
        if (h->own_stream) cudaStreamDestroy(h->own_stream);
    }
    delete h;
}

// ---- stateless primitives ---------------------------------------------
int dsanls_philox_field(uint64_t seed, uint32_t stream_id, uint64_t t, int64_t rows, int64_t cols, uint32_t *out,
                        void *stream) {
    if (rows < 0 || cols < 0 || rows > (1ll << 34) || cols > (1ll << 31) - 1) return DSANLS_EINVAL;
    if (rows * cols > 0 && !out) return DSANLS_EINVAL;
    return guarded(nullptr, [&]() {
        launch_field_words(seed, stream_id, t, rows, cols, out, (cudaStream_t)stream);
        return DSANLS_OK;
    });
}

int dsanls_gaussian_field(uint64_t seed, uint32_t stream_id, uint64_t t, int64_t rows, int64_t cols, float scale,
                          int32_t transposed, float *out, void *stream) {
    if (rows < 0 || cols < 0 || rows > (1ll << 34) || cols > (1ll << 31) - 1) return DSANLS_EINVAL;
    if (rows * cols > 0 && !out) return DSANLS_EINVAL;
    return guarded(nullptr, [&]() {
        launch_gaussian_field<float>(seed, stream_id, t, nullptr, rows, cols, scale, transposed != 0, out, DRAW_GAUSS,
                                     nullptr, (cudaStream_t)stream);
        return DSANLS_OK;
    });
}

int dsanls_rademacher_field(uint64_t seed, uint32_t stream_id, uint64_t t, int64_t rows, int64_t cols, float scale,
                            int32_t transposed, float *out, void *stream) {
    if (rows < 0 || cols < 0 || rows > (1ll << 34) || cols > (1ll << 31) - 1) return DSANLS_EINVAL;
    if (rows * cols > 0 && !out) return DSANLS_EINVAL;
    return guarded(nullptr, [&]() {
        launch_gaussian_field<float>(seed, stream_id, t, nullptr, rows, cols, scale, transposed != 0, out,
                                     DRAW_RADEMACHER, nullptr, (cudaStream_t)stream);
        return DSANLS_OK;
    });
}

int dsanls_count_field(uint64_t seed, uint32_t side, uint64_t t, int64_t rows, int64_t cols, int32_t transposed,
                       float *out, void *stream) {
    if (rows < 0 || cols < 1 || rows > (1ll << 34) || cols > (1ll << 31) - 1 || side > 0xf) return DSANLS_EINVAL;
    if (rows * cols > 0 && !out) return DSANLS_EINVAL;
    return guarded(nullptr, [&]() {
        launch_gaussian_field<float>(seed, side, t, nullptr, rows, cols, 1.0f, transposed != 0, out, DRAW_COUNT,
                                     nullptr, (cudaStream_t)stream);
        return DSANLS_OK;
    });
}

int dsanls_srht_field(uint64_t seed, uint32_t side, uint64_t t, int64_t rows, int64_t cols, float scale,
                      int32_t transposed, float *out, void *stream) {
    if (rows < 1 || cols < 1 || rows > (1ll << 30) || cols > srht_pad(rows) || side > 0xf || !out)
        return DSANLS_EINVAL;
    return guarded(nullptr, [&]() {
        const int64_t p = srht_pad(rows);
        cudaStream_t s = (cudaStream_t)stream;
        int32_t *J = nullptr;      // scratch: the sampled Hadamard columns
        uint32_t *bits = nullptr;  // scratch: their membership bitmap
        DSANLS_CUDA(cudaMalloc((void **)&J, (size_t)cols * sizeof(int32_t)));
        const cudaError_t ea = cudaMalloc((void **)&bits, (size_t)ceil_div(p, 32) * sizeof(uint32_t));
        if (ea != cudaSuccess) {
            cudaFree(J);
            DSANLS_CUDA(ea);
        }
        try {
            launch_subsample(seed, 0x40u | side, t, nullptr, p, (int)cols, J, bits, s);
            launch_gaussian_field<float>(seed, side, t, nullptr, rows, cols, scale, transposed != 0, out, DRAW_SRHT,
                                         J, s);
        } catch (...) {
            cudaFree(J);
            cudaFree(bits);
            throw;
        }
        const cudaError_t e = cudaStreamSynchronize(s);
        cudaFree(J);
        cudaFree(bits);
        DSANLS_CUDA(e);
        return DSANLS_OK;
    });
}

int dsanls_uniform_field(uint64_t seed, uint32_t stream_id, uint64_t t, int64_t rows, int64_t cols, float *out,
                         void *stream) {
    if (rows < 0 || cols < 0 || rows > (1ll << 34) || cols > (1ll << 31) - 1) return DSANLS_EINVAL;
    if (rows * cols > 0 && !out) return DSANLS_EINVAL;
    return guarded(nullptr, [&]() {
        launch_uniform_field(seed, stream_id, t, rows, cols, out, (cudaStream_t)stream);
        return DSANLS_OK;
    });
}

int dsanls_subsample_indices(uint64_t seed, uint32_t side, uint64_t t, int64_t n, int32_t d, int32_t *J,
                             void *stream) {
    if (n < 1 || n > (1ll << 31) - 1 || d < 1 || d > n || !J || side > 0xef) return DSANLS_EINVAL;
    return guarded(nullptr, [&]() {
        uint32_t *bits = nullptr;  // scratch bitmap of this call
        DSANLS_CUDA(cudaMalloc((void **)&bits, (size_t)ceil_div(n, 32) * sizeof(uint32_t)));
        try {
            launch_subsample(seed, side, t, nullptr, n, d, J, bits, (cudaStream_t)stream);
        } catch (...) {
            cudaFree(bits);
            throw;
        }
        const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        cudaFree(bits);
        DSANLS_CUDA(e);
        return DSANLS_OK;
    });
}

}  // extern "C"
