// C ABI of the batched form: many independent dense problems, one persistent
// work-queue launch per phase, one CUDA graph per outer iteration, and an
// autotuner for the persistent launch geometry.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <initializer_list>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/dsanls.h"
#include "batch.cuh"
#include "common.cuh"
#include "kernels.cuh"

using namespace dsanls;

struct dsanls_batch_ctx {
    int device = 0;
    std::vector<BatchInst> h;
    BatchDev g;
    BatchLaunch cfg;
    bool tuned = false;
    int forced_tile[2] = {0, 0};  // per side: a tile set by dsanls_batch_set_tile (code of apply_tile), 0: tune
    dsanls_options opt{};
    int64_t t_host = 0;
    cudaStream_t own_stream = nullptr;
    // forked iteration: the main path on `lead` (highest priority), the Gram and
    // the V-half sketch on the fork's streams (lower priorities)
    cudaStream_t lead = nullptr;
    BatchFork fork;
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;
    cudaGraphExec_t graph = nullptr;
    uint64_t graph_launches = 0;
    std::vector<char> has_data;
    int64_t data_elems = 0;   // packed M_i and M_i^T
    int64_t datap_elems = 0, st_elems = 0, yt_elems = 0;  // padded bf16 data, S^T, Y^T (tensor-core form)
    bool bf16_stale = true;   // the bf16 copies of data no longer match it
    std::vector<double> mm;  // ||M_i||^2
    double *work = nullptr;
    double *dres = nullptr;  // residual^2 per instance
    std::string err;
    cudaStream_t stream() const { return opt.stream ? (cudaStream_t)opt.stream : own_stream; }
};

namespace {

constexpr int64_t B_WORK = 152 * 8;

template <typename T>
void balloc(T *&p, int64_t count) {
    if (p) cudaFree(p);
    p = nullptr;
    if (count <= 0) return;
    if (cudaMalloc((void **)&p, (size_t)count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        throw std::bad_alloc();
    }
}

template <typename T>
void bfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

template <typename F>
int bguard(dsanls_batch_ctx *b, F &&body) {
    try {
        return body();
    } catch (const CudaError &e) {
        b->err = std::string("CUDA error: ") + cudaGetErrorString(e.err) + " (" + e.where + ")";
        cudaGetLastError();
        return DSANLS_ECUDA;
    } catch (const ArgError &e) {
        b->err = e.what;
        return DSANLS_EINVAL;
    } catch (const std::bad_alloc &) {
        b->err = "out of memory";
        return DSANLS_ENOMEM;
    } catch (...) {
        b->err = "unexpected internal error";
        return DSANLS_ECUDA;
    }
}

void drop_graph(dsanls_batch_ctx *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

// One outer iteration on s.  The work forks from s onto the handle's streams
// and joins back into it, so that everything after it on s (and a graph
// captured on s) sees the iteration complete: the main path runs on `lead`; the
// Gram of each half-step starts on fork.gram once B is done and joins before the
// update; in the tensor-core form the V-half sketch S_1^T (it needs only the
// seed and t) is drawn on fork.sketch from the start of the iteration and
// joined before the V-half's B.
void iteration(dsanls_batch_ctx *b, cudaStream_t s) {
    BatchFork f = b->fork;
    cudaStream_t ls = b->lead;
    f.sketch_ahead = b->g.tc && b->g.bf16 && b->g.order == DSANLS_ORDER_PAPER;
    DSANLS_CUDA(cudaEventRecord(b->ev_start, s));
    DSANLS_CUDA(cudaStreamWaitEvent(ls, b->ev_start, 0));
    if (f.sketch_ahead) {
        DSANLS_CUDA(cudaStreamWaitEvent(f.sketch, b->ev_start, 0));
        launch_batch_sketch_t(b->g, 1, f.sketch);
        DSANLS_CUDA(cudaEventRecord(f.s_done, f.sketch));
    }
    batch_half_step(b->g, 0, b->cfg, ls, nullptr, &f);
    batch_half_step(b->g, 1, b->cfg, ls, nullptr, &f);
    launch_increment_t(b->g.t_dev, 1, ls);
    DSANLS_CUDA(cudaEventRecord(b->ev_end, ls));
    DSANLS_CUDA(cudaStreamWaitEvent(s, b->ev_end, 0));
}

// bf16 form: bring the bf16 copy of the packed data (CUDA-core kernels) or its
// padded copy (tensor-core product) up to date after set_dense
void refresh_bf16(dsanls_batch_ctx *b, cudaStream_t s) {
    if (b->g.bf16 && b->bf16_stale) {
        if (b->g.tc)
            launch_batch_pad_bf16(b->g, s);
        else
            launch_copy_cast_bf16(b->g.data, b->data_elems, b->g.data_b, s);
        b->bf16_stale = false;
    }
}

// ---- autotuner: persistent CTAs per SM, cached per batch shape and dtype ----
std::mutex g_tune_mutex;
std::map<std::string, int> g_tune_cache;

std::string tune_key(const dsanls_batch_ctx *b) {
    std::vector<std::string> shapes;
    for (const BatchInst &i : b->h) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "%lld,%lld,%d,%d,%d", (long long)i.m, (long long)i.n, i.k, i.d, i.dv);
        shapes.push_back(buf);
    }
    std::sort(shapes.begin(), shapes.end());
    const std::string form = std::string(b->g.bf16 ? "bf16" : "f32") + (b->g.order == 1 ? "r" : "") +
                             (b->g.tc ? "tc10" : "");
    std::string key = form;
    for (const std::string &sh : shapes) key += ";" + sh;
    return std::to_string(std::hash<std::string>()(key)) + "/" + form;
}

std::string cache_path() {
    const char *p = std::getenv("DSANLS_TUNE_CACHE");
    return p ? std::string(p) : std::string();
}

bool cache_lookup(const std::string &key, int &value) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
        value = it->second;
        return true;
    }
    const std::string path = cache_path();
    if (path.empty()) return false;
    FILE *f = std::fopen(path.c_str(), "r");
    if (!f) return false;
    char k[256];
    int v;
    bool found = false;
    while (std::fscanf(f, "%255s %d", k, &v) == 2) {
        g_tune_cache[k] = v;
        if (key == k) {
            value = v;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const std::string &key, int value) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = value;
    const std::string path = cache_path();
    if (path.empty()) return;
    FILE *f = std::fopen(path.c_str(), "a");
    if (!f) return;
    std::fprintf(f, "%s %d\n", key.c_str(), value);
    std::fclose(f);
}

// A tile of the tensor-core product: 1000000 x the pipeline (0 cp.async ring, 1
// TMA ring, 2 TMA ring with the epilogue off the copy path) + 10000 x the row
// tiles per item + 1000 x the ring stages + the chunk width.
void apply_tile(dsanls_batch_ctx *b, int side, int code, int sms) {
    TcTile &t = b->cfg.tc[side];
    t.mode = code / 1000000;
    t.rt = (code / 10000) % 10;
    t.stages = (code / 1000) % 10;
    t.nc = code % 1000;
    if (!batch_tc_tile_built(t.nc, t.stages, t.rt, t.mode)) throw ArgError{"tuned tile configuration not built"};
    t.ctas = sms * batch_tc_ctas_per_sm(t.nc, t.stages, t.rt, t.mode);
    b->cfg.tc_b_ctas = sms * batch_tc_b_ctas_per_sm();
}

// The candidate tiles of the tensor-core product.
std::vector<int> tile_candidates() {
    std::vector<int> c;
    // (chunk, stages, row tiles) of the cp.async and TMA rings
    const int tiles[10][3] = {{64, 4, 1}, {128, 3, 1}, {128, 4, 1}, {256, 4, 1}, {64, 2, 1},
                              {64, 4, 2}, {128, 3, 2}, {128, 4, 2}, {192, 3, 2}, {64, 2, 2}};
    for (const auto &tl : tiles)
        for (int mode : {0, 1}) c.push_back(mode * 1000000 + tl[2] * 10000 + tl[1] * 1000 + tl[0]);
    // the ring with the epilogue off the copy path (two row tiles per item)
    const int ws_tiles[4][2] = {{256, 3}, {192, 3}, {128, 4}, {64, 5}};
    for (const auto &tl : ws_tiles) c.push_back(2 * 1000000 + 2 * 10000 + tl[1] * 1000 + tl[0]);
    return c;
}

// Tensor-core form: the tile of each half-step is chosen by the time of a full
// outer iteration (forked as in a step, so a tile whose shared memory leaves no
// room for the side streams' kernels pays for it), the other half-step's tile
// held; then the CTAs per SM of the CUDA-core kernels.  Other forms: the CTAs per
// SM.  Each candidate runs two iterations, the second timed; the factors and t
// are restored after the trials.
void autotune(dsanls_batch_ctx *b) {
    int sms = 152;
    DSANLS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    const std::string key = tune_key(b);
    int per_sm = 0, code[2] = {0, 0};
    bool cached = cache_lookup(key + "#p", per_sm);
    if (b->g.tc)
        for (int side = 0; side < 2; ++side)
            cached = cached && (b->forced_tile[side] || cache_lookup(key + "#" + std::to_string(side), code[side]));
    if (!cached) {
        cudaStream_t s = b->stream();
        int64_t fbytes = 0;
        for (const BatchInst &i : b->h) fbytes = std::max<int64_t>(fbytes, i.offV + i.n * i.k);
        float *backup = nullptr;
        balloc(backup, fbytes);
        int64_t t_backup = 0;
        DSANLS_CUDA(cudaMemcpyAsync(&t_backup, b->g.t_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        DSANLS_CUDA(cudaMemcpyAsync(backup, b->g.factors, fbytes * sizeof(float), cudaMemcpyDeviceToDevice, s));
        cudaEvent_t ev[6] = {};
        int created = 0;
        auto restore = [&]() {
            DSANLS_CUDA(cudaMemcpyAsync(b->g.factors, backup, fbytes * sizeof(float), cudaMemcpyDeviceToDevice, s));
            DSANLS_CUDA(cudaMemcpyAsync(b->g.t_dev, &t_backup, sizeof(int64_t), cudaMemcpyHostToDevice, s));
            DSANLS_CUDA(cudaStreamSynchronize(s));
        };
        // two forked outer iterations, the second timed (ms)
        auto time_iteration = [&]() -> float {
            iteration(b, s);
            DSANLS_CUDA(cudaEventRecord(ev[0], s));
            iteration(b, s);
            DSANLS_CUDA(cudaEventRecord(ev[1], s));
            DSANLS_CUDA(cudaEventSynchronize(ev[1]));
            float ms = 0.0f;
            DSANLS_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
            return ms;
        };
        try {
            for (; created < 6; ++created) DSANLS_CUDA(cudaEventCreate(&ev[created]));
            b->cfg.persistent_blocks = 152 * 2;
            if (b->g.tc) {
                const std::vector<int> cand = tile_candidates();
                const int start = 1 * 1000000 + 2 * 10000 + 3 * 1000 + 192;  // TMA ring, (192, 3, 2)
                for (int side = 0; side < 2; ++side) {
                    code[side] = b->forced_tile[side] ? b->forced_tile[side] : start;
                    apply_tile(b, side, code[side], sms);
                }
                for (int side = 0; side < 2; ++side) {
                    if (b->forced_tile[side]) continue;
                    float best = 1e30f;
                    for (int c : cand) {
                        apply_tile(b, side, c, sms);
                        const float ms = time_iteration();
                        if (ms < best) {
                            best = ms;
                            code[side] = c;
                        }
                    }
                    apply_tile(b, side, code[side], sms);
                    restore();
                }
            }
            float best = 1e30f;
            for (int c : b->g.tc ? std::vector<int>{2, 4} : std::vector<int>{1, 2, 4, 8}) {
                b->cfg.persistent_blocks = 152 * c;
                const float ms = time_iteration();
                if (ms < best) {
                    best = ms;
                    per_sm = c;
                }
                restore();
            }
        } catch (...) {
            for (int i = 0; i < created; ++i) cudaEventDestroy(ev[i]);
            bfree(backup);
            throw;
        }
        for (int i = 0; i < created; ++i) cudaEventDestroy(ev[i]);
        bfree(backup);
        cache_store(key + "#p", per_sm);
        if (b->g.tc)
            for (int side = 0; side < 2; ++side)
                if (!b->forced_tile[side]) cache_store(key + "#" + std::to_string(side), code[side]);
    }
    b->cfg.persistent_blocks = 152 * per_sm;
    if (b->g.tc)
        for (int side = 0; side < 2; ++side) apply_tile(b, side, b->forced_tile[side] ? b->forced_tile[side] : code[side], sms);
    b->tuned = true;
}

int bfail(dsanls_batch_ctx *b, int code, const char *msg) {
    b->err = msg;
    return code;
}

}  // namespace

extern "C" {

int dsanls_batch_create(int32_t count, const int64_t *m, const int64_t *n, const int32_t *k, const int32_t *d,
                        const int32_t *d_v, const uint64_t *seeds, dsanls_batch_t *out) {
    if (!out) return DSANLS_EINVAL;
    *out = nullptr;
    if (count < 1 || !m || !n || !k || !d || !d_v || !seeds) return DSANLS_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (m[i] < 1 || n[i] < 1 || m[i] > (1 << 24) || n[i] > (1 << 24)) return DSANLS_EINVAL;
        if (k[i] < 1 || k[i] > 32 || d[i] < 1 || d_v[i] < 1 || d[i] > (1 << 20) || d_v[i] > (1 << 20))
            return DSANLS_EINVAL;
    }
    dsanls_batch_ctx *b = nullptr;
    try {
        b = new dsanls_batch_ctx();
    } catch (...) {
        return DSANLS_ENOMEM;
    }
    dsanls_default_options(&b->opt);
    const int rc = bguard(b, [&]() {
        DSANLS_CUDA(cudaGetDevice(&b->device));
        DSANLS_CUDA(cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking));
        {
            int least = 0, greatest = 0;  // numerically: greatest <= least
            DSANLS_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
            DSANLS_CUDA(cudaStreamCreateWithPriority(&b->lead, cudaStreamNonBlocking, greatest));
            DSANLS_CUDA(cudaStreamCreateWithPriority(&b->fork.gram, cudaStreamNonBlocking, (least + greatest) / 2));
            DSANLS_CUDA(cudaStreamCreateWithPriority(&b->fork.sketch, cudaStreamNonBlocking, least));
            for (cudaEvent_t *e : {&b->ev_start, &b->ev_end, &b->fork.b_done[0], &b->fork.b_done[1],
                                   &b->fork.g_done[0], &b->fork.g_done[1], &b->fork.s_done})
                DSANLS_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        }
        prime_kernel_attributes();
        b->h.resize(count);
        int64_t offM = 0, offF = 0, offS = 0, offB = 0, offR = 0, offG = 0, offMp = 0, offSt = 0, offYt = 0;
        auto pad8 = [](int64_t x) { return (x + 7) & ~(int64_t)7; };
        for (int i = 0; i < count; ++i) {
            BatchInst &x = b->h[i];
            std::memset(&x, 0, sizeof x);
            x.m = m[i];
            x.n = n[i];
            x.k = k[i];
            x.d = d[i];
            x.dv = d_v[i];
            x.seed = seeds[i];
            x.scale[0] = (float)(1.0 / std::sqrt((double)d[i]));
            x.scale[1] = (float)(1.0 / std::sqrt((double)d_v[i]));
            x.offM = offM;
            offM += 2 * x.m * x.n;
            x.offU = offF;
            offF += x.m * x.k;
            x.offV = offF;
            offF += x.n * x.k;
            x.offS = offS;
            offS += std::max(x.n * x.d, x.m * x.dv);
            x.offB = offB;
            offB += (int64_t)x.k * std::max(x.d, x.dv);
            x.offR = offR;
            offR += std::max(x.m, x.n) * x.k;
            x.offG = offG;
            offG += (int64_t)x.k * x.k + 4;
            x.offMp = offMp;
            offMp += pad8(x.m * pad8(x.n)) + pad8(x.n * pad8(x.m));
            x.offSt = offSt;
            offSt += pad8((int64_t)x.d * pad8(x.n));
            x.offSt1 = offSt;
            offSt += pad8((int64_t)x.dv * pad8(x.m));
            x.offYt = offYt;
            offYt += pad8((int64_t)x.k * std::max(pad8(x.n), pad8(x.m)));
        }
        b->datap_elems = offMp;
        b->st_elems = offSt;
        b->yt_elems = offYt;
        cudaStream_t s = b->stream();
        BatchDev &g = b->g;
        g.count = count;
        balloc(g.inst, count);
        balloc(g.data, offM);
        b->data_elems = offM;
        balloc(g.factors, offF);
        balloc(g.S, offS);
        balloc(g.B, offB);
        balloc(g.R, offR);
        balloc(g.P, offR);
        balloc(g.G, offG);
        balloc(g.counters, 12);
        balloc(g.t_dev, 1);
        balloc(g.flag, 1);
        balloc(b->work, B_WORK);
        balloc(b->dres, count);
        DSANLS_CUDA(cudaMemcpyAsync(g.inst, b->h.data(), count * sizeof(BatchInst), cudaMemcpyHostToDevice, s));
        DSANLS_CUDA(cudaMemsetAsync(g.t_dev, 0, sizeof(int64_t), s));
        DSANLS_CUDA(cudaMemsetAsync(g.flag, 0, sizeof(int), s));
        for (int side = 0; side < 2; ++side) {
            std::vector<int2> bi, ai, ui, pi;
            std::vector<int64_t> pre;
            batch_build_items(b->h, side, bi, ai, ui, pi, pre);
            balloc(g.pitems[side], (int64_t)pi.size());
            g.np[side] = (int)pi.size();
            DSANLS_CUDA(cudaMemcpyAsync(g.pitems[side], pi.data(), pi.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
            balloc(g.bitems[side], (int64_t)bi.size());
            balloc(g.aritems[side], (int64_t)ai.size());
            balloc(g.uitems[side], (int64_t)ui.size());
            balloc(g.sketch_prefix[side], (int64_t)pre.size());
            g.nb[side] = (int)bi.size();
            g.nar[side] = (int)ai.size();
            g.nu[side] = (int)ui.size();
            DSANLS_CUDA(cudaMemcpyAsync(g.bitems[side], bi.data(), bi.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
            DSANLS_CUDA(cudaMemcpyAsync(g.aritems[side], ai.data(), ai.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
            DSANLS_CUDA(cudaMemcpyAsync(g.uitems[side], ui.data(), ui.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
            DSANLS_CUDA(cudaMemcpyAsync(g.sketch_prefix[side], pre.data(), pre.size() * sizeof(int64_t),
                                        cudaMemcpyHostToDevice, s));
            std::vector<int2> ti, ti2, tb;
            batch_build_tc_items(b->h, side, ti, ti2, tb);
            balloc(g.tcitems[side], (int64_t)ti.size());
            balloc(g.tcitems2[side], (int64_t)ti2.size());
            balloc(g.tcbitems[side], (int64_t)tb.size());
            g.ntc[side] = (int)ti.size();
            g.ntc2[side] = (int)ti2.size();
            g.ntcb[side] = (int)tb.size();
            DSANLS_CUDA(cudaMemcpyAsync(g.tcitems[side], ti.data(), ti.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
            DSANLS_CUDA(cudaMemcpyAsync(g.tcitems2[side], ti2.data(), ti2.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                        s));
            DSANLS_CUDA(cudaMemcpyAsync(g.tcbitems[side], tb.data(), tb.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
            DSANLS_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
        }
        batch_init_factors(g.inst, count, g.factors, s);
        b->has_data.assign(count, 0);
        b->mm.assign(count, 0.0);
        DSANLS_CUDA(cudaStreamSynchronize(s));
        return DSANLS_OK;
    });
    if (rc != DSANLS_OK) {
        record_handleless_error(b->err);
        dsanls_batch_destroy(b);
        return rc;
    }
    *out = b;
    return DSANLS_OK;
}

int dsanls_batch_set_options(dsanls_batch_t b, const dsanls_options *opt) {
    if (!b) return DSANLS_EINVAL;
    if (!opt) return bfail(b, DSANLS_EINVAL, "options pointer is NULL");
    if (opt->solver != DSANLS_SOLVER_PGD && opt->solver != DSANLS_SOLVER_RCD) return bfail(b, DSANLS_EINVAL, "unknown solver");
    if (opt->precision != DSANLS_PREC_FP32 && opt->precision != DSANLS_PREC_BF16)
        return bfail(b, DSANLS_EINVAL, "the batched form computes in binary32 or bf16");
    if (opt->power_iters < 0 || opt->power_iters > 10000 || !(opt->alpha >= 0.0) || !(opt->beta >= 0.0) ||
        !std::isfinite(opt->alpha) || !std::isfinite(opt->beta) || opt->t < 0)
        return bfail(b, DSANLS_EINVAL, "bad power_iters, alpha, beta or t");
    if (opt->bound_clamp) return bfail(b, DSANLS_EINVAL, "the batched form has no bound clamp");
    if (opt->inner_iters != 1) return bfail(b, DSANLS_EINVAL, "the batched form takes one solver step per half");
    if (opt->order != DSANLS_ORDER_PAPER && opt->order != DSANLS_ORDER_REASSOCIATED)
        return bfail(b, DSANLS_EINVAL, "unknown order");
    return bguard(b, [&]() {
        DSANLS_CUDA(cudaStreamSynchronize(b->stream()));
        b->opt = *opt;
        b->g.solver = opt->solver;
        b->g.alpha = opt->alpha;
        b->g.beta = opt->beta;
        b->g.power_iters = opt->power_iters;
        if (b->g.order != opt->order || b->g.bf16 != (opt->precision == DSANLS_PREC_BF16))
            b->tuned = false;  // the launch geometry is tuned per form
        b->g.order = opt->order;
        b->g.bf16 = opt->precision == DSANLS_PREC_BF16 ? 1 : 0;
        // bf16 in the paper order runs the right-hand side on tensor cores
        b->g.tc = (b->g.bf16 && b->g.order == DSANLS_ORDER_PAPER) ? 1 : 0;
        if (b->g.bf16 && !b->g.tc && !b->g.data_b) balloc(b->g.data_b, b->data_elems);
        if (b->g.tc && !b->g.data_p) {
            balloc(b->g.data_p, b->datap_elems);
            balloc(b->g.St, b->st_elems);
            balloc(b->g.Yt, b->yt_elems);
            std::vector<CUtensorMap> maps;
            batch_tc_encode_maps(b->h, b->g, maps);
            balloc(b->g.tmaps, (int64_t)maps.size());
            DSANLS_CUDA(cudaMemcpy(b->g.tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
        }
        b->bf16_stale = true;
        drop_graph(b);
        if (opt->t != b->t_host) {
            b->t_host = opt->t;
            DSANLS_CUDA(cudaMemcpyAsync(b->g.t_dev, &b->t_host, sizeof(int64_t), cudaMemcpyHostToDevice, b->stream()));
        }
        DSANLS_CUDA(cudaStreamSynchronize(b->stream()));
        return DSANLS_OK;
    });
}

int dsanls_batch_set_dense(dsanls_batch_t b, int32_t i, const float *M, int64_t ld, int32_t on_device) {
    if (!b) return DSANLS_EINVAL;
    if (i < 0 || i >= (int)b->h.size()) return bfail(b, DSANLS_EINVAL, "instance index out of range");
    const BatchInst &x = b->h[i];
    if (!M || ld < x.n) return bfail(b, DSANLS_EINVAL, "M is NULL or ld < n");
    return bguard(b, [&]() {
        cudaStream_t s = b->stream();
        float *dst = b->g.data + x.offM;
        DSANLS_CUDA(cudaMemcpy2DAsync(dst, x.n * sizeof(float), M, ld * sizeof(float), x.n * sizeof(float), x.m,
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        launch_transpose(dst, x.n, x.m, x.n, dst + x.m * x.n, x.m, s);
        launch_sumsq(dst, x.m * x.n, b->work, B_WORK, b->dres + i, s);
        double v = 0.0;
        DSANLS_CUDA(cudaMemcpyAsync(&v, b->dres + i, sizeof(double), cudaMemcpyDeviceToHost, s));
        DSANLS_CUDA(cudaStreamSynchronize(s));
        b->mm[i] = v;
        b->has_data[i] = 1;
        b->bf16_stale = true;
        return DSANLS_OK;
    });
}

int dsanls_batch_set_factors(dsanls_batch_t b, int32_t i, const float *U, const float *V, int32_t on_device) {
    if (!b) return DSANLS_EINVAL;
    if (i < 0 || i >= (int)b->h.size()) return bfail(b, DSANLS_EINVAL, "instance index out of range");
    const BatchInst &x = b->h[i];
    return bguard(b, [&]() {
        cudaStream_t s = b->stream();
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (U) DSANLS_CUDA(cudaMemcpyAsync(b->g.factors + x.offU, U, x.m * x.k * sizeof(float), kind, s));
        if (V) DSANLS_CUDA(cudaMemcpyAsync(b->g.factors + x.offV, V, x.n * x.k * sizeof(float), kind, s));
        DSANLS_CUDA(cudaStreamSynchronize(s));
        return DSANLS_OK;
    });
}

int dsanls_batch_step(dsanls_batch_t b, int32_t outer_iters) {
    if (!b) return DSANLS_EINVAL;
    if (outer_iters < 0) return bfail(b, DSANLS_EINVAL, "outer_iters < 0");
    for (char c : b->has_data)
        if (!c) return bfail(b, DSANLS_ESTATE, "every instance needs dsanls_batch_set_dense first");
    return bguard(b, [&]() {
        cudaStream_t s = b->stream();
        refresh_bf16(b, s);
        if (!b->tuned) autotune(b);
        if (b->opt.use_graph) {
            if (!b->graph) {
                cudaGraph_t gr = nullptr;
                const uint64_t before = launch_count();
                DSANLS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                try {
                    iteration(b, s);
                } catch (...) {
                    cudaGraph_t dummy = nullptr;
                    cudaStreamEndCapture(s, &dummy);
                    if (dummy) cudaGraphDestroy(dummy);
                    throw;
                }
                DSANLS_CUDA(cudaStreamEndCapture(s, &gr));
                b->graph_launches = launch_count() - before;
                add_launches(0 - b->graph_launches);
                // the kernel nodes keep the priorities of the streams they were captured on
                const cudaError_t e = cudaGraphInstantiate(&b->graph, gr, cudaGraphInstantiateFlagUseNodePriority);
                cudaGraphDestroy(gr);
                DSANLS_CUDA(e);
            }
            for (int it = 0; it < outer_iters; ++it) DSANLS_CUDA(cudaGraphLaunch(b->graph, s));
            add_launches(b->graph_launches * (uint64_t)outer_iters);
        } else {
            for (int it = 0; it < outer_iters; ++it) iteration(b, s);
        }
        b->t_host += outer_iters;
        return DSANLS_OK;
    });
}

int dsanls_batch_get_factors(dsanls_batch_t b, int32_t i, float *U, float *V, int32_t on_device) {
    if (!b) return DSANLS_EINVAL;
    if (i < 0 || i >= (int)b->h.size()) return bfail(b, DSANLS_EINVAL, "instance index out of range");
    const BatchInst &x = b->h[i];
    return bguard(b, [&]() {
        cudaStream_t s = b->stream();
        DSANLS_CUDA(cudaStreamSynchronize(s));
        int flag = 0;
        DSANLS_CUDA(cudaMemcpy(&flag, b->g.flag, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) {
            DSANLS_CUDA(cudaMemset(b->g.flag, 0, sizeof(int)));
            return bfail(b, DSANLS_ENUMERIC, "an update produced NaN or Inf");
        }
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (U) DSANLS_CUDA(cudaMemcpyAsync(U, b->g.factors + x.offU, x.m * x.k * sizeof(float), kind, s));
        if (V) DSANLS_CUDA(cudaMemcpyAsync(V, b->g.factors + x.offV, x.n * x.k * sizeof(float), kind, s));
        DSANLS_CUDA(cudaStreamSynchronize(s));
        return DSANLS_OK;
    });
}

int dsanls_batch_rel_error(dsanls_batch_t b, double *out) {
    if (!b) return DSANLS_EINVAL;
    if (!out) return bfail(b, DSANLS_EINVAL, "out is NULL");
    return bguard(b, [&]() {
        cudaStream_t s = b->stream();
        const int count = (int)b->h.size();
        for (int i = 0; i < count; ++i) {
            const BatchInst &x = b->h[i];
            launch_dense_residual(b->g.data + x.offM, x.n, b->g.factors + x.offU, b->g.factors + x.offV, x.m, x.n,
                                  x.k, b->work, B_WORK, b->dres + i, s);
        }
        std::vector<double> r(count);
        DSANLS_CUDA(cudaMemcpyAsync(r.data(), b->dres, count * sizeof(double), cudaMemcpyDeviceToHost, s));
        DSANLS_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < count; ++i) out[i] = b->mm[i] > 0.0 ? std::sqrt(std::max(r[i], 0.0) / b->mm[i]) : 0.0;
        return DSANLS_OK;
    });
}

int dsanls_batch_profile(dsanls_batch_t b, double *ms) {
    if (!b || !ms) return DSANLS_EINVAL;
    for (char c : b->has_data)
        if (!c) return bfail(b, DSANLS_ESTATE, "every instance needs dsanls_batch_set_dense first");
    cudaEvent_t ev[6] = {};
    int created = 0;
    const int rc = bguard(b, [&]() {
        refresh_bf16(b, b->stream());
        if (!b->tuned) autotune(b);
        for (; created < 6; ++created) DSANLS_CUDA(cudaEventCreate(&ev[created]));
        cudaStream_t s = b->stream();
        for (int side = 0; side < 2; ++side) {
            batch_half_step(b->g, side, b->cfg, s, ev);
            DSANLS_CUDA(cudaEventSynchronize(ev[5]));
            for (int p = 0; p < 5; ++p) {
                float t = 0.0f;
                DSANLS_CUDA(cudaEventElapsedTime(&t, ev[p], ev[p + 1]));
                ms[side * 5 + p] = t;
            }
        }
        return DSANLS_OK;
    });
    for (int i = 0; i < created; ++i) cudaEventDestroy(ev[i]);
    return rc;
}

int dsanls_batch_tuned_blocks(dsanls_batch_t b, int32_t *persistent_ctas) {
    if (!b || !persistent_ctas) return DSANLS_EINVAL;
    *persistent_ctas = b->tuned ? b->cfg.persistent_blocks : 0;
    return DSANLS_OK;
}

int dsanls_batch_set_tile(dsanls_batch_t b, int32_t side, int32_t chunk, int32_t stages, int32_t row_tiles,
                          int32_t pipeline) {
    if (!b) return DSANLS_EINVAL;
    if (side < -1 || side > 1) return bfail(b, DSANLS_EINVAL, "side must be 0, 1 or -1 (both)");
    int code = 0;
    if (!(chunk == 0 && stages == 0 && row_tiles == 0)) {
        if (!batch_tc_tile_built(chunk, stages, row_tiles, pipeline))
            return bfail(b, DSANLS_EINVAL, "no such tile: pipeline 0 or 1 with (64,4,1) (128,3,1) (128,4,1) (256,4,1) "
                                           "(64,2,1) (64,4,2) (128,3,2) (128,4,2) (192,3,2) (64,2,2); pipeline 2 "
                                           "with (256,3,2) (192,3,2) (128,4,2) (64,5,2)");
        code = pipeline * 1000000 + row_tiles * 10000 + stages * 1000 + chunk;
    }
    for (int sd = 0; sd < 2; ++sd)
        if (side == -1 || side == sd) b->forced_tile[sd] = code;
    b->tuned = false;
    drop_graph(b);
    return DSANLS_OK;
}

int dsanls_batch_tuned_tile(dsanls_batch_t b, int32_t side, int32_t *chunk, int32_t *ctas, int32_t *row_tiles,
                            int32_t *pipeline) {
    if (!b || !chunk || !ctas || side < 0 || side > 1) return DSANLS_EINVAL;
    const bool tc = b->tuned && b->g.tc;
    const TcTile &t = b->cfg.tc[side];
    *chunk = tc ? t.nc : 0;
    *ctas = tc ? t.ctas : 0;
    if (row_tiles) *row_tiles = tc ? t.rt : 0;
    if (pipeline) *pipeline = tc ? t.mode : 0;
    return DSANLS_OK;
}

const char *dsanls_batch_last_error(dsanls_batch_t b) { return b ? b->err.c_str() : "invalid handle"; }

void dsanls_batch_destroy(dsanls_batch_t b) {
    if (!b) return;
    if (b->own_stream) cudaStreamSynchronize(b->own_stream);
    if (b->opt.stream) cudaStreamSynchronize((cudaStream_t)b->opt.stream);
    drop_graph(b);
    BatchDev &g = b->g;
    bfree(g.inst); bfree(g.data); bfree(g.factors); bfree(g.S); bfree(g.B); bfree(g.R); bfree(g.P); bfree(g.G); bfree(g.data_b);
    bfree(g.data_p); bfree(g.St); bfree(g.Yt); bfree(g.tmaps);
    for (int side = 0; side < 2; ++side) {
        bfree(g.bitems[side]); bfree(g.aritems[side]); bfree(g.uitems[side]); bfree(g.sketch_prefix[side]); bfree(g.pitems[side]);
        bfree(g.tcitems[side]); bfree(g.tcitems2[side]); bfree(g.tcbitems[side]);
    }
    bfree(g.counters); bfree(g.t_dev); bfree(g.flag); bfree(b->work); bfree(b->dres);
    for (cudaStream_t st : {b->lead, b->fork.gram, b->fork.sketch})
        if (st) cudaStreamSynchronize(st);
    for (cudaEvent_t e : {b->ev_start, b->ev_end, b->fork.b_done[0], b->fork.b_done[1], b->fork.g_done[0],
                          b->fork.g_done[1], b->fork.s_done})
        if (e) cudaEventDestroy(e);
    for (cudaStream_t st : {b->lead, b->fork.gram, b->fork.sketch})
        if (st) cudaStreamDestroy(st);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete b;
}

}  // extern "C"
