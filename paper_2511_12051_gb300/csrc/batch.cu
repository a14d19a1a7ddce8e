// Batches of independent stacks (uneven N, one window): scratch owned by the
// batch, a launch schedule tuned per (N, window) on the first run, and the
// whole batch recorded as one CUDA graph (stacks spread over several streams,
// longest first) that every run launches with a single call.  Host code only.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "api_internal.h"

using namespace plkapi;

struct plk_batch {
    static constexpr int kStreams = 4;
    struct Stack {
        plk_stack_desc d;
        plk::Geom g;
        plk::Planes z;
        long long npix, nout;
        float c;                   // GLRT threshold for n_eff = N (single precision)
        float *sum_pow;            // [H][W]
        uint64_t *mask;            // [Ho][Wo][nwords]
        uint16_t *count;           // [Ho][Wo]
        float2 *C;                 // [Ho][Wo][ntri(N)]
        unsigned long long *work;  // this stack's FP64 re-solve work area
        double cost;               // relative work, for the stream assignment
        int stream;
    };
    int device = -1;
    plk_window win{};
    plk::EmiParams prm{};
    int cov_precision = PLK_COV_FP32;
    std::vector<Stack> st;
    void *scratch = nullptr;
    cudaStream_t origin = nullptr;  // the stream the graph is recorded from
    cudaStream_t streams[kStreams] = {};
    cudaEvent_t fork = nullptr, join[kStreams] = {};
    cudaGraphExec_t exec = nullptr;
    int nodes = 0;
};

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

const plk::Schedule *find_tuned(const plk_ctx *ctx, int N, plk_window w) {
    for (int i = 0; i < ctx->n_tuned; ++i) {
        const auto &t = ctx->tuned[i];
        if (t.N == N && t.wy == w.wy && t.wx == w.wx && t.sy == w.sy && t.sx == w.sx) return &t.sch;
    }
    return nullptr;
}

// S1-S6 of one stack on stream s with schedule sch.
cudaError_t enqueue_stack(const plk_batch *b, const plk_batch::Stack &k, cudaStream_t s, const plk::Schedule *sch) {
    const int N = k.d.N;
    cudaError_t e =
        plk::launch_amp_stats(reinterpret_cast<const float2 *>(k.d.slc), N, k.npix, k.sum_pow, nullptr, 0, s);
    if (e != cudaSuccess) return e;
    e = plk::launch_shp(k.sum_pow, k.g, k.c, k.mask, k.count, s);
    if (e != cudaSuccess) return e;
    e = plk::launch_covariance(k.z, N, k.g, k.mask, k.C, s, b->cov_precision, sch);
    if (e != cudaSuccess) return e;
    plk::EmiParams prm = b->prm;
    prm.work = k.work;
    const plk::StackSource src{&k.z, &k.g, k.mask};
    return plk::launch_phase_link(k.C, N, k.nout, k.d.ref_idx, prm, k.d.phase, k.d.tcoh, nullptr, k.d.status, s,
                                  nullptr, &src, sch);
}

void release(plk_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (int i = 0; i < plk_batch::kStreams; ++i) {
        if (b->streams[i]) cudaStreamDestroy(b->streams[i]);
        if (b->join[i]) cudaEventDestroy(b->join[i]);
    }
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->scratch) cudaFree(b->scratch);
    delete b;
}

}  // namespace

extern "C" {

plk_status plk_batch_create(plk_ctx *ctx, const plk_stack_desc *stacks, int n_stacks, plk_window win,
                            const plk_params *params, plk_batch **out) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_batch_create: null ctx");
    if (!out || !stacks || n_stacks < 1 || !window_ok(win))
        return fail(ctx, PLK_EINVAL, "plk_batch_create: bad argument");
    *out = nullptr;
    plk::EmiParams prm;
    double alpha;
    int cov_precision = PLK_COV_FP32;
    plk_status ps = resolve_params(ctx, params, &prm, &alpha, &cov_precision);
    if (ps != PLK_OK) return ps;
    for (int i = 0; i < n_stacks; ++i) {
        const plk_stack_desc &d = stacks[i];
        if (!d.slc || d.N < 2 || d.N > PLK_MAX_N || d.H < 1 || d.W < 1 || d.ref_idx < 0 || d.ref_idx >= d.N)
            return fail(ctx, PLK_EINVAL, "plk_batch_create: stack %d: bad N, size or ref_idx", i);
        const long long nout = (long long)(d.H / win.sy) * (d.W / win.sx);
        if (nout > 0 && (!d.phase || !d.status))
            return fail(ctx, PLK_EINVAL, "plk_batch_create: stack %d: null output", i);
        if (!aligned(d.slc, 8) || !aligned(d.phase, 4) || !aligned(d.tcoh, 4))
            return fail(ctx, PLK_EINVAL, "plk_batch_create: stack %d: misaligned pointer", i);
        if (cov_precision != PLK_COV_FP32 && d.N > 32)
            return fail(ctx, PLK_EUNSUPPORTED, "plk_batch_create: stack %d: tensor-core coherence modes need N <= 32", i);
    }
    DeviceGuard dg(ctx->device);
    plk_batch *b = new (std::nothrow) plk_batch;
    if (!b) return fail(ctx, PLK_ENOMEM, "plk_batch_create: out of host memory");
    b->device = ctx->device;
    b->win = win;
    b->prm = prm;
    b->cov_precision = cov_precision;
    b->st.resize(n_stacks);
    size_t total = 0;
    const int nwords = plk_mask_words(win);
    for (int i = 0; i < n_stacks; ++i) {
        plk_batch::Stack &k = b->st[i];
        k.d = stacks[i];
        k.g = plk::make_geom(k.d.H, k.d.W, win);
        k.npix = (long long)k.d.H * k.d.W;
        k.nout = (long long)k.g.Ho * k.g.Wo;
        for (int t = 0; t < k.d.N; ++t) k.z.p[t] = reinterpret_cast<const float2 *>(k.d.slc) + (long long)t * k.npix;
        double c;
        plk_glrt_threshold(alpha, k.d.N, &c);
        k.c = (float)c;
        k.cost = (double)k.nout * ((double)k.d.N * k.d.N * win.wy * win.wx + (double)k.d.N * k.d.N * k.d.N);
        total += align256(k.npix * sizeof(float)) + align256(k.nout * nwords * sizeof(uint64_t)) +
                 align256(k.nout * sizeof(uint16_t)) + align256(k.nout * plk::ntri(k.d.N) * sizeof(float2)) + align256(plk::kEmiWorkBytes);
    }
    cudaError_t e = plk::dev_malloc((void **)&b->scratch, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        release(b);
        return fail(ctx, PLK_ENOMEM, "plk_batch_create: cannot allocate %zu bytes of scratch", total);
    }
    char *p = static_cast<char *>(b->scratch);
    for (auto &k : b->st) {
        k.sum_pow = reinterpret_cast<float *>(p);
        p += align256(k.npix * sizeof(float));
        k.mask = reinterpret_cast<uint64_t *>(p);
        p += align256(k.nout * nwords * sizeof(uint64_t));
        k.count = reinterpret_cast<uint16_t *>(p);
        p += align256(k.nout * sizeof(uint16_t));
        k.C = reinterpret_cast<float2 *>(p);
        p += align256(k.nout * plk::ntri(k.d.N) * sizeof(float2));
        k.work = reinterpret_cast<unsigned long long *>(p);
        p += align256(plk::kEmiWorkBytes);
    }
    // The graph's origin and branch streams (non-blocking: the legacy default
    // stream cannot be recorded from).
    e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
    for (int i = 0; i < plk_batch::kStreams && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        release(b);
        return cuda_fail(ctx, e, "plk_batch_create: streams");
    }
    // Stacks longest first, each to the least loaded branch.
    std::vector<int> order(n_stacks);
    for (int i = 0; i < n_stacks; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return b->st[x].cost > b->st[y].cost; });
    double load[plk_batch::kStreams] = {0};
    for (int i : order) {
        const int s = (int)(std::min_element(load, load + plk_batch::kStreams) - load);
        b->st[i].stream = s;
        load[s] += b->st[i].cost;
    }
    *out = b;
    return PLK_OK;
}

plk_status plk_batch_destroy(plk_batch *b) {
    if (!b) return PLK_OK;
    DeviceGuard dg(b->device);
    release(b);
    return PLK_OK;
}

plk_status plk_batch_info(const plk_batch *b, int *graph_built, int *streams, int *nodes) {
    if (!b) return fail(nullptr, PLK_EINVAL, "plk_batch_info: null batch");
    if (graph_built) *graph_built = b->exec ? 1 : 0;
    if (streams) *streams = plk_batch::kStreams;
    if (nodes) *nodes = b->nodes;
    return PLK_OK;
}

plk_status plk_tuned_schedule(const plk_ctx *ctx, int N, plk_window win, int *cov_tile_y, int *cov_tile_x,
                              int *emi_lanes) {
    if (!ctx || !cov_tile_y || !cov_tile_x || !emi_lanes)
        return fail(nullptr, PLK_EINVAL, "plk_tuned_schedule: null argument");
    const plk::Schedule *s = find_tuned(ctx, N, win);
    if (!s) return fail(const_cast<plk_ctx *>(ctx), PLK_EINVAL, "plk_tuned_schedule: (N, window) not tuned");
    *cov_tile_y = s->cov_TY;
    *cov_tile_x = s->cov_TX;
    *emi_lanes = s->emi_np;
    return PLK_OK;
}

}  // extern "C"

namespace {

// Time one launch sequence on stream s (after one untimed run), in ms.
template <class F>
float time_ms(cudaStream_t s, F &&f, cudaError_t &err) {
    cudaEvent_t e0, e1;
    if ((err = cudaEventCreate(&e0)) != cudaSuccess) return 0.f;
    if ((err = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return 0.f;
    }
    float ms = 0.f;
    err = f();
    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
    if (err == cudaSuccess) err = f();
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

// Tune the schedule of stack k's (N, window) on its own data: the coherence
// tile among the heuristic's three best candidates (single precision only),
// then the EMI lanes per pixel (the smallest group that holds a row, or the
// next wider one).
cudaError_t tune(plk_ctx *ctx, const plk_batch *b, const plk_batch::Stack &k, plk::Schedule &best) {
    cudaStream_t s = ctx->stream;
    const int N = k.d.N;
    cudaError_t e =
        plk::launch_amp_stats(reinterpret_cast<const float2 *>(k.d.slc), N, k.npix, k.sum_pow, nullptr, 0, s);
    if (e == cudaSuccess) e = plk::launch_shp(k.sum_pow, k.g, k.c, k.mask, k.count, s);
    if (e != cudaSuccess) return e;
    best = plk::Schedule{};
    if (b->cov_precision == PLK_COV_FP32) {
        int tiles[3][2];
        const int nc = plk::covariance_tile_candidates(N, k.g, tiles, 3);
        float best_ms = 1e30f;
        for (int i = 0; i < nc; ++i) {
            plk::Schedule c{};
            c.cov_TY = tiles[i][0];
            c.cov_TX = tiles[i][1];
            const float ms =
                time_ms(s, [&] { return plk::launch_covariance(k.z, N, k.g, k.mask, k.C, s, 0, &c); }, e);
            if (e != cudaSuccess) return e;
            if (ms < best_ms) {
                best_ms = ms;
                best.cov_TY = c.cov_TY;
                best.cov_TX = c.cov_TX;
            }
        }
    }
    e = plk::launch_covariance(k.z, N, k.g, k.mask, k.C, s, b->cov_precision, &best);
    if (e != cudaSuccess) return e;
    // EMI rows: the smallest that holds N, and the next wider.
    const int np0 = plk::emi_row_length(N);
    const int cands[2] = {np0, plk::emi_row_length(np0 + 1)};
    float best_ms = 1e30f;
    for (int ci = 0; ci < (np0 == 32 ? 1 : 2); ++ci) {
        const int np = cands[ci];
        plk::Schedule c = best;
        c.emi_np = np;
        plk::EmiParams prm = b->prm;
        prm.work = k.work;
        const plk::StackSource src{&k.z, &k.g, k.mask};
        const float ms = time_ms(
            s,
            [&] {
                return plk::launch_phase_link(k.C, N, k.nout, k.d.ref_idx, prm, k.d.phase, k.d.tcoh, nullptr,
                                              k.d.status, s, nullptr, &src, &c);
            },
            e);
        if (e != cudaSuccess) return e;
        if (ms < best_ms) {
            best_ms = ms;
            best.emi_np = np;
        }
    }
    return cudaSuccess;
}

// Record the batch: fork from the origin stream to the branch streams, each
// stack's S1-S6 on its branch, join back.  Recording runs nothing.
cudaError_t record(plk_ctx *ctx, plk_batch *b) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    cudaError_t ee = cudaEventRecord(b->fork, b->origin);
    for (int i = 0; i < plk_batch::kStreams && ee == cudaSuccess; ++i) ee = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
    for (const auto &k : b->st) {
        if (ee != cudaSuccess) break;
        if (k.nout == 0) continue;
        ee = enqueue_stack(b, k, b->streams[k.stream], find_tuned(ctx, k.d.N, b->win));
    }
    for (int i = 0; i < plk_batch::kStreams && ee == cudaSuccess; ++i) {
        ee = cudaEventRecord(b->join[i], b->streams[i]);
        if (ee == cudaSuccess) ee = cudaStreamWaitEvent(b->origin, b->join[i], 0);
    }
    e = cudaStreamEndCapture(b->origin, &graph);
    if (ee != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return ee != cudaSuccess ? ee : e;
    }
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    b->nodes = (int)nn;
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) b->exec = nullptr;
    return e;
}

}  // namespace

extern "C" {

plk_status plk_batch_run(plk_ctx *ctx, plk_batch *b) {
    if (!ctx) return fail(nullptr, PLK_EINVAL, "plk_batch_run: null ctx");
    if (!b) return fail(ctx, PLK_EINVAL, "plk_batch_run: null batch");
    if (b->device != ctx->device) return fail(ctx, PLK_EINVAL, "plk_batch_run: batch on another device");
    DeviceGuard dg(ctx->device);
    if (!b->exec) {
        for (const auto &k : b->st) {
            if (k.nout == 0 || find_tuned(ctx, k.d.N, b->win)) continue;
            plk::Schedule sch;
            cudaError_t e = tune(ctx, b, k, sch);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_batch_run: tuning");
            if (ctx->n_tuned < 64) {
                auto &t = ctx->tuned[ctx->n_tuned++];
                t.N = k.d.N;
                t.wy = b->win.wy;
                t.wx = b->win.wx;
                t.sy = b->win.sy;
                t.sx = b->win.sx;
                t.sch = sch;
            }
        }
        const cudaError_t e = record(ctx, b);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_batch_run: recording the graph");
    }
    const cudaError_t e = cudaGraphLaunch(b->exec, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plk_batch_run: graph launch");
    return PLK_OK;
}

}  // extern "C"
