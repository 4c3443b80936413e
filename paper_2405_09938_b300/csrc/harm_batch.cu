// Batched scenes: work list, project-written autotuner of the launch shape (tile
// height and time-Taylor window per scene-size class, CTAs per SM for the
// launch), and CUDA-graph capture / replay of the persistent batched launch.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "harm.h"
#include "harm_internal.cuh"
#include "harm_kernels.cuh"

namespace harm {
harm_status set_error(harm_status s, const char *msg);
}

struct harm_batch {
    std::vector<harm_scene *> scenes;
    cudaStream_t user = nullptr;     // the first scene's stream (ordering of run())
    cudaStream_t stream = nullptr;   // the batch's own stream (graph capture needs a non-default stream)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int device = 0;
    int nc = 0, taps = 8;
    int variant = 0;
    int share3 = 0;
    int ctas = 0;
    int sms = 0;                // SMs of the device
    int ctas_per_sm = 2;
    std::vector<int> ty;        // tile rows by scene
    std::vector<int> win;       // pulses per work item by scene (time-Taylor window)
    std::vector<int> order;     // processing order (largest first)
    std::vector<void *> allocs;
    void *d_args = nullptr;
    int *d_start = nullptr, *d_tiles = nullptr, *d_ty = nullptr, *d_order = nullptr;
    float **d_iq = nullptr;
    unsigned int *d_counter = nullptr;
    int total = 0;
    // graph state
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void *> graph_iq;
    int graph_zero = -1;
};

namespace {

harm_status fail(harm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return harm::set_error(s, buf);
}

harm_status cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? HARM_E_OOM : HARM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define BCUDA(call, what)                                    \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
    } while (0)

double scene_cost(const harm_scene *s)
{
    return (double)s->desc.nx * s->desc.ny * s->desc.n_pulses * s->desc.n_channels;
}

// Size class used by the autotuner: facet count below 1e6, below 4e6, above.
int size_class(const harm_scene *s)
{
    double nf = (double)s->desc.nx * s->desc.ny;
    return nf < 1e6 ? 0 : (nf < 4e6 ? 1 : 2);
}

// Choices of the autotuner, kept for the life of the process: per (device,
// per-pulse code variant, channel count, taps, channel layout, size class) the
// tile height and window; per (the same without the class, plus the classes
// present) the CTAs per SM of the launch.
struct TuneKey {
    int device, variant, nc, taps, share3, cls;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(device, variant, nc, taps, share3, cls) <
               std::tie(o.device, o.variant, o.nc, o.taps, o.share3, o.cls);
    }
};
struct ClassChoice {
    int ty, win;
};
std::mutex g_tune_mutex;
std::map<TuneKey, ClassChoice> g_class_choice;
std::map<TuneKey, int> g_ctas_choice;  // cls = bit mask of the classes present

template <typename T>
harm_status dalloc(harm_batch *b, T **p, size_t count)
{
    void *q = nullptr;
    BCUDA(cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)), "cudaMalloc batch");
    b->allocs.push_back(q);
    *p = (T *)q;
    return HARM_OK;
}

// Work list for the current tile heights and windows, limited to the work items
// that cover the first max_pulses pulses of each scene (max_pulses <= 0: all),
// restricted to scenes with use[s] set. Uploads start / tiles / ty / order.
harm_status plan(harm_batch *b, int max_pulses, const std::vector<char> &use, int *total)
{
    const int n = (int)b->scenes.size();
    std::vector<int> start(n + 1, 0), tiles(n, 0);
    for (int s = 0; s < n; ++s) tiles[s] = harm::batch_tiles(b->scenes[s], b->ty[s]);
    for (int k = 0; k < n; ++k) {
        int s = b->order[k];
        const harm_scene *sc = b->scenes[s];
        int nb = harm::batch_windows(sc, b->win[s]);
        if (max_pulses > 0) nb = std::min(nb, (max_pulses + b->win[s] - 1) / b->win[s]);
        long long items = use[s] ? (long long)tiles[s] * nb : 0;
        if ((long long)start[k] + items > 0x7fffffffll) return fail(HARM_E_INVALID, "batch has more than 2^31 work items");
        start[k + 1] = start[k] + (int)items;
    }
    *total = start[n];
    BCUDA(cudaMemcpyAsync(b->d_start, start.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, b->stream), "upload");
    BCUDA(cudaMemcpyAsync(b->d_tiles, tiles.data(), n * sizeof(int), cudaMemcpyHostToDevice, b->stream), "upload");
    BCUDA(cudaMemcpyAsync(b->d_ty, b->ty.data(), n * sizeof(int), cudaMemcpyHostToDevice, b->stream), "upload");
    BCUDA(cudaStreamSynchronize(b->stream), "upload");
    return HARM_OK;
}

harm::BatchLaunch launch_desc(harm_batch *b, int total)
{
    harm::BatchLaunch L;
    L.args = b->d_args;
    L.start = b->d_start;
    L.tiles = b->d_tiles;
    L.ty = b->d_ty;
    L.order = b->d_order;
    L.iq = b->d_iq;
    L.counter = b->d_counter;
    L.poly = &b->scenes[0]->mixed;
    L.n = (int)b->scenes.size();
    L.total = total;
    L.nc = b->nc;
    L.taps = b->taps;
    L.ctas = b->ctas_per_sm * b->sms;
    L.variant = b->variant;
    L.share3 = b->share3;
    return L;
}

size_t iq_bytes(const harm_scene *s)
{
    return (size_t)s->desc.n_channels * s->desc.n_pulses * s->desc.n_range * 8;
}

harm_status set_outputs(harm_batch *b, void *const *iq)
{
    if (!iq) return fail(HARM_E_INVALID, "iq_dev is NULL");
    const int n = (int)b->scenes.size();
    for (int s = 0; s < n; ++s) {
        if (!iq[s]) return fail(HARM_E_INVALID, "iq_dev[%d] is NULL", s);
        char what[32];
        snprintf(what, sizeof(what), "iq_dev[%d]", s);
        harm_status st = harm::check_device_span(iq[s], iq_bytes(b->scenes[s]), what);
        if (st != HARM_OK) return st;
    }
    BCUDA(cudaMemcpyAsync(b->d_iq, iq, n * sizeof(void *), cudaMemcpyHostToDevice, b->stream), "upload outputs");
    BCUDA(cudaStreamSynchronize(b->stream), "upload outputs");
    return HARM_OK;
}

// Scenes whose window changes get their launch arguments rebuilt and uploaded.
harm_status set_windows(harm_batch *b, const std::vector<int> &win)
{
    const size_t ab = harm::batch_args_bytes();
    std::vector<unsigned char> tmp(ab);
    for (size_t s = 0; s < b->scenes.size(); ++s) {
        if (win[s] == b->win[s]) continue;
        b->win[s] = win[s];
        harm::batch_fill_args(b->scenes[s], tmp.data(), win[s]);
        BCUDA(cudaMemcpyAsync((unsigned char *)b->d_args + ab * s, tmp.data(), ab, cudaMemcpyHostToDevice, b->stream),
              "upload scene arguments");
        BCUDA(cudaStreamSynchronize(b->stream), "upload scene arguments");
    }
    return HARM_OK;
}

// Median device time of `reps` launches (after one untimed) over the work items
// of the first max_pulses pulses of the scenes in `use`.
harm_status time_sample(harm_batch *b, int max_pulses, const std::vector<char> &use, int reps, cudaEvent_t e0,
                        cudaEvent_t e1, float *ms_out)
{
    int total = 0;
    harm_status st = plan(b, max_pulses, use, &total);
    if (st != HARM_OK) return st;
    std::vector<float> ms;
    for (int rep = 0; rep <= reps; ++rep) {
        BCUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), b->stream), "memset");
        BCUDA(cudaEventRecord(e0, b->stream), "event");
        BCUDA(harm::batch_launch(launch_desc(b, total), b->stream), "batched launch");
        BCUDA(cudaEventRecord(e1, b->stream), "event");
        BCUDA(cudaEventSynchronize(e1), "event");
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0) ms.push_back(t);
    }
    std::sort(ms.begin(), ms.end());
    *ms_out = ms[ms.size() / 2];
    return HARM_OK;
}

void drop_graph(harm_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_iq.clear();
    b->graph_zero = -1;
}

}  // namespace

extern "C" {

harm_status harm_batch_create(harm_scene *const *scenes, int32_t n, harm_batch **out)
{
    if (!out) return fail(HARM_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!scenes || n < 1) return fail(HARM_E_INVALID, "need at least one scene");
    for (int s = 0; s < n; ++s) {
        const harm_scene *sc = scenes[s];
        if (!sc) return fail(HARM_E_INVALID, "scene %d is NULL", s);
        if (sc->desc.precision != HARM_PREC_MIXED) return fail(HARM_E_UNSUPPORTED, "scene %d is not mixed precision", s);
        if (sc->device != scenes[0]->device) return fail(HARM_E_INVALID, "scenes on different devices");
        if (sc->desc.n_channels != scenes[0]->desc.n_channels)
            return fail(HARM_E_INVALID, "scenes must have the same number of channels");
        if (sc->desc.taps != scenes[0]->desc.taps || sc->desc.kaiser_beta != scenes[0]->desc.kaiser_beta)
            return fail(HARM_E_INVALID, "scenes must share taps and kaiser_beta");
        if (harm::batch_variant(sc) != harm::batch_variant(scenes[0]))
            return fail(HARM_E_INVALID, "scenes must share the surface model (CWM) and the pattern kind (u-v grids)");
    }
    harm_batch *b = new (std::nothrow) harm_batch;
    if (!b) return fail(HARM_E_OOM, "host allocation failed");
    b->scenes.assign(scenes, scenes + n);
    b->user = scenes[0]->stream;
    b->device = scenes[0]->device;
    {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            harm_batch_destroy(b);
            return cuda_fail(e, "batch stream");
        }
    }
    b->nc = scenes[0]->desc.n_channels;
    b->taps = scenes[0]->desc.taps;
    b->variant = harm::batch_variant(scenes[0]);
    b->share3 = 1;
    for (int s = 0; s < n; ++s)
        if (!harm::batch_share3(scenes[s])) b->share3 = 0;
    b->ctas = harm::batch_ctas(b->device, b->variant);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    b->ctas_per_sm = b->sms > 0 ? std::max(1, b->ctas / b->sms) : 2;
    b->ty.assign(n, 16);
    b->win.resize(n);
    for (int s = 0; s < n; ++s) b->win[s] = scenes[s]->mixed.nb;
    b->order.resize(n);
    for (int s = 0; s < n; ++s) b->order[s] = s;
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int a, int c) { return scene_cost(b->scenes[a]) > scene_cost(b->scenes[c]); });
    harm_status st;
    size_t ab = harm::batch_args_bytes();
    std::vector<unsigned char> args(ab * n);
    for (int s = 0; s < n; ++s) harm::batch_fill_args(b->scenes[s], args.data() + ab * s, b->win[s]);
    unsigned char *d_args = nullptr;
    if ((st = dalloc(b, &d_args, args.size())) != HARM_OK ||
        (st = dalloc(b, &b->d_start, n + 1)) != HARM_OK || (st = dalloc(b, &b->d_tiles, n)) != HARM_OK ||
        (st = dalloc(b, &b->d_ty, n)) != HARM_OK || (st = dalloc(b, &b->d_order, n)) != HARM_OK ||
        (st = dalloc(b, &b->d_iq, n)) != HARM_OK || (st = dalloc(b, &b->d_counter, 1)) != HARM_OK) {
        harm_batch_destroy(b);
        return st;
    }
    b->d_args = d_args;
    cudaError_t e = cudaMemcpy(d_args, args.data(), args.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_order, b->order.data(), n * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        harm_batch_destroy(b);
        return cuda_fail(e, "upload batch");
    }
    std::vector<char> all(n, 1);
    if ((st = plan(b, 0, all, &b->total)) != HARM_OK) {
        harm_batch_destroy(b);
        return st;
    }
    *out = b;
    return HARM_OK;
}

harm_status harm_batch_tile_rows(const harm_batch *b, int32_t *rows)
{
    if (!b || !rows) return fail(HARM_E_INVALID, "NULL argument");
    for (size_t s = 0; s < b->scenes.size(); ++s) rows[s] = b->ty[s];
    return HARM_OK;
}

harm_status harm_batch_set_tile_rows(harm_batch *b, const int32_t *rows)
{
    if (!b || !rows) return fail(HARM_E_INVALID, "NULL argument");
    const int n = (int)b->scenes.size();
    for (int s = 0; s < n; ++s)
        if (rows[s] != 8 && rows[s] != 16) return fail(HARM_E_INVALID, "tile rows of scene %d: %d (8 or 16)", s, rows[s]);
    BCUDA(cudaStreamSynchronize(b->stream), "sync");
    drop_graph(b);
    for (int s = 0; s < n; ++s) b->ty[s] = rows[s];
    std::vector<char> all(n, 1);
    return plan(b, 0, all, &b->total);
}

harm_status harm_batch_tune(harm_batch *b, void *const *iq)
{
    if (!b) return fail(HARM_E_INVALID, "batch is NULL");
    BCUDA(cudaStreamSynchronize(b->user), "sync");
    harm_status st = set_outputs(b, iq);
    if (st != HARM_OK) return st;
    drop_graph(b);
    const int n = (int)b->scenes.size();
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCUDA(cudaEventCreate(&e0), "event");
    BCUDA(cudaEventCreate(&e1), "event");
    // the sample a candidate is timed on: the first kSamplePulses pulses of the
    // class's largest scenes, as many as give at least kSampleWaves waves of work
    // items to the persistent launch (a sample that does not fill the GPU favours
    // shapes with more, smaller items)
    const int kSamplePulses = 256, kSampleWaves = 8, kReps = 3;
    // a candidate replaces the default shape (timed first) only when it is faster by
    // more than this margin: smaller differences on the sample are within its
    // run-to-run spread and do not carry over to the whole batch
    const float kMargin = 0.98f;
    std::vector<char> sample_all(n, 0);
    int class_mask = 0;
    for (int cls = 0; cls < 3 && st == HARM_OK; ++cls) {
        std::vector<int> members;
        for (int k = 0; k < n; ++k)
            if (size_class(b->scenes[b->order[k]]) == cls) members.push_back(b->order[k]);  // largest first
        if (members.empty()) continue;
        class_mask |= 1 << cls;
        std::vector<char> use(n, 0);
        long long items = 0;
        const long long want = (long long)kSampleWaves * b->ctas_per_sm * b->sms;
        for (int i = 0; i < (int)members.size() && items < want; ++i) {
            const harm_scene *sc = b->scenes[members[i]];
            use[members[i]] = sample_all[members[i]] = 1;
            items += (long long)harm::batch_tiles(sc, 16) * ((kSamplePulses + sc->mixed.nb - 1) / sc->mixed.nb);
        }
        const TuneKey key{b->device, b->variant, b->nc, b->taps, b->share3, cls};
        ClassChoice best{16, b->scenes[members[0]]->mixed.nb};
        auto it = g_class_choice.find(key);
        if (it != g_class_choice.end()) {
            best = it->second;
        } else {
            float best_ms = 1e30f;
            const int rows[2] = {16, 8};
            const int wins[2] = {b->scenes[members[0]]->mixed.nb, b->scenes[members[0]]->mixed.alt_nb};
            for (int r = 0; r < 2 && st == HARM_OK; ++r)
                for (int w = 0; w < 2 && st == HARM_OK; ++w) {
                    const bool is_default = r == 0 && w == 0;
                    std::vector<int> win = b->win;
                    for (int m : members) {
                        b->ty[m] = rows[r];
                        win[m] = wins[w];
                    }
                    float ms = 0.0f;
                    if ((st = set_windows(b, win)) != HARM_OK) break;
                    if ((st = time_sample(b, kSamplePulses, use, kReps, e0, e1, &ms)) != HARM_OK) break;
                    if (is_default || ms < kMargin * best_ms) {
                        best_ms = ms;
                        best = ClassChoice{rows[r], wins[w]};
                    }
                }
            if (st == HARM_OK) g_class_choice[key] = best;
        }
        std::vector<int> win = b->win;
        for (int m : members) {
            b->ty[m] = best.ty;
            win[m] = best.win;
        }
        if (st == HARM_OK) st = set_windows(b, win);
    }
    // CTAs per SM of the launch, timed on the samples of every class together
    if (st == HARM_OK) {
        const TuneKey key{b->device, b->variant, b->nc, b->taps, b->share3, 8 + class_mask};
        auto it = g_ctas_choice.find(key);
        if (it != g_ctas_choice.end()) {
            b->ctas_per_sm = it->second;
        } else {
            const int most = (b->variant & 1) ? 1 : 2;  // the Choppy Wave Model's registers allow one CTA per SM
            float best_ms = 1e30f;
            int best_c = most;
            for (int c = most; c >= 1 && st == HARM_OK; --c) {
                b->ctas_per_sm = c;
                float ms = 0.0f;
                if ((st = time_sample(b, kSamplePulses, sample_all, kReps, e0, e1, &ms)) != HARM_OK) break;
                if (c == most || ms < kMargin * best_ms) {
                    best_ms = ms;
                    best_c = c;
                }
            }
            b->ctas_per_sm = best_c;
            if (st == HARM_OK) g_ctas_choice[key] = best_c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HARM_OK) return st;
    std::vector<char> all(n, 1);
    return plan(b, 0, all, &b->total);
}

harm_status harm_batch_config(const harm_batch *b, int32_t *rows, int32_t *windows, int32_t *ctas_per_sm)
{
    if (!b) return fail(HARM_E_INVALID, "batch is NULL");
    for (size_t s = 0; s < b->scenes.size(); ++s) {
        if (rows) rows[s] = b->ty[s];
        if (windows) windows[s] = b->win[s];
    }
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
    return HARM_OK;
}

harm_status harm_batch_set_config(harm_batch *b, const int32_t *rows, const int32_t *windows, int32_t ctas_per_sm)
{
    if (!b || !rows || !windows) return fail(HARM_E_INVALID, "NULL argument");
    const int n = (int)b->scenes.size();
    for (int s = 0; s < n; ++s) {
        if (rows[s] != 8 && rows[s] != 16) return fail(HARM_E_INVALID, "tile rows of scene %d: %d (8 or 16)", s, rows[s]);
        const harm::MixedTables &M = b->scenes[s]->mixed;
        if (windows[s] != M.nb && windows[s] != M.alt_nb)
            return fail(HARM_E_INVALID, "window of scene %d: %d (%d or %d pulses)", s, windows[s], M.nb, M.alt_nb);
    }
    const int most = (b->variant & 1) ? 1 : 2;
    if (ctas_per_sm < 1 || ctas_per_sm > most)
        return fail(HARM_E_INVALID, "ctas_per_sm %d (1 .. %d for this batch)", ctas_per_sm, most);
    BCUDA(cudaStreamSynchronize(b->stream), "sync");
    drop_graph(b);
    for (int s = 0; s < n; ++s) b->ty[s] = rows[s];
    std::vector<int> win(windows, windows + n);
    harm_status st = set_windows(b, win);
    if (st != HARM_OK) return st;
    b->ctas_per_sm = ctas_per_sm;
    std::vector<char> all(n, 1);
    return plan(b, 0, all, &b->total);
}

harm_status harm_batch_run(harm_batch *b, void *const *iq, int32_t zero_first)
{
    if (!b) return fail(HARM_E_INVALID, "batch is NULL");
    if (!iq) return fail(HARM_E_INVALID, "iq_dev is NULL");
    const int n = (int)b->scenes.size();
    bool same = b->exec && b->graph_zero == (zero_first ? 1 : 0) && (int)b->graph_iq.size() == n;
    for (int s = 0; same && s < n; ++s) same = b->graph_iq[s] == iq[s];
    if (!same) {
        drop_graph(b);
        harm_status st = set_outputs(b, iq);
        if (st != HARM_OK) return st;
        BCUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e = cudaSuccess;
        if (zero_first)
            for (int s = 0; s < n && e == cudaSuccess; ++s) e = cudaMemsetAsync(iq[s], 0, iq_bytes(b->scenes[s]), b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), b->stream);
        if (e == cudaSuccess) e = harm::batch_launch(launch_desc(b, b->total), b->stream);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(e != cudaSuccess ? e : e2, "capture batched launch");
        }
        b->graph = g;
        BCUDA(cudaGraphInstantiate(&b->exec, g, 0), "instantiate graph");
        b->graph_iq.assign(iq, iq + n);
        b->graph_zero = zero_first ? 1 : 0;
    }
    BCUDA(cudaEventRecord(b->ev_in, b->user), "event");
    BCUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0), "stream wait");
    BCUDA(cudaGraphLaunch(b->exec, b->stream), "graph launch");
    BCUDA(cudaEventRecord(b->ev_out, b->stream), "event");
    BCUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0), "stream wait");
    return HARM_OK;
}

harm_status harm_batch_destroy(harm_batch *b)
{
    if (!b) return HARM_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (void *p : b->allocs) cudaFree(p);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return HARM_OK;
}

}  // extern "C"
