// Allocation-free variant of the batched forward launch.
//
// Some callers cannot allocate device memory at the point where they run the echo:
// an ingest loop with a fixed, pre-planned device-memory budget, or code running
// inside a framework whose caching allocator owns the whole device (cudaMalloc and
// cudaFree can synchronise the device and can fail under memory pressure). For
// them, harm_batch_run_noalloc runs the same persistent batched launch as
// harm_batch_run, but keeps the launch's scratch memory (per-scene arguments,
// work list, output pointer table and the work counter) in one file-scope device
// array of fixed size instead of buffers from cudaMalloc. Scenes and outputs are
// still passed in by the caller.
#include <cstddef>
#include <cstring>
#include <mutex>

#include "harm.h"
#include "harm_internal.cuh"
#include "harm_kernels.cuh"

namespace harm {
harm_status set_error(harm_status s, const char *msg);
}

namespace {

constexpr int kMaxScenes = 64;       // scenes per call
constexpr int kArgsBytes = 2048;     // bytes reserved per scene argument block
constexpr int kMaxDevices = 64;

// Layout of the scratch image (host copy uploaded in one transfer per call): the
// small tables first and the per-scene argument blocks last, so that a call
// uploads only the tables and the blocks of its own scenes.
struct ScratchImage {
    int start[kMaxScenes + 1];
    int tiles[kMaxScenes];
    int ty[kMaxScenes];
    int order[kMaxScenes];
    float *iq[kMaxScenes];
    unsigned int counter;
    alignas(16) unsigned char args[kMaxScenes * kArgsBytes];
};

// The scratch memory: every GPU that loads the library holds one copy until the
// process exits. Host code must not use this name as a device address; the
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(ScratchImage)];

std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};
ScratchImage g_host_image;  // host staging copy, guarded by g_mutex

harm_status fail(harm_status s, const char *msg) { return harm::set_error(s, msg); }

// Device address of the scratch array on `device` (which must be current),
// looked up once per device.
harm_status scratch_address(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices) return fail(HARM_E_INVALID, "device index out of range");
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(HARM_E_CUDA, "cudaGetSymbolAddress of the no-alloc scratch array failed");
        }
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return HARM_OK;
}

}  // namespace

extern "C" harm_status harm_batch_run_noalloc(harm_scene *const *scenes, int32_t n, void *const *iq_dev,
                                              int32_t zero_first)
{
    if (!scenes || !iq_dev) return fail(HARM_E_INVALID, "scenes and iq_dev must not be NULL");
    if (n < 1) return fail(HARM_E_INVALID, "need at least one scene");
    if (n > kMaxScenes) return fail(HARM_E_INVALID, "harm_batch_run_noalloc takes at most 64 scenes per call");
    if (harm::batch_args_bytes() > (size_t)kArgsBytes)
        return fail(HARM_E_INVALID, "scene argument block larger than the no-alloc scratch slot");
    for (int s = 0; s < n; ++s) {
        const harm_scene *sc = scenes[s];
        if (!sc) return fail(HARM_E_INVALID, "a scene is NULL");
        if (!iq_dev[s]) return fail(HARM_E_INVALID, "an output pointer is NULL");
        if (sc->desc.precision != HARM_PREC_MIXED) return fail(HARM_E_UNSUPPORTED, "scenes must be mixed precision");
        if (sc->device != scenes[0]->device) return fail(HARM_E_INVALID, "scenes on different devices");
        if (sc->desc.n_channels != scenes[0]->desc.n_channels)
            return fail(HARM_E_INVALID, "scenes must have the same number of channels");
        if (sc->desc.taps != scenes[0]->desc.taps || sc->desc.kaiser_beta != scenes[0]->desc.kaiser_beta)
            return fail(HARM_E_INVALID, "scenes must share taps and kaiser_beta");
        if (harm::batch_variant(sc) != harm::batch_variant(scenes[0]))
            return fail(HARM_E_INVALID, "scenes must share the surface model (CWM) and the pattern kind (u-v grids)");
        const size_t bytes = (size_t)sc->desc.n_channels * sc->desc.n_pulses * sc->desc.n_range * 8;
        harm_status st = harm::check_device_span(iq_dev[s], bytes, "an output buffer");
        if (st != HARM_OK) return st;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != scenes[0]->device)
        return fail(HARM_E_INVALID, "the scenes' device must be current");

    std::lock_guard<std::mutex> lock(g_mutex);
    void *base = nullptr;
    harm_status st = scratch_address(dev, &base);
    if (st != HARM_OK) return st;

    // Work list: 16-row tiles, scenes largest first.
    ScratchImage &h = g_host_image;
    const size_t ab = harm::batch_args_bytes();
    double cost[kMaxScenes];
    for (int s = 0; s < n; ++s) {
        const harm_scene *sc = scenes[s];
        harm::batch_fill_args(sc, h.args + (size_t)s * ab, sc->mixed.nb);  // the kernel strides by the block size
        h.ty[s] = 16;
        h.tiles[s] = harm::batch_tiles(sc, 16);
        h.iq[s] = (float *)iq_dev[s];
        h.order[s] = s;
        cost[s] = (double)sc->desc.nx * sc->desc.ny * sc->desc.n_pulses;
    }
    for (int i = 1; i < n; ++i)  // insertion sort by cost, descending, stable
        for (int j = i; j > 0 && cost[h.order[j]] > cost[h.order[j - 1]]; --j) {
            int t = h.order[j];
            h.order[j] = h.order[j - 1];
            h.order[j - 1] = t;
        }
    h.start[0] = 0;
    for (int k = 0; k < n; ++k) {
        const harm_scene *sc = scenes[h.order[k]];
        long long items = (long long)h.tiles[h.order[k]] * sc->mixed.n_batches;
        if ((long long)h.start[k] + items > 0x7fffffffll) return fail(HARM_E_INVALID, "more than 2^31 work items");
        h.start[k + 1] = h.start[k] + (int)items;
    }
    h.counter = 0u;  // the work counter must start at zero on every call

    cudaStream_t stream = scenes[0]->stream;
    const size_t used = offsetof(ScratchImage, args) + (size_t)n * ab;
    cudaError_t e = cudaMemcpyAsync(base, &h, used, cudaMemcpyHostToDevice, stream);
    for (int s = 0; e == cudaSuccess && zero_first && s < n; ++s) {
        const harm_scene *sc = scenes[s];
        e = cudaMemsetAsync(iq_dev[s], 0, (size_t)sc->desc.n_channels * sc->desc.n_pulses * sc->desc.n_range * 8,
                            stream);
    }
    if (e == cudaSuccess) {
        ScratchImage *d = reinterpret_cast<ScratchImage *>(base);
        harm::BatchLaunch L;
        L.args = d->args;
        L.start = d->start;
        L.tiles = d->tiles;
        L.ty = d->ty;
        L.order = d->order;
        L.iq = d->iq;
        L.counter = &d->counter;
        L.poly = &scenes[0]->mixed;
        L.n = n;
        L.total = h.start[n];
        L.nc = scenes[0]->desc.n_channels;
        L.taps = scenes[0]->desc.taps;
        L.variant = harm::batch_variant(scenes[0]);
        L.share3 = 1;
        for (int s = 0; s < n; ++s)
            if (!harm::batch_share3(scenes[s])) L.share3 = 0;
        L.ctas = harm::batch_ctas(dev, L.variant);
        e = harm::batch_launch(L, stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HARM_E_CUDA, cudaGetErrorString(e));
    }
    return HARM_OK;
}
