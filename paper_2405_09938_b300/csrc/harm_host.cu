// Echo into host memory: the burst is computed in pulse blocks into a ring of two
// device buffers owned by the scene, and each block is copied to the caller's
// page-locked host array on a copy stream while the next block is computed
// (the raw-data output stage of Sec. IV-B: the GPU keeps computing while earlier
// parts of the echo leave it). Even blocks run on the scene's stream, odd blocks
// on a second compute stream, so that one block's last wave of CTAs overlaps the
// next block's first.
//
// Ordering (all on the device, no host waits inside the call), b = k mod 2,
// compute stream c[b] (c[0] = the scene's stream, c[1] = the second one, which
// first waits for everything ordered before the call on the scene's stream):
//   c[b]        : [wait free[b]] memset(ring[b]) accumulate(block k) record ready[b]
//   copy stream : wait ready[b]  copy ring[b] -> host block k    record free[b]
// At the end the scene stream waits for both free events (each copy follows its
// block's computation), so whatever the caller orders after the call on the scene
// stream (and harm_scene_sync) sees the host array complete.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "harm.h"
#include "harm_internal.cuh"
#include "harm_kernels.cuh"

namespace harm {
harm_status set_error(harm_status s, const char *msg);
int mixed_batch_pulses();
}

namespace {

constexpr int kDefaultBlocks = 8;

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

#define HCUDA(call, what)                                    \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
    } while (0)

// Pulses per block: the caller's choice, else about an eighth of the burst
// rounded up to whole generator windows, never more than the burst.
int block_size(int np, int block_pulses)
{
    if (block_pulses > 0) return std::min(block_pulses, np);
    // default blocks are whole time-Taylor windows of the mixed path, so that no
    // window's generator contraction runs twice
    const int q = harm::mixed_batch_pulses();
    const int b = (np + kDefaultBlocks - 1) / kDefaultBlocks;
    return std::min(np, std::max(q, (b + q - 1) / q * q));
}

// Streams, events and a ring large enough for `bytes` per buffer. A ring that
// must grow is freed only after the copies of earlier calls have finished.
harm_status ensure_ring(harm_scene *s, size_t bytes)
{
    if (!s->copy_stream) HCUDA(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking), "copy stream");
    if (!s->aux_stream) HCUDA(cudaStreamCreateWithFlags(&s->aux_stream, cudaStreamNonBlocking), "compute stream");
    if (!s->fork) HCUDA(cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming), "event");
    for (int b = 0; b < 2; ++b) {
        if (!s->ring_ready[b]) HCUDA(cudaEventCreateWithFlags(&s->ring_ready[b], cudaEventDisableTiming), "event");
        if (!s->ring_free[b]) HCUDA(cudaEventCreateWithFlags(&s->ring_free[b], cudaEventDisableTiming), "event");
    }
    if (s->ring_bytes >= bytes) return HARM_OK;
    HCUDA(cudaStreamSynchronize(s->copy_stream), "wait for earlier host copies");
    HCUDA(cudaStreamSynchronize(s->aux_stream), "wait for the second compute stream");
    HCUDA(cudaStreamSynchronize(s->stream), "wait for the scene stream");
    for (int b = 0; b < 2; ++b) {
        if (s->ring[b]) cudaFree(s->ring[b]);
        s->ring[b] = nullptr;
    }
    s->ring_bytes = 0;
    for (int b = 0; b < 2; ++b) HCUDA(cudaMalloc(&s->ring[b], bytes), "cudaMalloc host-output ring");
    s->ring_bytes = bytes;
    return HARM_OK;
}

// Blocks of the burst: compute on alternating streams, copy out on the copy stream.
harm_status enqueue_blocks(harm_scene *s, int32_t n0, int32_t np, void *iq_host, harm_dtype dtype, int B, size_t row)
{
    const int nc = s->desc.n_channels;
    const int nblocks = (np + B - 1) / B;
    const cudaStream_t cs[2] = {s->stream, s->aux_stream};
    if (nblocks > 1) {
        HCUDA(cudaEventRecord(s->fork, s->stream), "record fork");
        HCUDA(cudaStreamWaitEvent(s->aux_stream, s->fork, 0), "second compute stream wait");
    }
    for (int k = 0; k < nblocks; ++k) {
        const int b = k & 1;
        const int p0 = k * B, pb = std::min(B, np - p0);
        if (k >= 2) HCUDA(cudaStreamWaitEvent(cs[b], s->ring_free[b], 0), "wait for the ring buffer");
        HCUDA(cudaMemsetAsync(s->ring[b], 0, (size_t)nc * pb * row, cs[b]), "clear ring buffer");
        cudaError_t e = harm::launch_accumulate_on(s, cs[b], n0 + p0, pb, s->ring[b], dtype);
        if (e != cudaSuccess) return cuda_fail(e, "echo accumulator launch");
        HCUDA(cudaEventRecord(s->ring_ready[b], cs[b]), "record block ready");
        HCUDA(cudaStreamWaitEvent(s->copy_stream, s->ring_ready[b], 0), "copy stream wait");
        // block k of every channel: nc rows of pb pulses, strided np pulses apart in iq_host
        HCUDA(cudaMemcpy2DAsync((char *)iq_host + (size_t)p0 * row, (size_t)np * row, s->ring[b], (size_t)pb * row,
                                (size_t)pb * row, nc, cudaMemcpyDeviceToHost, s->copy_stream),
              "copy block to host");
        HCUDA(cudaEventRecord(s->ring_free[b], s->copy_stream), "record block copied");
    }
    return HARM_OK;
}

}  // namespace

namespace harm {

void release_host_ring(harm_scene *s)
{
    if (s->aux_stream) cudaStreamSynchronize(s->aux_stream);
    if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
    for (int b = 0; b < 2; ++b) {
        if (s->ring[b]) cudaFree(s->ring[b]);
        if (s->ring_ready[b]) cudaEventDestroy(s->ring_ready[b]);
        if (s->ring_free[b]) cudaEventDestroy(s->ring_free[b]);
        s->ring[b] = nullptr;
        s->ring_ready[b] = s->ring_free[b] = nullptr;
    }
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->aux_stream) cudaStreamDestroy(s->aux_stream);
    if (s->fork) cudaEventDestroy(s->fork);
    s->copy_stream = s->aux_stream = nullptr;
    s->fork = nullptr;
    s->ring_bytes = 0;
}

}  // namespace harm

extern "C" harm_status harm_echo_accumulate_host(harm_scene *s, int32_t n0, int32_t np, void *iq_host,
                                                 harm_dtype dtype, int32_t block_pulses)
{
    if (!s) return fail(HARM_E_INVALID, "scene is NULL");
    if (np < 0 || n0 < 0 || (int64_t)n0 + np > s->desc.n_pulses)
        return fail(HARM_E_INVALID, "pulse window [%d, %d) outside [0, %d)", n0, n0 + np, s->desc.n_pulses);
    if (dtype != HARM_C64 && dtype != HARM_C128) return fail(HARM_E_INVALID, "unknown dtype %d", (int)dtype);
    if (s->dev.det && dtype != HARM_C128)
        return fail(HARM_E_UNSUPPORTED, "deterministic sums need complex128 output");
    int dev = -1;
    HCUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != s->device) return fail(HARM_E_INVALID, "scene lives on device %d, current device is %d", s->device, dev);
    if (np == 0) return HARM_OK;
    if (!iq_host) return fail(HARM_E_INVALID, "iq_host is NULL");
    cudaPointerAttributes a;
    HCUDA(cudaPointerGetAttributes(&a, iq_host), "cudaPointerGetAttributes");
    if (a.type != cudaMemoryTypeHost)
        return fail(HARM_E_INVALID, "iq_host is not page-locked host memory (use cudaHostAlloc or cudaHostRegister)");

    const int nc = s->desc.n_channels, nr = s->desc.n_range;
    const size_t elem = dtype == HARM_C64 ? 8 : 16;
    const int B = block_size(np, block_pulses);
    const size_t row = (size_t)nr * elem;  // bytes of one pulse of one channel
    harm_status st = ensure_ring(s, (size_t)nc * B * row);
    if (st != HARM_OK) return st;

    const harm_status qs = enqueue_blocks(s, n0, np, iq_host, dtype, B, row);
    // join the second compute stream and the copy stream back into the scene's
    // stream, also after a failed launch, so that harm_scene_sync covers them
    cudaError_t e = cudaEventRecord(s->fork, s->aux_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->fork, 0);
    if (e == cudaSuccess) e = cudaEventRecord(s->fork, s->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->fork, 0);
    if (qs != HARM_OK) return qs;
    if (e != cudaSuccess) return cuda_fail(e, "join the host-output streams");
    return HARM_OK;
}
