// Internal interface between the host core and the kernel translation units.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "harm.h"
#include "harm_internal.cuh"

namespace harm {

// Mixed-precision path tables (FP32 separable waves and the Taylor-in-time
// tables of each pulse batch, plus the tap polynomials).
constexpr int kTapDeg = 7;      // degree of each tap polynomial in t = 2f - 1 (fit error 9e-7)
constexpr int kSincDeg = 7;     // degree of the sinc^2 polynomial in t = 2x^2 - 1, |x| <= 1
constexpr int kOrders = 6;      // Taylor orders in time: tau^0 .. tau^5

struct MixedTables {
    int nb = 0;             // pulses per batch (time-Taylor expansion window)
    int n_batches = 0;
    int nf = 3;             // state fields: 3 (linear surface) or 8 (Choppy Wave Model)
    int tile_x = 32, tile_y = 16;
    const float2 *ex = nullptr;   // [n_sets][nw][nx]  e^{i kx x}
    const float2 *ey = nullptr;   // [n_sets][nw][ny]  a e^{i phi} e^{i ky y}
    const float2 *tc = nullptr;   // [n_batches][n_sets][nw] e^{-i omega t_c} at the batch centre
    const float *cr = nullptr;    // [n_sets][nw][nf][kOrders] signed real Taylor coefficients
    const float *tau = nullptr;   // [np_total] t_s(n) - t_centre(batch)
    // the same time tables for windows of half the length (alt_nb pulses), which the
    // batched launch's autotuner may pick per scene-size class
    int alt_nb = 0, alt_n_batches = 0;
    const float2 *alt_tc = nullptr;  // [alt_n_batches][n_sets][nw]
    const float *alt_tau = nullptr;  // [np_total]
    float tap[8][kTapDeg + 1];    // Kaiser-sinc tap h(j - f), j = -3..4, monomials in t
    float sinc2[kSincDeg + 1];    // sinc^2(x) for |x| <= 1, monomials in t = 2 x^2 - 1
};

}  // namespace harm

struct harm_scene {
    harm_scene_desc desc{};
    std::vector<harm_antenna> rx;
    std::vector<double> het_u10, het_dir;  // corner spectra of a heterogeneous sea state
    std::vector<harm::PatLut> luts;        // [1 + nc] u-v gain grids (host copy of the descriptors)
    std::vector<void *> lut_mem;           // [1 + nc] device memory of each grid (or null)
    harm::PatLut *luts_dev = nullptr;      // [1 + nc] descriptors on the device
    cudaStream_t stream = nullptr;
    int device = 0;
    harm::DevScene dev{};
    harm::MixedTables mixed{};
    std::vector<void *> allocs;
    std::vector<double> r0;
    int64_t nf = 0;
    int nw = 0;
    // echo into host memory: a second compute stream (consecutive blocks overlap),
    // a copy stream and a ring of two device blocks
    cudaStream_t aux_stream = nullptr, copy_stream = nullptr;
    cudaEvent_t fork = nullptr;
    void *ring[2] = {nullptr, nullptr};
    size_t ring_bytes = 0;
    cudaEvent_t ring_ready[2] = {nullptr, nullptr}, ring_free[2] = {nullptr, nullptr};
};

namespace harm {

struct Wave {
    double kx, ky, om, amp, ph;
};

// Wave sets of a scene: [n_sets][nw] components (one set for a homogeneous sea
// state, one per corner of a heterogeneous one).
struct WaveSets {
    int n_sets = 1, nw = 0;
    std::vector<Wave> w;
    const Wave &at(int set, int m) const { return w[(size_t)set * nw + m]; }
};

harm_status build_scene_tables(harm_scene *s);
// Check that p is device memory of the current device and that the allocation
// holding it extends at least `bytes` past p (HARM_E_INVALID with a message
// otherwise; NULL is invalid).
harm_status check_device_span(const void *p, size_t bytes, const char *what);

// Tensor map (CUtensorMap, 128 bytes at map) of a float32 state array
// [np][nf][ny][nx] for bulk tensor stores of [nf][box_y][box_x] boxes, one pulse at
// a time; needs nx % 4 == 0 and a 16-byte aligned state pointer. Fails (without
// touching the device) when the driver offers no tensor-map encoder or rejects
// the layout.
cudaError_t encode_state_map(void *map, float *state, int nx, int ny, int nf, int np, int box_x, int box_y);
void release_host_ring(harm_scene *s);  // copy stream, events and ring of harm_echo_accumulate_host
harm_status build_mixed_tables(harm_scene *s, const std::vector<PulseState> &ps, const WaveSets &waves);
// Separable phasor tables of every wave set, computed on the device in FP64 and
// stored as T2 (float2 or double2) on the scene's stream; tt (FP64 path only,
// e^{-i omega t_s(n)} per pulse) needs the uploaded pulse states ps_dev.
template <typename T2>
cudaError_t phasor_tables(harm_scene *s, const WaveSets &W, const PulseState *ps_dev, const T2 **ex, const T2 **ey,
                          const T2 **tt);

cudaError_t launch_generate(harm_scene *s, int n0, int np, void *state);
cudaError_t launch_accumulate(harm_scene *s, int n0, int np, void *iq, harm_dtype dtype);
cudaError_t launch_accumulate_on(harm_scene *s, cudaStream_t st, int n0, int np, void *iq, harm_dtype dtype);
cudaError_t launch_adjoint(harm_scene *s, int n0, int np, const void *resid, harm_dtype dtype, double *g_sigma0,
                           double *g_uv);

// plain paths (every per-facet step in double, fp64 = true, or in float)
cudaError_t launch_generate_plain(const DevScene &S, bool fp64, cudaStream_t st, int n0, int np, void *state);
cudaError_t launch_accumulate_plain(const DevScene &S, bool fp64, cudaStream_t st, int n0, int np, void *iq,
                                    harm_dtype dtype);
cudaError_t launch_probe_plain(const DevScene &S, bool fp64, cudaStream_t st, int n0, int np, int *bins,
                               void *speckle, void *words, int *cells);
// mixed path
cudaError_t launch_generate_mixed(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                                  float *state);
cudaError_t launch_accumulate_mixed(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                                    void *iq, harm_dtype dtype);
// Device-side description of a batched launch (arrays in device memory).
struct BatchLaunch {
    const void *args;        // [n] per-scene kernel arguments (opaque, batch_args_bytes() each)
    const int *start;        // [n + 1] item prefix sums in processing order
    const int *tiles;        // [n] tiles per pulse batch (by scene)
    const int *ty;           // [n] tile rows (8 or 16, by scene)
    const int *order;        // [n] scene processed at position k
    float *const *iq;        // [n] complex64 outputs (by scene)
    unsigned int *counter;   // work counter (zeroed before the launch)
    const MixedTables *poly; // tap / sinc polynomials (shared)
    int n, total, nc, taps, ctas;
    int variant;             // per-pulse code variant shared by the scenes (see batch_variant)
    int share3;              // every scene: 6 channels, two receive antennas of 3 phase centres
};
size_t batch_args_bytes();
// Launch arguments of a scene for a batched launch whose work items span `window`
// pulses (the scene's time-Taylor window, or the half-length alternative).
void batch_fill_args(const harm_scene *s, void *dst, int window);
int batch_windows(const harm_scene *s, int window);  // work items along the burst for that window
int batch_tiles(const harm_scene *s, int ty);
int batch_variant(const harm_scene *s);  // surface model / pattern kind of the per-pulse code
bool batch_share3(const harm_scene *s);  // 6 channels in two antennas of 3 phase centres
int batch_ctas(int device, int variant);
cudaError_t batch_launch(const BatchLaunch &L, cudaStream_t st);

// Index probe of the mixed accumulator (see harm_probe_indices).
cudaError_t launch_probe_mixed(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np, int *bins,
                               void *speckle, void *words, int *cells);
cudaError_t launch_adjoint_mixed(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                                 const void *resid, harm_dtype dtype, double *g_sigma, double *g_uv);

}  // namespace harm
