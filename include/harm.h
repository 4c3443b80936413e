/*
 * harm.h -- C ABI of the B300-native facet-to-IQ echo generator.
 *
 * The library computes the raw-data hot path of a bistatic SAR/ATI scene-and-
 * instrument simulator (HEEPS/MARE, Sec. II-B and Sec. IV of the paper): for
 * every pulse and receive channel, sea-surface facets are advanced to the pulse
 * time, their complex amplitudes (Eq. 3, Eq. 16) are weighted by the transmit
 * and receive antenna patterns, carry the two-way phase
 * exp(-i K0 (r_t + r_r + v_c t)) with v_c from Eq. 4, and are summed into range
 * samples (Eq. 17, here with a short Kaiser-windowed sinc in place of the box).
 *
 * Conventions shared by every entry point:
 *   - Frame: flat-earth local frame, x along-track, y ground range away from the
 *     radars, z up, origin at the scene centre on the mean surface [m].
 *   - Device memory passed in (iq, state, residual, gradients) belongs to the
 *     caller and must be device memory of the current CUDA device whose allocation
 *     extends over every byte the call touches (both are checked before any launch:
 *     HARM_E_INVALID otherwise; a buffer carved from a larger allocation is only
 *     checked against that allocation's end). The scene owns
 *     only its own tables (and, once harm_echo_accumulate_host has been called,
 *     that call's device ring and streams); no other call allocates.
 *   - Every call is asynchronous on the scene's CUDA stream. A returned status
 *     reports launch-time errors; device-side errors are reported by the next
 *     call or by harm_scene_sync().
 *   - No C++ exception crosses this boundary. On any non-OK status,
 *     harm_last_error() returns a thread-local message.
 *   - A scene may be used by one host thread at a time.
 *
 * Complex outputs are interleaved (re, im) in the element type given by
 * harm_dtype; IQ layout is [n_channels][np][n_range], range fastest.
 */
#ifndef HARM_H
#define HARM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HARM_ABI_VERSION 2u
#define HARM_MAX_CHANNELS 16

typedef enum {
    HARM_OK = 0,
    HARM_E_INVALID = 1,     /* bad argument or descriptor */
    HARM_E_CUDA = 2,        /* CUDA runtime error (message has the CUDA text) */
    HARM_E_OOM = 3,         /* device or host allocation failed */
    HARM_E_TIMEOUT = 4,     /* a bounded device wait gave up */
    HARM_E_UNSUPPORTED = 5  /* valid request this build does not implement */
} harm_status;

typedef enum {
    HARM_C64 = 0,  /* complex64: float re, float im */
    HARM_C128 = 1  /* complex128: double re, double im */
} harm_dtype;

typedef enum {
    HARM_PREC_FP64 = 0,  /* every step in double precision */
    HARM_PREC_MIXED = 1, /* FP64 only for per-pulse state, reference ranges and
                            per-tile range offsets; FP32 for the rest */
    HARM_PREC_FP32 = 2   /* the plain method of HARM_PREC_FP64 with every per-facet
                            step in single precision (per-pulse state built in FP64
                            on the host and rounded): ranges, phases and taps carry
                            FP32 rounding of the ~1e6 m ranges and ~1e5 rad phases,
                            which is what the mixed path's FP64 references avoid */
} harm_precision;

/* One antenna phase centre moving linearly: P(t) = pos0 + vel * t, t = 0 at the
   first pulse of the burst. len_az / len_el are the aperture lengths used by the
   sinc^2 pattern (Sec. III-B, Eq. 16). */
typedef struct {
    double pos0[3];
    double vel[3];
    double len_az;
    double len_el;
} harm_antenna;

/* Scene, instrument and acquisition descriptor (the inputs of Sec. II-B: instrument,
   geometry, acquisition mode and geophysical scene). All fields are copied by
   harm_scene_create; the rx and hetero_* arrays may be freed afterwards.
   Version 1 descriptors (abi_version = 1, struct_size = offsetof(harm_scene_desc,
   speckle_tau_s)) are accepted and run with every version-2 variant off. */
typedef struct {
    uint32_t abi_version;   /* HARM_ABI_VERSION */
    uint32_t struct_size;   /* sizeof(harm_scene_desc) */
    double f0_hz;           /* carrier frequency */
    double fs_hz;           /* range sampling rate; bin = c / fs of bistatic path */
    double prf_hz;          /* pulse repetition frequency; t_n = n / prf */
    int32_t n_pulses;       /* pulses in the burst */
    int32_t n_range;        /* range samples per pulse and channel */
    harm_antenna tx;        /* transmitter */
    int32_t n_channels;     /* receive channels, 1 .. HARM_MAX_CHANNELS */
    const harm_antenna *rx; /* [n_channels] receive phase centres (host memory) */
    int32_t nx, ny;         /* facet grid; facet id f = iy * nx + ix */
    double facet_m;         /* facet edge; centre x = (ix + 1/2 - nx/2) facet_m */
    int32_t n_omega;        /* wave grid: frequency bins (0 = no waves) */
    int32_t n_theta;        /* wave grid: directions */
    double u10;             /* wind speed [m/s] (JONSWAP fetch laws) */
    double fetch_m;         /* fetch [m] */
    double wind_dir_rad;    /* direction the wind blows toward, from +x */
    double spread_s;        /* cos^2s spreading exponent s */
    double gamma;           /* JONSWAP peak enhancement */
    uint64_t wave_seed;     /* Philox key of the wave phases */
    double current_u;       /* uniform surface current [m/s] (Eq. 4) */
    double current_v;
    double sigma0_base;     /* NRCS base value */
    double wind_mod;        /* NRCS wind modulation m in (1 + m cos phi_wind) */
    int32_t epoch_pulses;   /* pulses per speckle coherence epoch (0 = one epoch) */
    uint64_t speckle_seed;  /* Philox key of the speckle */
    int32_t static_surface; /* 1: heights 0 and NRCS = sigma0_base everywhere */
    int32_t taps;           /* 1 (Eq. 17 box) or 8 (Kaiser-windowed sinc) */
    double kaiser_beta;     /* Kaiser window beta for taps = 8 */
    int32_t precision;      /* harm_precision */
    /* ---- abi_version >= 2: surface and scattering variants (Sec. III) ---- */
    double speckle_tau_s;   /* correlation time tau_s of the order-1 autoregressive
                               speckle (Eq. 10): s_e = beta s_(e-1) + sqrt(1 - beta^2) w_e
                               between epochs, beta = exp(-epoch duration / tau_s);
                               0 = independent epochs */
    double speckle_doppler_hz; /* intra-facet Doppler shift f_s of Eq. 7 (uniform):
                               the speckle carries exp(2 i pi f_s t_n) */
    int32_t cwm;            /* 1: Choppy Wave Model -- facets move horizontally along
                               the waves' orbits (Sec. III); 0: linear surface */
    int32_t hetero_ncx;     /* heterogeneous sea state (Eq. 1, 2): corner grid of the */
    int32_t hetero_ncy;     /* TL tiles, corner (cx, cy) at the patch corner + (cx, cy) L;
                               0 = homogeneous. Needs (ncx - 1) L >= nx facet_m and
                               (ncy - 1) L >= ny facet_m, at most 1024 corners. */
    double hetero_tile_m;   /* TL tile size L */
    const double *hetero_u10;          /* [ncy][ncx] wind speed of corner spectrum S_i (host) */
    const double *hetero_wind_dir_rad; /* [ncy][ncx] wind direction of S_i (host); the NRCS
                                          wind term keeps wind_dir_rad */
} harm_scene_desc;

typedef struct harm_scene harm_scene; /* opaque, owned by the library */

/* Scene sizes, filled by harm_scene_query. */
typedef struct {
    int64_t n_facets;
    int32_t n_pulses, n_range, n_channels, n_waves;
    int32_t precision;
    int32_t pulse_batch;     /* pulses per work item of the accumulator */
    double range_bin_m;      /* c / fs */
    double range_start_m[HARM_MAX_CHANNELS]; /* R0 per channel */
} harm_scene_info;

/* Create a scene: validate the descriptor, build the wave component table
   (linear surface, Sec. III), per-pulse platform state with light time (Eq. 3)
   and range windows in FP64 on the host, upload them to the current device on
   `cuda_stream` (a cudaStream_t, NULL = default stream) and evaluate the separable
   wave phasor tables there. *out receives the scene.
   Errors: HARM_E_INVALID for a bad descriptor or NULL pointer, HARM_E_OOM,
   HARM_E_CUDA. On error *out is set to NULL and nothing is leaked. */
harm_status harm_scene_create(const harm_scene_desc *desc, void *cuda_stream, harm_scene **out);

/* Release a scene and its device tables after its stream has drained. NULL is OK. */
harm_status harm_scene_destroy(harm_scene *scene);

/* Fill *info with the scene's sizes. */
harm_status harm_scene_query(const harm_scene *scene, harm_scene_info *info);

/* Per-cell NRCS base and current (u, v), on cells of cell_m starting at the
   patch corner (cell index clamps at the edges). sigma0 [ncy*ncx] and uv
   [ncy*ncx*2] are DEVICE pointers to doubles; either may be NULL to keep the
   uniform value. The scene keeps the pointers: they must stay valid while the
   scene is used. ncx = 0 removes the cell fields. */
harm_status harm_scene_set_cells(harm_scene *scene, int32_t ncx, int32_t ncy, double cell_m,
                                 const double *sigma0_dev, const double *uv_dev);

/* Antenna gain from a u-v grid (Sec. III-B: patterns given in any form are
   converted to u-v grids and looked up per facet and pulse) in place of the
   analytic sinc^2 pattern. antenna = -1 for the transmitter, 0 .. n_channels - 1
   for a receive channel. The grid holds complex gains (field weights) at
   direction cosines u = u0 + i du along the antenna's azimuth axis and
   v = v0 + j dv along its elevation axis: gain_host[j][i] interleaved (re, im)
   doubles, nv x nu nodes, in HOST memory, copied into the scene (double for FP64
   scenes, float for mixed ones). Between nodes the gain is bilinear; outside the
   grid it is zero. gain_host = NULL removes the grid (back to sinc^2). nu, nv in
   2 .. 65536, du, dv > 0. Synchronous with respect to the scene's stream.
   Errors: HARM_E_INVALID, HARM_E_OOM, HARM_E_CUDA. */
harm_status harm_scene_set_pattern(harm_scene *scene, int32_t antenna, int32_t nu, int32_t nv, double u0, double du,
                                   double v0, double dv, const double *gain_host);

/* Facet generator (Sec. III surface; the per-tile surface synthesis of Sec. IV-B): writes
   the state of every facet for pulses [n0, n0 + np) at the bounce time of each
   pulse, to state_dev laid out [np][F][n_facets], in double for HARM_PREC_FP64
   scenes and in float for HARM_PREC_MIXED and HARM_PREC_FP32 scenes. F = 3 fields (eta, eta_x,
   eta_y) for the linear surface; F = 8 with the Choppy Wave Model: (eta, eta_x,
   eta_y, D_x, D_y, dD_x/dx, dD_x/dy, dD_y/dy), D the horizontal displacement and
   every derivative taken with respect to the rest position. For mixed scenes with
   F = 3, nx % 4 == 0 and a 16-byte aligned state_dev the states leave the GPU's
   shared memory by bulk tensor stores (one [3][16][32] box per tile and pulse); any
   other layout takes direct stores. Both write the same bits. state_dev is owned by
   the caller and must hold np * F * n_facets elements of device memory.
   Errors: HARM_E_INVALID for an out-of-range pulse window, a NULL, host or too-short
   pointer; HARM_E_CUDA for a launch failure. */
harm_status harm_facets_generate(harm_scene *scene, int32_t n0, int32_t np, void *state_dev);

/* Echo accumulator (Eq. 3, 4, 16, 17): adds the echo of every facet for pulses
   [n0, n0 + np) and every channel into iq_dev, laid out [n_channels][np][n_range]
   complex of `dtype`. zero_first = 1 clears iq_dev first (on the stream).
   Sums use floating-point atomics: repeated runs agree to rounding, not bit for
   bit, unless the scene is in deterministic mode (harm_scene_set_deterministic).
   Errors: HARM_E_INVALID (window, pointer, dtype), HARM_E_UNSUPPORTED (a
   complex64 output in deterministic mode). */
harm_status harm_echo_accumulate(harm_scene *scene, int32_t n0, int32_t np, void *iq_dev,
                                 harm_dtype dtype, int32_t zero_first);

/* Deterministic mode of a plain-path scene (HARM_PREC_FP64 or HARM_PREC_FP32;
   on = 0 turns it off): harm_echo_accumulate and harm_echo_accumulate_host then
   round every contribution to a multiple of 2^-40 and add it as a 64-bit integer,
   so that the sums are exact and repeated runs give bit-identical IQ whatever
   order the atomic additions take (the output must be complex128; the buffer
   holds the fixed-point values during the call and FP64 again when it ends).
   Range: every real and imaginary IQ part, including values already in the
   buffer when zero_first = 0, below 2^23 in magnitude (larger values already
   present are clamped and reported by harm_scene_sync as a bounds error). The
   rounding adds at most 2^-41 per contribution. Errors: HARM_E_INVALID (NULL),
   HARM_E_UNSUPPORTED (a mixed-precision scene). */
harm_status harm_scene_set_deterministic(harm_scene *scene, int32_t on);

/* Echo into HOST memory (Sec. IV-B: raw data leave the GPU while the next part
   is computed): writes the IQ of pulses [n0, n0 + np) to iq_host, laid out
   [n_channels][np][n_range] complex of `dtype` (overwritten, not added to). The
   burst runs in blocks of block_pulses pulses (<= 0: about an eighth of the
   burst, a multiple of the mixed path's time-Taylor window of
   harm_scene_info.pulse_batch = 256 pulses) into a ring of two device buffers that the
   scene owns, alternating between the scene's stream and a second compute
   stream; each block is copied to iq_host on a copy stream while the next one is
   computed. iq_host must be page-locked (cudaHostAlloc / cudaHostRegister)
   and stay valid until the scene's stream has passed the call: like every call
   here it is asynchronous, and iq_host is complete after harm_scene_sync (or a
   wait on the scene's stream, which the call joins to the other two). The ring
   (2 x n_channels x block x n_range elements) and the streams are kept for later
   calls and freed with the scene.
   Errors: HARM_E_INVALID (window, NULL or pageable iq_host, dtype), HARM_E_OOM
   (ring allocation), HARM_E_CUDA. */
harm_status harm_echo_accumulate_host(harm_scene *scene, int32_t n0, int32_t np, void *iq_host,
                                      harm_dtype dtype, int32_t block_pulses);

/* Adjoint of harm_echo_accumulate with respect to the per-cell NRCS base and the
   per-cell current (the transposed scatter as a gather over range bins): for the
   misfit L = sum |IQ - target|^2 and residual r = IQ - target (resid_dev, same
   layout and dtype as the IQ), adds dL/dsigma0_cell to grad_sigma0_dev [ncy*ncx]
   and dL/d(u, v)_cell to grad_uv_dev [ncy*ncx*2] (device doubles, either may be
   NULL). Requires cells set by harm_scene_set_cells. Facet states are recomputed,
   not stored. Errors: HARM_E_INVALID, HARM_E_UNSUPPORTED. */
harm_status harm_echo_adjoint(harm_scene *scene, int32_t n0, int32_t np, const void *resid_dev,
                              harm_dtype dtype, double *grad_sigma0_dev, double *grad_uv_dev);

/* ----------------------------------------------------------------------------
   Batched scenes (Sec. IV-B: the scene is processed as a batch of tiles; here a
   batch of independent scenes of uneven size runs as one persistent launch).
   ------------------------------------------------------------------------- */
typedef struct harm_batch harm_batch; /* opaque, owned by the library */

/* Group n_scenes mixed-precision scenes (same device, same channel count, same
   taps and Kaiser beta) into one batched forward launch on the first scene's
   stream. The batch keeps pointers to the scenes: they must outlive it, and it
   copies their launch arguments (cells, u-v grids) when it is created, so a
   scene changed afterwards needs a new batch. All scenes share the surface model
   (cwm) and the pattern kind (with or without u-v grids). The work
   list is every (scene, 32 x rows facet tile, pulse window) item over the full
   burst of every scene, largest scenes first; a pulse window is the mixed path's
   time-Taylor window (harm_scene_info.pulse_batch pulses). Errors: HARM_E_INVALID (NULL,
   n_scenes < 1, mixed devices, channel counts or tap settings),
   HARM_E_UNSUPPORTED (an FP64 scene), HARM_E_OOM, HARM_E_CUDA. */
harm_status harm_batch_create(harm_scene *const *scenes, int32_t n_scenes, harm_batch **out);

/* Autotuner of the launch shape. Per scene-size class (fewer than 1e6 facets,
   fewer than 4e6, more) it times the persistent launch on the first 256 pulses
   of the class's largest scenes (as many as give the launch at least eight waves
   of work items) with each tile height (16 or 8 facet rows)
   and each time-Taylor window (harm_scene_info.pulse_batch pulses per work item,
   or half of it) -- 1 untimed and 3 timed launches per candidate, median -- and
   keeps the fastest, where a candidate replaces the default shape (16 rows, full
   window, timed first) only when it is more than 2 % faster; then it times the
   launch over all classes' samples with 2 and 1 CTAs per SM (1 only for the
   Choppy Wave Model) and keeps the faster under the same rule. The
   choices are remembered for the life of the process per (device, surface model
   and pattern kind, channel count, taps, channel layout, size class), so a later
   batch of the same kind is configured without timing. The tile width (32
   facets, the warp's lanes) is fixed. iq_dev[s] are the scenes' complex64 IQ
   buffers [n_channels][n_pulses][n_range] (device); their contents are
   overwritten. Synchronous. */
harm_status harm_batch_tune(harm_batch *batch, void *const *iq_dev);

/* The launch shape in use: tile rows and pulses per work item of each scene
   (rows[n_scenes], windows[n_scenes], host memory; either may be NULL) and the
   CTAs per SM of the launch (may be NULL). */
harm_status harm_batch_config(const harm_batch *batch, int32_t *rows, int32_t *windows, int32_t *ctas_per_sm);

/* Pin the launch shape instead of tuning: rows[s] 8 or 16, windows[s] the
   scene's pulse_batch or half of it, ctas_per_sm 1 or 2 (1 for the Choppy Wave
   Model). The next harm_batch_run captures its graph again. Synchronous with
   respect to the batch's earlier launches. Errors: HARM_E_INVALID. */
harm_status harm_batch_set_config(harm_batch *batch, const int32_t *rows, const int32_t *windows,
                                  int32_t ctas_per_sm);

/* Tile heights chosen for each scene (rows[n_scenes], host memory). */
harm_status harm_batch_tile_rows(const harm_batch *batch, int32_t *rows);

/* Set the tile height of each scene (rows[n_scenes], host memory, each 8 or 16
   facet rows) instead of tuning: 16-row tiles run two facets per thread on
   adjacent rows, 8-row tiles one (less padding on scenes few rows high). The
   next harm_batch_run captures its graph again. Synchronous with respect to the
   batch's earlier launches. Errors: HARM_E_INVALID (NULL, a value other than 8 or
   16), HARM_E_CUDA. */
harm_status harm_batch_set_tile_rows(harm_batch *batch, const int32_t *rows);

/* Echo of every scene over its full burst into iq_dev[s] (complex64, device),
   as one persistent launch replayed from a CUDA graph; the graph is captured on
   the first call and again whenever the output pointers or zero_first change.
   zero_first = 1 clears the outputs first (inside the graph). Asynchronous on
   the batch's stream. */
harm_status harm_batch_run(harm_batch *batch, void *const *iq_dev, int32_t zero_first);

/* Release the batch (waits for its stream). NULL is OK. */
harm_status harm_batch_destroy(harm_batch *batch);

/* Allocation-free batched forward run (the paper has no counterpart; this is a
   service for callers that cannot allocate device memory where they run the
   echo, e.g. a loop with a fixed device-memory budget or code inside a framework
   whose caching allocator owns the device, where cudaMalloc / cudaFree could
   synchronise the device or fail). Same result as harm_batch_create +
   harm_batch_run over `scenes` (16-row tiles, no tuning, no graph), but the
   launch's scratch memory -- per-scene arguments, work list, output pointers and
   the work counter -- lives in one file-scope device array of fixed size (about
   132 KB, held on every GPU that loads the library until the process exits), and
   the call makes no cudaMalloc, cudaFree or other allocating call.
   scenes[n_scenes]: mixed-precision scenes on the current device with the same
   channel count, taps and Kaiser beta; iq_dev[n_scenes]: their complex64 IQ
   buffers [n_channels][n_pulses][n_range] (device). zero_first = 1 clears them
   first. Asynchronous on the first scene's stream.
   Limits and sharing: at most 64 scenes per call (more -> HARM_E_INVALID). All
   calls share the one array; each call rewrites it completely (including the
   work counter, which starts at zero), but two calls whose launches overlap on
   the GPU (different streams, no ordering between them) race on it: order such
   calls on one stream or with events. The first call on a device looks up the
   array's device address (cudaGetSymbolAddress); make that first call before any
   stream capture. Errors: HARM_E_INVALID, HARM_E_UNSUPPORTED (an FP64 scene),
   HARM_E_CUDA. */
harm_status harm_batch_run_noalloc(harm_scene *const *scenes, int32_t n_scenes, void *const *iq_dev,
                                   int32_t zero_first);

/* Index probe (diagnostic; the parity tests use it to compare the accumulator's
   integer work bit for bit): runs the work items of harm_echo_accumulate over
   pulses [n0, n0 + np) with the same per-facet code -- tile references, surface,
   speckle, ranges -- up to the scatter, and instead of adding contributions
   records, per facet f (grid index iy * nx + ix) and pulse j = n - n0:
     bins_dev    [np][n_channels][n_facets] int32: first range bin of the facet's
                 taps in each channel (floor(p) - 3 for the 8-tap kernel, floor(p)
                 for the Eq. 17 box, p the bin position of Eq. 17's range sum);
     speckle_dev [np][n_facets] complex (complex128 for HARM_PREC_FP64 scenes,
                 complex64 otherwise): the speckle draw z of pulse n's coherence
                 epoch (Eq. 7 at f_s = 0, or the recurrence of Eq. 10);
     words_dev   [np][n_facets][4] uint32: the Philox4x32-10 words of counter
                 (f, 0, epoch, 0) under the speckle key, the draw's source;
     cells_dev   [n_facets] int32: the facet's cell index (-1 without cells).
   All four are device buffers of the current device (none may be NULL); they
   are overwritten. Every precision (the plain paths run their own accumulator
   with the same recording). Asynchronous on the scene's stream.
   Errors: HARM_E_INVALID (window, pointers), HARM_E_CUDA. */
harm_status harm_probe_indices(harm_scene *scene, int32_t n0, int32_t np, int32_t *bins_dev, void *speckle_dev,
                               uint32_t *words_dev, int32_t *cells_dev);

/* Wait for the scene's stream and report device-side errors (bounded waits that
   timed out, bounds flags) raised since the last check. */
harm_status harm_scene_sync(harm_scene *scene);

/* Thread-local text of the last non-OK status on this thread ("" if none). */
const char *harm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HARM_H */
