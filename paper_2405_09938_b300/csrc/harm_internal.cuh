// Internal data layout of the CUDA echo path (not part of the ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "harm.h"

namespace harm {

constexpr double kC = 299792458.0;
constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxCh = HARM_MAX_CHANNELS;
constexpr int kMaxI0Terms = 40;

// State of one antenna phase centre for one pulse (FP64): position at its
// transmit / receive time, steered antenna frame, and range to the scene centre.
struct AntState {
    double p[3];
    double a[3];  // azimuth axis
    double e[3];  // elevation axis
    double rref;  // |p - 0|
};

// Per-pulse record (FP64, host-computed at scene creation).
struct PulseState {
    double t;   // transmit time t_n
    double ts;  // bounce time at the scene centre
    AntState tx;
};

// Per (pulse, channel) record: receive antenna state plus the reference phase
// and range-bin offset of the scene centre.
struct RxState {
    AntState rx;
    double psi;     // -K0 (R_t + R_r) reduced to (-pi, pi]
    double p_ref;   // (R_t + R_r - R0_c) / dr: bin position of the scene centre
};

// u-v gain grid of one antenna (device copy owned by the scene).
struct PatLut {
    int nu, nv;
    double u0, inv_du, v0, inv_dv;
    const double2 *g64;  // [nv][nu] (FP64 scenes)
    const float4 *g32;   // [nv][nu - 1] node pairs (g[j][i], g[j][i + 1]) (mixed scenes)
};

// Scene constants passed by value to every kernel.
struct DevScene {
    int nx, ny, nc, nr, np_total, nw, taps, static_surface, epoch_pulses;
    int n_i0;               // terms of the Kaiser window series
    double dx, k0, inv_lambda, inv_dr, area;
    double tx_laz, tx_lel;
    double rx_laz[kMaxCh], rx_lel[kMaxCh];
    double sigma0_base, wind_mod, wcos, wsin, cur_u, cur_v;
    uint64_t speckle_seed;
    double i0c[kMaxI0Terms];  // window series coefficients / I0(beta)
    // per-cell fields (device pointers owned by the caller) or null
    int ncx, ncy;
    double cell;
    const double *cell_sigma0;
    const double *cell_uv;
    // scene tables (device)
    const PulseState *pulses;  // [np_total]
    const RxState *rx;         // [np_total][nc]
    const double *kx, *ky, *om;  // [nw]
    const double2 *ex;          // [nw][nx]   e^{i kx x}
    const double2 *ey;          // [nw][ny]   a e^{i phi} e^{i ky y}
    const double2 *tt;          // [nw][np_total] e^{-i omega t_s}
    // the same tables in float (FP32 plain path)
    const float2 *ex32, *ey32, *tt32;
    unsigned int *flags;        // device error / overflow counters [4]
    // variants of Sec. III
    int cwm;                    // Choppy Wave Model: 8 state fields instead of 3
    int n_sets;                 // wave sets: 1, or one per corner of a heterogeneous sea state
    int het_ncx, het_ncy;       // corner grid (0 = homogeneous)
    double het_l, het_x0, het_y0;  // TL tile size, position of corner (0, 0)
    double spk_beta, spk_q;     // AR(1) speckle s_e = beta s_(e-1) + q w_e (beta = 0: independent)
    int spk_terms;              // AR(1) terms kept when a pulse window starts mid-burst
    double fd_hz;               // intra-facet Doppler shift f_s
    unsigned int lut_mask;      // bit 0: transmitter grid, bit 1 + c: receive channel c grid
    const PatLut *luts;         // [1 + nc] (device)
    const double *kn;           // [n_sets][nw] |k| (CWM direction cosines of the waves)
    int det;                    // plain paths: deterministic fixed-point sums (complex128 output)
    unsigned int rx_share;      // bit c: channel c is a phase centre of channel c - 1's receive
                                // antenna (mixed path: the analytic pattern gain is shared)
};

// Mixed-precision tables (FP32 separable waves, Taylor time tables).
struct DevMixed {
    int nb;          // pulses per batch
    int n_order;     // Taylor orders in time (M + 1)
    int n_batches;
    const float2 *ex;   // [nw][nx]
    const float2 *ey;   // [nw][ny]
    const float4 *wt;   // [n_batches][nw][n_order] : (E.re, E.im, omega-free k terms packed)
    const float *tau;   // [np_total] t_s(n) - t_centre(batch(n))
    const float *kx, *ky; // [nw]
};

}  // namespace harm
