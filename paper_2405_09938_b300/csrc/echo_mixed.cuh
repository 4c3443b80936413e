// Mixed-precision echo path: FP64 only for per-pulse platform state, the
// reference bistatic range and each tile's range offset; FP32 for the per-facet
// geometry, antenna patterns, NRCS, phase, interpolation taps and accumulation.
//
// Work decomposition (one CTA = a 32 x 16 facet tile x a 256-pulse batch):
//  1. Facet generator: the surface of the tile over the batch is expanded in time
//     about the batch centre, eta(t_c + tau) = sum_m eta_m tau^m (m <= 5), with
//     the Taylor coefficients accumulated over the wave components: each is a
//     real factor times the real or imaginary part of the component's phasor
//     Q_w = e^{i kx x} a e^{i (ky y + phi)} e^{-i omega t_c} (FP32, packed over
//     pairs of orders; 64-component chunks of the factors and of the tile's
//     column and row phasors staged in shared memory).
//  2. FP64 tile references, per 16-pulse chunk: for every pulse and antenna, the
//     range R from the antenna to the tile's reference point on the mean surface,
//     its unit vector and the tile's reduced reference phase and range-bin offset.
//     Per facet, r - R is a small offset that FP32 carries to ~1e-8 m:
//        r - R = a + (b - a^2) / (2R) + (a^3 - a b) / (2R^2),  a = u.xi, b = |xi|^2
//     for the facet offset xi from the reference point; the linear phase term
//     K0 (u_t + u_r).xi is split into exactly-reduced lattice steps.
//  3. For each pulse: each thread evaluates its two facets (adjacent rows 2w and
//     2w + 1 of the tile) together in packed FP32x2 arithmetic: Horner in time,
//     then per channel the contribution (Eq. 3, 4, 16) and its 8 Kaiser-sinc taps
//     (polynomials in the fractional bin). The two facets' first bins differ by at
//     most one, so each lane merges their taps into 9 values; the warp pre-reduces
//     its 32 lanes: each lane writes its values into its own (row-rotated) column
//     of a per-warp [16 bin x 32 lane] shared buffer at the rows of its bins, then
//     each lane sums one bin-row half with vector loads; one shared atomic per
//     (bin, component) adds the warp's window to the CTA range tile, which is
//     flushed to the IQ with one vector atomic per bin and channel.
//  The adjoint runs the same per-pulse arithmetic and gathers the residual
//  through the same taps instead of scattering.
//
// Variants of Sec. III are template parameters V of the per-pulse code (bit 0:
// Choppy Wave Model, 8 state fields; bit 1: u-v antenna gain grids) or run-time
// switches of the per-item setup (heterogeneous sea state: the generator sums
// the wave sets of the tile's corners with the weights of Eq. 2; AR(1) speckle:
// the epoch recurrence of Eq. 10). Each V is compiled in its own translation
// unit, which includes this file and instantiates MixedLaunch<V>.
#pragma once
#include <cuda.h>  // CUtensorMap (type only: the library does not link the driver library)
#include <cuda_runtime.h>

#include <climits>
#include <cstring>

#include "harm_internal.cuh"
#include "harm_kernels.cuh"
#include "philox.cuh"

namespace harm {
namespace {

constexpr int TX = 32;        // facets along x per tile (= warp lanes)
constexpr int TY = 16;        // facets along y per tile (2 rows per warp)
constexpr int NT = 256;       // threads per CTA
constexpr int NWARP = NT / 32;
constexpr int WT = 48;        // range bins per channel in the CTA tile
constexpr int WT_LO = 22;     // tile window starts WT_LO bins below the reference bin
constexpr int WA = 32;        // range bins per channel of the adjoint's residual window
constexpr int WA_LO = 14;     // (a 32 x 16 facet tile spans about +-10 bins around its
                              // reference bin, taps and heights included; residuals
                              // outside the window are read from global memory)
constexpr int NBR = 32;       // pulses per chunk of FP64 tile references
constexpr int NBG = 256;      // pulses per work item (time-Taylor window of the generator;
                              // |omega tau| <= 0.2 on the headline wave spectrum)
constexpr int WCH = 64;       // wave components per shared-memory chunk of the generator
constexpr int SROW = 72;      // floats per bin row of the warp buffer (2 halves of 32 + pad)
constexpr int SHALF = 36;     // float offset of lanes 16..31 in a row
constexpr int SBINS = 16;     // bins per warp window
constexpr int kTileBufs = 4;  // CTA range tiles in flight (a ring over consecutive pulses)
constexpr float kPiF = 3.14159265358979f;

// Variant bits of the per-pulse code.
constexpr int kVarCwm = 1;  // Choppy Wave Model: 8 state fields, displaced facets
constexpr int kVarLut = 2;  // u-v antenna gain grids (complex gains)

template <int V>
struct Var {
    static constexpr bool CWM = (V & kVarCwm) != 0;
    static constexpr bool LUT = (V & kVarLut) != 0;
    static constexpr int NF = CWM ? 8 : 3;        // state fields
    static constexpr int MIN_BLOCKS = CWM ? 1 : 2; // CTAs per SM the registers allow
    // channel-loop unroll of the forward pulse body (measured: 2 for the linear
    // surface; the Choppy Wave Model, at one CTA per SM, runs best rolled). With
    // the six-channel two-antenna layout known at compile time the loop is
    // unrolled fully (by three, one antenna, for the Choppy Wave Model).
    static constexpr int FWD_CU = CWM ? 1 : 2;
};

// FP32 tile reference of one antenna for one pulse (16 floats).
struct __align__(16) AntRec {
    float ux, uy, uz, invR;      // unit vector to the tile reference point, 1/R
    float inv2R, inv2R2, u0, v0; // 1/(2R), 1/(2R^2), pattern direction cosines
    float aRx, aRy, aRz, ampr;   // azimuth axis / R, Rbar / R
    float eRx, eRy, eRz, pad;    // elevation axis / R
};

// Per (pulse, channel) phase and range references of the tile.
struct __align__(16) ChanRec {
    float psi, ax, ay, gam;  // reduced reference phase, lattice phase steps, vertical phase rate
    float pfrac;             // fractional bin of the reference point
    int kbase;               // integer bin of the reference point
    float gx, gy;            // horizontal phase rates -K0 (u_t + u_r)_{x,y} (CWM displacement)
};

struct __align__(16) PulseRec {
    float tau, k0t;
    int epoch;
    int pad;
};

// The same references with every value duplicated into a pair (v, v), formed in
// registers where a packed two-facet step reads a record (dup_rec, dup_chan):
// the packed FP32x2 arithmetic takes each reference as one 64-bit operand, while
// shared memory holds only the scalar records (half the bytes and loads of a
// duplicated layout, which leaves room for 32-pulse reference chunks).
struct __align__(16) AntRec2 {
    float2 ux, uy, uz, invR;
    float2 inv2R, inv2R2, u0, v0;
    float2 aRx, aRy, aRz, ampr;
    float2 eRx, eRy, eRz, pad;
};

struct __align__(16) ChanRec2 {
    float2 psi, ax, ay, gam;
    float2 pfrac;
    int kbase;
    float gx, gy;
    int pad0;
};

// u-v gain grid of one antenna in FP32 (shared memory copy of the descriptor).
struct PatLutF {
    const float4 *g;  // [nv][nu - 1] node pairs
    int nu, nv;
    float u0, inv_du, v0, inv_dv;
    float umax, vmax;  // nu - 1, nv - 1
};

struct MixedArgs {
    DevScene S;
    const float2 *ex, *ey, *tc;
    const float *cr;
    const float *tau;
    int nb, n_batches;
    // FP32 constants
    float tx_laz_l, tx_lel_l;  // aperture / wavelength
    float rx_laz_l[kMaxCh], rx_lel_l[kMaxCh];
    float wcos, wsin, wind_mod, area, k0, inv_dr;
};

// Polynomial tables shared by every scene of a launch (they depend only on the
// Kaiser beta): passed as kernel parameters so the inner loops read them from
// the constant bank.
// Each coefficient is stored as the pair (c, c) so that the packed two-facet
// evaluation reads it as one 64-bit constant operand; scalar code reads .x.
// The Kaiser-sinc taps are symmetric, h_(7-j)(t) = h_j(-t) for t = 2f - 1 (the
// window is even), so taps j and 7 - j come from the even and odd parts of one
// polynomial: h_j = E_j(t^2) + t O_j(t^2), h_(7-j) = E_j(t^2) - t O_j(t^2), j = 0..3.
constexpr int kTapEven = kTapDeg / 2 + 1;        // coefficients of E_j in t^2
constexpr int kTapOdd = (kTapDeg + 1) / 2;       // coefficients of O_j in t^2
struct PolyArgs {
    float2 tap_e[4][kTapEven];
    float2 tap_o[4][kTapOdd];
    float2 sinc2[kSincDeg + 1];
};

// Bytes of one generator chunk in shared memory: the real Taylor factors of WCH
// wave components (nf fields x kOrders orders, float) and their phasors on the
// tile's TX columns and TY rows (float2).
__host__ __device__ constexpr int wave_chunk_bytes(int nf) { return WCH * (nf * kOrders * 4 + (TX + TY) * 8); }

// Shared-memory layout (bytes), sized for nc channels and nf state fields.
struct Layout {
    int w, tile, tx, rx, ch, pr, txd, stage, lut, coef, total;
};

// The wave-table chunk (generator phase) and the warp buffers (pulse loop) are
// never live at the same time and share one region; the warp buffers are
// cleared after the generator phase.
// Every region starts on a 16-byte boundary (regions are read with 128-bit loads).
__host__ __device__ inline int align16(int o) { return (o + 15) & ~15; }

__host__ __device__ inline Layout layout(int nc, int nf)
{
    Layout L;
    int o = 0;
    const int wbytes = wave_chunk_bytes(nf);
    const int sbytes = NWARP * SBINS * SROW * 4;
    L.w = o;
    L.stage = o;
    o += wbytes > sbytes ? wbytes : sbytes;
    L.tile = o = align16(o);  o += kTileBufs * nc * WT * 8;
    L.tx = o = align16(o);    o += NBR * (int)sizeof(AntRec);
    L.rx = o = align16(o);    o += NBR * nc * (int)sizeof(AntRec);
    L.ch = o = align16(o);    o += NBR * nc * (int)sizeof(ChanRec);
    L.pr = o = align16(o);    o += NBR * (int)sizeof(PulseRec);
    L.txd = o = align16(o);   o += NBR * 4 * 8;
    L.lut = o = align16(o);   o += (1 + kMaxCh) * (int)sizeof(PatLutF);
    // Taylor coefficients of the thread's two facets, [3][kOrders / 2][NT] float4 (the
    // pairs of orders 2q and 2q + 1), for the linear surface (the 8-field CWM keeps
    // them in registers)
    L.coef = o = align16(o);  o += nf == 3 ? 3 * kOrders * NT * 8 : 0;
    L.total = align16(o);
    return L;
}

struct Smem {
    float2 *w;       // [WCH][nf][kOrders / 2] real Taylor factors, order pairs (2p, 2p + 1)
    float2 *wx;      // [WCH][TX] e^{i kx x} of the tile's columns
    float2 *wy;      // [WCH][TY] a e^{i (ky y + phi)} of the tile's rows
    float2 *tile;    // [kTileBufs][nc][WT]
    AntRec *tx;      // [NBR]
    AntRec *rx;      // [NBR][nc]
    ChanRec *ch;     // [NBR][nc]
    PulseRec *pr;    // [NBR]
    double *txd;     // [NBR][4]
    float *stage;    // [NWARP][SBINS][SROW]
    PatLutF *lut;    // [1 + nc] u-v gain grids (LUT variant)
    float2 *coef;    // [3][kOrders / 2][NT] float4 Taylor coefficients (linear surface)
};

__device__ __forceinline__ Smem carve(unsigned char *raw, int nc, int nf)
{
    Layout L = layout(nc, nf);
    Smem s;
    s.w = reinterpret_cast<float2 *>(raw + L.w);
    s.wx = reinterpret_cast<float2 *>(raw + L.w + WCH * nf * kOrders * 4);
    s.wy = s.wx + WCH * TX;
    s.tile = reinterpret_cast<float2 *>(raw + L.tile);
    s.tx = reinterpret_cast<AntRec *>(raw + L.tx);
    s.rx = reinterpret_cast<AntRec *>(raw + L.rx);
    s.ch = reinterpret_cast<ChanRec *>(raw + L.ch);
    s.pr = reinterpret_cast<PulseRec *>(raw + L.pr);
    s.txd = reinterpret_cast<double *>(raw + L.txd);
    s.stage = reinterpret_cast<float *>(raw + L.stage);
    s.lut = reinterpret_cast<PatLutF *>(raw + L.lut);
    s.coef = reinterpret_cast<float2 *>(raw + L.coef);
    return s;
}

// sinc^2(x): polynomial for |x| <= 1 (main lobe and the start of the first
// sidelobe), sin(pi x) / (pi x) otherwise.
__device__ __forceinline__ float sinc2f(const PolyArgs &P, float x)
{
    float u = x * x;
    if (u <= 1.0f) {
        float t = fmaf(2.0f, u, -1.0f);
        float r = P.sinc2[kSincDeg].x;
#pragma unroll
        for (int d = kSincDeg - 1; d >= 0; --d) r = fmaf(r, t, P.sinc2[d].x);
        return r;
    }
    float s = __fdividef(sinpif(x), kPiF * x);
    return s * s;
}

// Packed FP32x2 arithmetic (two facets per thread: .x and .y).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }

// sinc^2 of two arguments: the packed polynomial when both are within |x| <= 1.
__device__ __forceinline__ float2 sinc2_2(const PolyArgs &P, float2 x)
{
    const float2 u = mul2(x, x);
    if (u.x <= 1.0f && u.y <= 1.0f) {
        const float2 t = fma2(make_float2(2.0f, 2.0f), u, make_float2(-1.0f, -1.0f));
        float2 r = P.sinc2[kSincDeg];
#pragma unroll
        for (int d = kSincDeg - 1; d >= 0; --d) r = fma2(r, t, P.sinc2[d]);
        return r;
    }
    return make_float2(sinc2f(P, x.x), sinc2f(P, x.y));
}

__device__ __forceinline__ double wrap_pi(double a)
{
    return a - 2.0 * kPi * rint(a * (0.5 / kPi));
}

// FP64 tile reference of one antenna (state A) for the tile reference point
// X = (xr, yr, 0): D = X - p, R = |D|, u = D / R, and the stable offset
// R - |p| = (|X|^2 - 2 p.X) / (R + |p|).
// 1 / sqrt(s) and 1 / x in FP64 from an FP32 estimate and one Newton-Raphson
// step (y <- y (3 - s y^2) / 2, y <- y (2 - x y)): quadratic convergence takes the
// estimate's ~2^-23 relative error to ~2^-45, i.e. below 1e-13 relative (1e-7 m
// on the 880 km ranges here), at a third of the FP64 operations of a correctly
// rounded sqrt and division (FP64 runs at 1/64 of the FP32 rate on this part).
__device__ __forceinline__ double rsqrt_nr(double s)
{
    const double y = (double)rsqrtf((float)s);
    return y * fma(-0.5 * s, y * y, 1.5);
}
__device__ __forceinline__ double rcp_nr(double x)
{
    const double y = (double)(1.0f / (float)x);
    return fma(y, fma(-x, y, 1.0), y);
}

__device__ void tile_ref(const AntState &A, double xr, double yr, double u[3], double &dref, AntRec &o)
{
    double D[3] = {xr - A.p[0], yr - A.p[1], -A.p[2]};
    const double s = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
    const double iR = rsqrt_nr(s);
    const double R = s * iR;
    for (int i = 0; i < 3; ++i) u[i] = D[i] * iR;
    double xx = xr * xr + yr * yr;
    dref = (xx - 2.0 * (A.p[0] * xr + A.p[1] * yr)) * rcp_nr(R + A.rref);
    // the record's factors need only FP32: form them from FP32-rounded inputs
    // (FP64 runs at 1/64 of the FP32 rate here)
    const float ux = (float)u[0], uy = (float)u[1], uz = (float)u[2], ir = (float)iR;
    const float ax = (float)A.a[0], ay = (float)A.a[1], az = (float)A.a[2];
    const float ex = (float)A.e[0], ey = (float)A.e[1], ez = (float)A.e[2];
    o.ux = ux;
    o.uy = uy;
    o.uz = uz;
    o.invR = ir;
    o.inv2R = 0.5f * ir;
    o.inv2R2 = 0.5f * ir * ir;
    o.u0 = fmaf(ux, ax, fmaf(uy, ay, uz * az));
    o.v0 = fmaf(ux, ex, fmaf(uy, ey, uz * ez));
    o.aRx = ax * ir;
    o.aRy = ay * ir;
    o.aRz = az * ir;
    o.ampr = (float)(A.rref * iR);
    o.eRx = ex * ir;
    o.eRy = ey * ir;
    o.eRz = ez * ir;
    o.pad = 0.0f;
}

__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }

// The pair forms of a record at its use (see AntRec2).
__device__ __forceinline__ AntRec2 dup_rec(const AntRec &r)
{
    AntRec2 o;
    o.ux = dup(r.ux); o.uy = dup(r.uy); o.uz = dup(r.uz); o.invR = dup(r.invR);
    o.inv2R = dup(r.inv2R); o.inv2R2 = dup(r.inv2R2); o.u0 = dup(r.u0); o.v0 = dup(r.v0);
    o.aRx = dup(r.aRx); o.aRy = dup(r.aRy); o.aRz = dup(r.aRz); o.ampr = dup(r.ampr);
    o.eRx = dup(r.eRx); o.eRy = dup(r.eRy); o.eRz = dup(r.eRz); o.pad = dup(0.0f);
    return o;
}

__device__ __forceinline__ ChanRec2 dup_chan(const ChanRec &q)
{
    ChanRec2 o;
    o.psi = dup(q.psi); o.ax = dup(q.ax); o.ay = dup(q.ay); o.gam = dup(q.gam); o.pfrac = dup(q.pfrac);
    o.kbase = q.kbase; o.gx = q.gx; o.gy = q.gy; o.pad0 = 0;
    return o;
}

// Transmit references of pulse pa + t: record, FP64 unit vector and range offset,
// pulse record.
__device__ __forceinline__ void tx_refs(const Smem &sm, const MixedArgs &A, int pa, int t, double xr, double yr)
{
    const DevScene &S = A.S;
    const int n = pa + t;
    const PulseState &P = S.pulses[n];
    double u[3], dref;
    AntRec r;
    tile_ref(P.tx, xr, yr, u, dref, r);
    sm.tx[t] = r;
    sm.txd[4 * t + 0] = u[0];
    sm.txd[4 * t + 1] = u[1];
    sm.txd[4 * t + 2] = u[2];
    sm.txd[4 * t + 3] = dref;
    PulseRec pr;
    pr.tau = A.tau[n];
    pr.k0t = (float)(S.k0 * P.t);
    pr.epoch = S.epoch_pulses > 0 ? n / S.epoch_pulses : 0;
    pr.pad = 0;
    sm.pr[t] = pr;
}

// Channel record t = (pulse pi, channel c) from the receive references (u, dref,
// r) and the pulse's transmit references in shared memory.
__device__ __forceinline__ void rx_combine(const Smem &sm, const MixedArgs &A, int pa, int t, const double u[3],
                                           double dref, const AntRec &r)
{
    const DevScene &S = A.S;
    const int pi = t / S.nc, c = t % S.nc;
    const int n = pa + pi;
    const RxState &Rs = S.rx[(size_t)n * S.nc + c];
    const double *td = sm.txd + 4 * pi;
    double off = td[3] + dref;  // (R_t + R_r) - (Rbar_t + Rbar_r)
    ChanRec q;
    // reference phase, with the intra-facet Doppler rotation 2 pi f_s t_n (Eq. 7)
    double psi = Rs.psi - S.k0 * off;
    if (S.fd_hz != 0.0) psi += 2.0 * kPi * S.fd_hz * S.pulses[n].t;
    q.psi = (float)wrap_pi(psi);
    q.ax = (float)wrap_pi(-S.k0 * (td[0] + u[0]) * S.dx);
    q.ay = (float)wrap_pi(-S.k0 * (td[1] + u[1]) * S.dx);
    q.gam = (float)(-S.k0 * (td[2] + u[2]));
    q.gx = q.gy = 0.0f;
    if (S.cwm) {
        q.gx = (float)(-S.k0 * (td[0] + u[0]));
        q.gy = (float)(-S.k0 * (td[1] + u[1]));
    }
    double p = Rs.p_ref + off * S.inv_dr;
    double kb = floor(p);
    q.kbase = (int)kb;
    q.pfrac = (float)(p - kb);
    sm.rx[t] = r;
    sm.ch[t] = q;
}

// FP64 references of the batch's pulses [pa, pe) for the tile reference point
// (xr, yr), thread-parallel over (pulse, antenna). With CONCURRENT the receive
// references (threads [0, npb x nc)) and the transmit references (the next
// warp-aligned threads) are formed at the same time and the channel records
// combine them after one barrier (the adjoint: 1.4 % faster); otherwise, and when
// the CTA has too few threads for that, the transmit stage runs first (the
// forward, whose pulse loop keeps more registers live across the call).
template <bool CONCURRENT>
__device__ void build_refs(const Smem &sm, const MixedArgs &A, int pa, int pe, double xr, double yr)
{
    const DevScene &S = A.S;
    const int npb = pe - pa;
    const int nrx = npb * S.nc;
    const int txb = (nrx + 31) & ~31;  // first transmit thread, on a warp boundary
    if (CONCURRENT && txb + npb <= NT) {
        const int t = threadIdx.x;
        double u[3] = {0.0, 0.0, 0.0}, dref = 0.0;
        AntRec r;
        if (t < nrx) {
            const RxState &Rs = S.rx[(size_t)(pa + t / S.nc) * S.nc + t % S.nc];
            tile_ref(Rs.rx, xr, yr, u, dref, r);
        } else if (t >= txb && t < txb + npb) {
            tx_refs(sm, A, pa, t - txb, xr, yr);
        }
        __syncthreads();
        if (t < nrx) rx_combine(sm, A, pa, t, u, dref, r);
        return;
    }
    for (int t = threadIdx.x; t < npb; t += NT) tx_refs(sm, A, pa, t, xr, yr);
    __syncthreads();
    for (int t = threadIdx.x; t < nrx; t += NT) {
        const RxState &Rs = S.rx[(size_t)(pa + t / S.nc) * S.nc + t % S.nc];
        double u[3], dref;
        AntRec r;
        tile_ref(Rs.rx, xr, yr, u, dref, r);
        rx_combine(sm, A, pa, t, u, dref, r);
    }
}

// Wave sets a tile needs: for a heterogeneous sea state, the corners of every
// TL tile that the facets [ix0, ix1] x [iy0, iy1] fall in; otherwise set 0.
struct SetRange {
    int cx0, cx1, cy0, cy1;
};

__device__ __forceinline__ int het_tile(double p, double p0, double l, int ncorner)
{
    return min(max((int)floor((p - p0) / l), 0), ncorner - 2);
}

__device__ SetRange set_range(const DevScene &S, int ix0, int ix1, int iy0, int iy1)
{
    SetRange r{0, 0, 0, 0};
    if (S.het_ncx > 0) {
        ix1 = min(ix1, S.nx - 1);
        iy1 = min(iy1, S.ny - 1);
        r.cx0 = het_tile((ix0 + 0.5 - 0.5 * S.nx) * S.dx, S.het_x0, S.het_l, S.het_ncx);
        r.cx1 = het_tile((ix1 + 0.5 - 0.5 * S.nx) * S.dx, S.het_x0, S.het_l, S.het_ncx) + 1;
        r.cy0 = het_tile((iy0 + 0.5 - 0.5 * S.ny) * S.dx, S.het_y0, S.het_l, S.het_ncy);
        r.cy1 = het_tile((iy1 + 0.5 - 0.5 * S.ny) * S.dx, S.het_y0, S.het_l, S.het_ncy) + 1;
    }
    return r;
}

// Weight of corner (cx, cy) at a facet's rest position (Eq. 2): the product form
// sqrt((1 - w_x)(1 - w_y)) = sqrt(1 - w_x - w_y + w_x w_y) with each factor
// clamped at zero, which is Eq. 2 for the four corners of the facet's TL tile and
// zero for every other corner.
__device__ __forceinline__ float het_weight(const DevScene &S, int cx, int cy, int ix, int iy)
{
    const double x = (ix + 0.5 - 0.5 * S.nx) * S.dx, y = (iy + 0.5 - 0.5 * S.ny) * S.dx;
    const float ax = fmaxf(0.0f, 1.0f - (float)(fabs(S.het_x0 + cx * S.het_l - x) / S.het_l));
    const float ay = fmaxf(0.0f, 1.0f - (float)(fabs(S.het_y0 + cy * S.het_l - y) / S.het_l));
    return sqrtf(ax * ay);
}

// Taylor coefficients in time of the NF state fields of two facets (column ix,
// rows iya / iyb of the tile at (tx0, ty0)), accumulated over the wave components
// of every wave set in R (weighted per facet by Eq. 2 for a heterogeneous sea
// state). Per chunk of WCH components the real Taylor factors and the tile's
// column and row phasors (the rows times e^{-i omega t_c}) are staged in shared
// memory; each coefficient pair (orders 2p, 2p + 1) takes one FFMA2 per facet.
template <int NF, bool HET, int UNROLL>
__device__ void taylor_coeffs(const Smem &sm, const MixedArgs &A, int batch, int tx0, int ty0, int ix, int iya,
                              int iyb, const SetRange &R, float2 C[NF][kOrders])
{
    const DevScene &S = A.S;
    static_assert(kOrders % 2 == 0, "the contraction packs pairs of Taylor orders");
    constexpr int KP = kOrders / 2;  // order pairs
    // accumulators packed over order pairs (2p, 2p + 1), one set per facet
    float2 ca[NF][KP], cb[NF][KP];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int p = 0; p < KP; ++p) ca[f][p] = cb[f][p] = make_float2(0.0f, 0.0f);
    const int nw = S.nw;
    const int ixc = min(ix, S.nx - 1), iyac = min(iya, S.ny - 1), iybc = min(iyb, S.ny - 1);
    // the thread's column and rows within the staged tile phasors
    const int cx_s = ixc - tx0, ra_s = iyac - ty0, rb_s = iybc - ty0;
    for (int cy = R.cy0; cy <= R.cy1; ++cy)
        for (int cx = R.cx0; cx <= R.cx1; ++cx) {
            const int q = HET ? cy * S.het_ncx + cx : 0;
            const float wa = HET ? het_weight(S, cx, cy, ixc, iyac) : 1.0f;
            const float wb = HET ? het_weight(S, cx, cy, ixc, iybc) : 1.0f;
            const size_t qw = (size_t)q * nw;
            for (int m0 = 0; m0 < nw; m0 += WCH) {
                const int cnt = min(WCH, nw - m0);
                __syncthreads();
                // real Taylor factors of the chunk, as order pairs
                const float2 *src = reinterpret_cast<const float2 *>(A.cr) + (qw + m0) * NF * KP;
                for (int i = threadIdx.x; i < cnt * NF * KP; i += NT) sm.w[i] = src[i];
                // phasors of the chunk's components on the tile's columns and rows
                // (clamped to the scene at its edges); the rows carry e^{-i omega t_c}
                const float2 *tcb = A.tc + ((size_t)batch * S.n_sets + q) * nw + m0;
                for (int i = threadIdx.x; i < cnt * TX; i += NT) {
                    const int m = i / TX, c = min(tx0 + i % TX, S.nx - 1);
                    sm.wx[i] = __ldg(A.ex + (qw + m0 + m) * S.nx + c);
                }
                for (int i = threadIdx.x; i < cnt * TY; i += NT) {
                    const int m = i / TY, r = min(ty0 + i % TY, S.ny - 1);
                    const float2 y = __ldg(A.ey + (qw + m0 + m) * S.ny + r), t = __ldg(tcb + m);
                    sm.wy[i] = make_float2(y.x * t.x - y.y * t.y, y.x * t.y + y.y * t.x);
                }
                __syncthreads();
                if (wa == 0.0f && wb == 0.0f) continue;
#pragma unroll UNROLL
                for (int m = 0; m < cnt; ++m) {
                    const float2 e = sm.wx[m * TX + cx_s];
                    const float2 ya = sm.wy[m * TY + ra_s];
                    const float2 yb = sm.wy[m * TY + rb_s];
                    // Q of the two facets (and with its parts swapped)
                    float2 qa = make_float2(e.x * ya.x - e.y * ya.y, e.x * ya.y + e.y * ya.x);
                    float2 qb = make_float2(e.x * yb.x - e.y * yb.y, e.x * yb.y + e.y * yb.x);
                    if (HET) {
                        qa = mul2(qa, dup(wa));
                        qb = mul2(qb, dup(wb));
                    }
                    const float2 sa = make_float2(qa.y, qa.x), sb = make_float2(qb.y, qb.x);
                    const float2 *wm = sm.w + m * NF * KP;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const bool real = f == 0 || f >= 5;  // c_f real: (Q_r, Q_i), else (Q_i, Q_r)
#pragma unroll
                        for (int p = 0; p < KP; ++p) {
                            const float2 w = wm[f * KP + p];
                            ca[f][p] = fma2(w, real ? qa : sa, ca[f][p]);
                            cb[f][p] = fma2(w, real ? qb : sb, cb[f][p]);
                        }
                    }
                }
            }
        }
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int p = 0; p < KP; ++p) {
            C[f][2 * p] = make_float2(ca[f][p].x, cb[f][p].x);
            C[f][2 * p + 1] = make_float2(ca[f][p].y, cb[f][p].y);
        }
}

// Speckle of facet f in epoch e: Box-Muller on two Philox words (FP32).
__device__ __forceinline__ float2 speckle_f(uint64_t seed, uint32_t f, uint32_t e)
{
    U32x4 w = philox_stream(seed, kStreamSpeckle, f, e);
    float u1 = fmaf(__uint2float_rz(w.x), 2.3283064365386963e-10f, 2.3283064365386963e-10f);
    float u2 = __uint2float_rz(w.y) * 2.3283064365386963e-10f;
    float rad = sqrtf(-logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    return make_float2(rad * c, rad * s);
}

// Speckle of a facet at epoch e under the AR(1) model of Eq. 10 given its value
// z at epoch e_prev (e_prev < 0: none yet): one step of the recurrence from
// e - 1, otherwise a restart that runs the recurrence over the last spk_terms
// epochs (from epoch 0 when e < spk_terms; earlier terms weigh below 2^-40).
// beta = 0 is the independent draw of epoch e.
__device__ float2 speckle_epoch(const DevScene &S, uint32_t fid, int e, int e_prev, float2 z)
{
    if (S.spk_beta == 0.0) return speckle_f(S.speckle_seed, fid, (uint32_t)e);
    const float b = (float)S.spk_beta, q = (float)S.spk_q;
    int j = e;
    if (!(e_prev >= 0 && e == e_prev + 1)) {
        j = max(0, e - S.spk_terms + 1);
        z = j == 0 ? speckle_f(S.speckle_seed, fid, 0u) : make_float2(0.0f, 0.0f);
        if (j == 0) ++j;
    }
    for (; j <= e; ++j) {
        const float2 w = speckle_f(S.speckle_seed, fid, (uint32_t)j);
        z = make_float2(fmaf(b, z.x, q * w.x), fmaf(b, z.y, q * w.y));
    }
    return z;
}

template <typename OutT>
__device__ __forceinline__ void gadd(OutT *iq, size_t idx, float re, float im);
template <>
__device__ __forceinline__ void gadd<float>(float *iq, size_t idx, float re, float im)
{
    atomicAdd(reinterpret_cast<float2 *>(iq) + idx, make_float2(re, im));
}
template <>
__device__ __forceinline__ void gadd<double>(double *iq, size_t idx, float re, float im)
{
    atomicAdd(iq + 2 * idx, (double)re);
    atomicAdd(iq + 2 * idx + 1, (double)im);
}

template <typename OutT>
__device__ __forceinline__ void gadd1(OutT *iq, size_t idx, int comp, float v)
{
    atomicAdd(iq + 2 * idx + comp, (OutT)v);
}

// Warp pre-reduction of the lanes' 8 complex taps at bins kb .. kb + 7 into a
// 16-bin window. Each lane writes its taps into its own column of the warp
// buffer (rows = bins relative to the warp's lowest bin; the buffer is all zero
// between calls); within a row the lane's column is rotated by 4 x row so that
// the 16 lanes of a half-warp always store to 16 distinct bank pairs whatever
// their rows. Lane (w, half) then sums half of bin row w with vector loads (rows
// beyond the warp's span are skipped), the halves combine by one shuffle, and one
// shared atomic per (bin, component) adds the window to the CTA range tile (a
// global atomic outside it). Lanes whose bins spread over more than 8 bins fall
// back to direct atomics.
template <typename OutT>
__device__ __forceinline__ void warp_scatter(float *buf, float2 *tile_c, int tile_base, int kb, bool valid,
                                             const float h[8], float sr, float si, int nr, OutT *grow,
                                             unsigned int *flags)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int kmin = __reduce_min_sync(FULL, valid ? kb : INT_MAX);
    if (kmin == INT_MAX) return;
    const int kmax = __reduce_max_sync(FULL, valid ? kb : INT_MIN);
    if (kmax - kmin <= SBINS - 8) {
        const int o = kb - kmin;
        const int ll = lane & 15;
        const int hb = lane < 16 ? 0 : SHALF;
        const int rot = (ll - 4 * o) & 15;
        // column of row o + j is hb + 2 ((rot - 4 j) & 15): four distinct values
        float *col[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) col[m] = buf + hb + 2 * ((rot - 4 * m) & 15) + o * SROW;
        if (valid) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                *reinterpret_cast<float2 *>(col[j & 3] + j * SROW) = make_float2(h[j] * sr, h[j] * si);
        }
        __syncwarp();
        const int w = lane >> 1, half = lane & 1;
        float ar = 0.0f, ai = 0.0f;
        if (w < kmax - kmin + 8) {
            const float4 *rp = reinterpret_cast<const float4 *>(buf + w * SROW + half * SHALF);
            float4 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = rp[q];
            // packed (re, im) pairwise sums: short dependency chains after the loads
            float2 c[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) c[q] = add2(make_float2(v[q].x, v[q].y), make_float2(v[q].z, v[q].w));
            const float2 sum =
                add2(add2(add2(c[0], c[1]), add2(c[2], c[3])), add2(add2(c[4], c[5]), add2(c[6], c[7])));
            ar = sum.x;
            ai = sum.y;
        }
        ar += __shfl_xor_sync(FULL, ar, 1);
        ai += __shfl_xor_sync(FULL, ai, 1);
        __syncwarp();
        if (valid) {
#pragma unroll
            for (int j = 0; j < 8; ++j) *reinterpret_cast<float2 *>(col[j & 3] + j * SROW) = make_float2(0.f, 0.f);
        }
        const float val = half ? ai : ar;
        const int k = kmin + w;
        if (val != 0.0f && k >= 0 && k < nr) {
            const int tw = k - tile_base;
            if (tw >= 0 && tw < WT) {
                atomicAdd(reinterpret_cast<float *>(tile_c + tw) + half, val);
            } else {
                gadd1<OutT>(grow, (size_t)k, half, val);
                atomicAdd(flags + 2, 1u);
            }
        }
    } else if (valid) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int k = kb + j;
            if (k < 0 || k >= nr || h[j] == 0.0f) continue;
            int tw = k - tile_base;
            if (tw >= 0 && tw < WT) {
                atomicAdd(&tile_c[tw].x, h[j] * sr);
                atomicAdd(&tile_c[tw].y, h[j] * si);
            } else {
                gadd<OutT>(grow, (size_t)k, h[j] * sr, h[j] * si);
                atomicAdd(flags + 2, 1u);
            }
        }
    }
}

// Warp pre-reduction of both facets of every lane in one pass. The facets sit
// in adjacent rows, so facet b's taps start at most one bin away from facet a's:
// each lane combines them into 9 complex values at bins k0 .. k0 + 8 (k0 the lower
// of the two first bins) and writes those into its rotated column as above. The
// pass needs every lane's first bins within one of each other and all lanes' k0
// within 7 bins; otherwise it returns false and the caller reduces the facets one
// at a time.
// Window of one pair reduction, decided as soon as the bins are known (the warp
// reductions then overlap the rest of the per-channel arithmetic).
struct PairPlan {
    int kmin;  // first bin of the warp window; INT_MAX when no facet of the warp is valid
    int span;  // rows of the window in use
    bool ok;   // the single-pass form applies
};

__device__ __forceinline__ PairPlan plan_pair(int kba, int kbb, bool va, bool vb)
{
    const unsigned FULL = 0xffffffffu;
    if (!va) kba = kbb;
    if (!vb) kbb = kba;
    const bool valid = va || vb;
    const int k0 = min(kba, kbb);
    PairPlan pl;
    pl.kmin = __reduce_min_sync(FULL, valid ? k0 : INT_MAX);
    pl.span = 0;
    pl.ok = true;
    if (pl.kmin == INT_MAX) return pl;
    // one reduction serves the window check: the lane's row offset, or a value
    // beyond the window when its two facets' first bins are more than one apart
    const int omax = __reduce_max_sync(FULL, valid ? (abs(kbb - kba) > 1 ? 1 << 20 : k0 - pl.kmin) : 0);
    pl.ok = omax <= SBINS - 9;
    pl.span = omax + 9;
    return pl;
}

template <typename OutT>
__device__ __forceinline__ void warp_scatter_pair(const PairPlan &pl, float *buf, float2 *tile_c, int tile_base,
                                                  int kba, int kbb, bool va, bool vb, const float ha[8],
                                                  const float hb[8], float2 vre, float2 vim, int nr, OutT *grow,
                                                  unsigned int *flags)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    // a masked facet contributes nothing and takes the other facet's bins
    float sra = vre.x, sia = vim.x, srb = vre.y, sib = vim.y;
    if (!va) {
        sra = sia = 0.0f;
        kba = kbb;
    }
    if (!vb) {
        srb = sib = 0.0f;
        kbb = kba;
    }
    const bool valid = va || vb;
    const int k0 = min(kba, kbb);
    const int kmin = pl.kmin;
    const int o = k0 - kmin;
    const int ll = lane & 15;
    const int hbase = lane < 16 ? 0 : SHALF;
    const int rot = (ll - 4 * o) & 15;
    float *col[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) col[m] = buf + hbase + 2 * ((rot - 4 * m) & 15) + o * SROW;
    if (valid) {
        const bool sa = kba != k0, sb = kbb != k0;  // the facet starts one bin above k0
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const float a = sa ? (j > 0 ? ha[j - 1] : 0.0f) : (j < 8 ? ha[j] : 0.0f);
            const float b = sb ? (j > 0 ? hb[j - 1] : 0.0f) : (j < 8 ? hb[j] : 0.0f);
            // (re, im) of the bin as one packed pair: b (srb, sib) + a (sra, sia)
            *reinterpret_cast<float2 *>(col[j & 3] + j * SROW) =
                fma2(dup(b), make_float2(srb, sib), mul2(dup(a), make_float2(sra, sia)));
        }
    }
    __syncwarp();
    const int w = lane >> 1, half = lane & 1;
    float ar = 0.0f, ai = 0.0f;
    if (w < pl.span) {
        const float4 *rp = reinterpret_cast<const float4 *>(buf + w * SROW + half * SHALF);
        float4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = rp[q];
        float2 c[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) c[q] = add2(make_float2(v[q].x, v[q].y), make_float2(v[q].z, v[q].w));
        const float2 sum =
            add2(add2(add2(c[0], c[1]), add2(c[2], c[3])), add2(add2(c[4], c[5]), add2(c[6], c[7])));
        ar = sum.x;
        ai = sum.y;
    }
    ar += __shfl_xor_sync(FULL, ar, 1);
    ai += __shfl_xor_sync(FULL, ai, 1);
    __syncwarp();
    if (valid) {
#pragma unroll
        for (int j = 0; j < 9; ++j) *reinterpret_cast<float2 *>(col[j & 3] + j * SROW) = make_float2(0.f, 0.f);
    }
    const float val = half ? ai : ar;
    const int k = kmin + w;
    if (val != 0.0f) {
        const int tw = k - tile_base;
        if ((unsigned)tw < (unsigned)WT) {
            // bins outside [0, nr) are dropped when the tile is flushed
            atomicAdd(reinterpret_cast<float *>(tile_c + tw) + half, val);
        } else if (k >= 0 && k < nr) {
            gadd1<OutT>(grow, (size_t)k, half, val);
            atomicAdd(flags + 2, 1u);
        }
    }
}

struct FacetGeo {
    float xi_y;          // y offset from the tile reference point (exact)
    float fj;            // row offset index
    float base, cu, cv;  // NRCS base and current (cell values or uniform)
    float base_area;     // NRCS base x facet area
    float amp_static;    // sqrt(base x area): the amplitude factor of a static surface
    float2 z;            // speckle of the current epoch
    int epoch;           // epoch the speckle belongs to
    uint32_t fid;
    int cell;            // cell index (per-cell fields) or -1
    bool valid;
};

// Forward sink: warp pre-reduction into the CTA range tile of the channel.
template <typename OutT>
struct ScatterSink {
    static constexpr bool kProbe = false;
    float *stage;
    float2 *tiles;    // [kTileBufs][nc][WT]
    OutT *iq;
    int n0, np;
    size_t cstride;   // elements between channels of the IQ
    float2 *tiles_p;  // the current pulse's range tiles, [nc][WT]
    OutT *iq_p;       // the current pulse's IQ row of channel 0
    PairPlan plan;
    // per-pulse bases, so that a channel adds one offset to each
    __device__ __forceinline__ void set_pulse(const MixedArgs &A, int n, int buf)
    {
        tiles_p = tiles + buf * A.S.nc * WT;
        iq_p = iq + 2 * (size_t)(n - n0) * A.S.nr;
    }
    // the bins of the channel's two facets are known: plan the warp window
    __device__ __forceinline__ void prepare(int kba, int kbb, bool va, bool vb) { plan = plan_pair(kba, kbb, va, vb); }
    // the two facets' taps and values: one warp reduction for both, or one each
    // when the single-pass form does not apply
    __device__ __forceinline__ void put2(const MixedArgs &A, int ch, int kbase, int kba, int kbb, const float ha[8],
                                         const float hb[8], float2 vre, float2 vim, float2, float2, float, bool va,
                                         bool vb)
    {
        if (plan.kmin == INT_MAX) return;
        float2 *tile_c = tiles_p + ch * WT;
        const int tile_base = kbase - WT_LO;
        OutT *grow = iq_p + ch * cstride;
        if (plan.ok) {
            warp_scatter_pair<OutT>(plan, stage, tile_c, tile_base, kba, kbb, va, vb, ha, hb, vre, vim, A.S.nr, grow,
                                    A.S.flags);
            return;
        }
        warp_scatter<OutT>(stage, tile_c, tile_base, kba, va, ha, vre.x, vim.x, A.S.nr, grow, A.S.flags);
        warp_scatter<OutT>(stage, tile_c, tile_base, kbb, vb, hb, vre.y, vim.y, A.S.nr, grow, A.S.flags);
    }
};

// Outputs of the index probe, indexed by facet grid position; pulses count
// from the first pulse of the probed window.
struct ProbeOut {
    int *bins;        // [np][nc][ny][nx] first range bin of the facet's taps (k0 - 3; k0 for the box)
    float2 *speckle;  // [np][ny][nx] speckle draw of the pulse's coherence epoch
    uint4 *words;     // [np][ny][nx] Philox4x32-10 words that draw was made from
    int *cells;       // [ny][nx] cell index of the facet (-1 without per-cell fields)
};

// Probe sink: the forward work item runs unchanged up to the scatter, and this
// sink records the integer results the scatter would use (both facets' first
// bins per channel) and the speckle of the pulse instead of adding anything.
struct ProbeSink : ScatterSink<float> {
    static constexpr bool kProbe = true;
    ProbeOut out;
    int ix, iya, iyb;  // the thread's facets (iyb < 0: one facet per thread)
    int n, epoch;      // current pulse and its speckle epoch
    float2 za, zb;     // the facets' speckle draws of that epoch
    __device__ __forceinline__ void set_pulse(const MixedArgs &A, int n_, int buf)
    {
        ScatterSink<float>::set_pulse(A, n_, buf);
        n = n_;
    }
    __device__ __forceinline__ void prepare(int, int, bool, bool) {}
    __device__ __forceinline__ void one(const DevScene &S, int ch, int iy, int kb, float2 z)
    {
        const size_t plane = (size_t)S.nx * S.ny, at = (size_t)iy * S.nx + ix, p = (size_t)(n - n0);
        out.bins[(p * S.nc + ch) * plane + at] = kb;
        if (ch == 0) {
            out.speckle[p * plane + at] = z;
            const U32x4 w = philox_stream(S.speckle_seed, kStreamSpeckle, (uint32_t)at, (uint32_t)epoch);
            out.words[p * plane + at] = make_uint4(w.x, w.y, w.z, w.w);
        }
    }
    __device__ __forceinline__ void put2(const MixedArgs &A, int ch, int, int kba, int kbb, const float *,
                                         const float *, float2, float2, float2, float2, float, bool va, bool vb)
    {
        if (va) one(A.S, ch, iya, kba, za);
        if (vb && iyb >= 0) one(A.S, ch, iyb, kbb, zb);
    }
};

// Adjoint sink of the packed path: the gathers of the two facets, then the
// chain-rule terms accumulated as pairs.
template <typename InT>
struct GatherSink2 {
    const float2 *win;  // [nc][WA] residual window of the pulse
    const InT *resid;
    int n, n0, np;
    float2 as, au, av;  // per-facet accumulators, facet a in .x, facet b in .y
    __device__ __forceinline__ void prepare(int, int, bool, bool) {}
    __device__ __forceinline__ float2 gather(const MixedArgs &A, const float2 *wc, int tb, const InT *grow, int kb,
                                             const float h[8]) const
    {
        float gr = 0.0f, gi = 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = kb + j;
            const int w = k - tb;
            float2 v;
            if ((unsigned)w < (unsigned)WA)
                v = wc[w];
            else if (k >= 0 && k < A.S.nr)
                v = make_float2((float)grow[2 * k], (float)grow[2 * k + 1]);
            else
                v = make_float2(0.f, 0.f);
            gr = fmaf(h[j], v.x, gr);
            gi = fmaf(h[j], v.y, gi);
        }
        return make_float2(gr, gi);
    }
    __device__ __forceinline__ void put2(const MixedArgs &A, int ch, int kbase, int kba, int kbb, const float ha[8],
                                         const float hb[8], float2 vre, float2 vim, float2 qx, float2 qy, float k0t,
                                         bool, bool)
    {
        const float2 *wc = win + ch * WA;
        const int tb = kbase - WA_LO;
        const InT *grow = resid + 2 * ((size_t)ch * np + (n - n0)) * A.S.nr;
        float2 ga, gb;
        const int k0 = min(kba, kbb), w0 = k0 - tb;
        if (abs(kbb - kba) <= 1 && w0 >= 0 && w0 + 8 < WA) {
            // both facets' bins lie in k0 .. k0 + 8 inside the window: read the 9
            // residual values once and gather both facets from them
            const bool sa = kba != k0, sb = kbb != k0;
            float2 v[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) v[j] = wc[w0 + j];
            float gar = 0.0f, gai = 0.0f, gbr = 0.0f, gbi = 0.0f;
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const float a = sa ? (j > 0 ? ha[j - 1] : 0.0f) : (j < 8 ? ha[j] : 0.0f);
                const float b = sb ? (j > 0 ? hb[j - 1] : 0.0f) : (j < 8 ? hb[j] : 0.0f);
                gar = fmaf(a, v[j].x, gar);
                gai = fmaf(a, v[j].y, gai);
                gbr = fmaf(b, v[j].x, gbr);
                gbi = fmaf(b, v[j].y, gbi);
            }
            ga = make_float2(gar, gai);
            gb = make_float2(gbr, gbi);
        } else {
            ga = gather(A, wc, tb, grow, kba, ha);
            gb = gather(A, wc, tb, grow, kbb, hb);
        }
        const float2 GR = make_float2(ga.x, gb.x), GI = make_float2(ga.y, gb.y);
        const float2 re_gs = fma2(GR, vre, mul2(GI, vim));
        const float2 im_gs = fma2(GR, vim, neg2(mul2(GI, vre)));
        as = add2(as, re_gs);
        const float2 mk = dup(-k0t);
        au = fma2(mul2(mk, qx), im_gs, au);
        av = fma2(mul2(mk, qy), im_gs, av);
    }
};

// Pin a per-item value (derived once from FP64 scene constants) in a register:
// the empty asm hides how it was computed, so under register pressure the
// compiler keeps or spills it instead of recomputing it, with FP64 multiplies
// and conversions, inside the pulse loop.
__device__ __forceinline__ float pin(float v)
{
    asm volatile("" : "+f"(v));
    return v;
}
__device__ __forceinline__ float2 pin(float2 v) { return make_float2(pin(v.x), pin(v.y)); }

// Per-thread pair of facets (same column, adjacent rows) for the packed path.
struct PairGeo {
    float2 xi_y, fj, base_area, amp_static, cu, cv, zr, zi;
    bool va, vb;
};

__device__ __forceinline__ float2 horner2(const float2 c[kOrders], float2 t)
{
    float2 r = c[kOrders - 1];
#pragma unroll
    for (int o = kOrders - 2; o >= 0; --o) r = fma2(r, t, c[o]);
    return r;
}

// Complex gain of a u-v grid at direction cosines (u, v): bilinear between the
// four surrounding nodes, zero outside the grid.
__device__ __forceinline__ float2 lut_gain_f(const PatLutF &L, float u, float v)
{
    const float fu = (u - L.u0) * L.inv_du, fv = (v - L.v0) * L.inv_dv;
    if (!(fu >= 0.0f && fu <= L.umax && fv >= 0.0f && fv <= L.vmax)) return make_float2(0.0f, 0.0f);
    const int iu = min((int)fu, L.nu - 2), iv = min((int)fv, L.nv - 2);
    const float a = fu - (float)iu, b = fv - (float)iv;
    // node pairs (g[iv][iu], g[iv][iu + 1]) and (g[iv + 1][iu], g[iv + 1][iu + 1])
    const float4 *g = L.g + (size_t)iv * (L.nu - 1) + iu;
    const float4 r0 = __ldg(g), r1 = __ldg(g + (L.nu - 1));
    const float2 lo = make_float2(fmaf(a, r0.z - r0.x, r0.x), fmaf(a, r0.w - r0.y, r0.y));
    const float2 hi = make_float2(fmaf(a, r1.z - r1.x, r1.x), fmaf(a, r1.w - r1.y, r1.y));
    return make_float2(fmaf(b, hi.x - lo.x, lo.x), fmaf(b, hi.y - lo.y, lo.y));
}

// Gains of the two facets (pair) for antenna slot `slot`: the u-v grid when the
// scene has one for that antenna (re in .x/.y of gr, im in gi), else the
// analytic sinc^2 pattern (real).
__device__ __forceinline__ void pair_gain(const Smem &sm, const DevScene &S, const PolyArgs &P, int slot, float laz_l,
                                          float lel_l, float2 u, float2 v, float2 &gr, float2 &gi)
{
    if (S.lut_mask & (1u << slot)) {
        const PatLutF &L = sm.lut[slot];
        const float2 a = lut_gain_f(L, u.x, v.x), b = lut_gain_f(L, u.y, v.y);
        gr = make_float2(a.x, b.x);
        gi = make_float2(a.y, b.y);
    } else {
        gr = mul2(sinc2_2(P, mul2(dup(laz_l), u)), sinc2_2(P, mul2(dup(lel_l), v)));
        gi = make_float2(0.0f, 0.0f);
    }
}

// Forward contribution of the thread's two facets for pulse pi (chunk index),
// every channel, on FP32x2 pairs (facet a in .x, facet b in .y); transcendentals
// and integer work per element. fs holds the NF state fields of the two facets
// at this pulse. V selects the variants: with the Choppy Wave Model the facets sit at
// their rest positions moved by the horizontal displacement, their normal is the
// cross product of the displaced surface's tangents and their area scales with
// its vertical component; with u-v grids the pattern gains are complex.
template <int TAPS, int V, int CU, int NCC, bool SH3, typename Sink>
__device__ __forceinline__ void facet_pulse2(const Smem &sm, const MixedArgs &A, const PolyArgs &P, const PairGeo &G,
                                             const float2 fs[Var<V>::NF], int pi, float xi_x, float fi,
                                             Sink &sink)
{
    constexpr bool CWM = Var<V>::CWM, LUT = Var<V>::LUT;
    const DevScene &S = A.S;
    const int nc = NCC > 0 ? NCC : S.nc;  // compile-time channel count when NCC > 0
    const float2 one = make_float2(1.0f, 1.0f);
    const PulseRec PR = sm.pr[pi];
    const float2 eta = fs[0];
    const float2 sx = fs[1];
    const float2 sy = fs[2];
    float2 X0 = dup(xi_x), X1 = G.xi_y;
    float2 Dx, Dy, nvx, nvy, nvz, areaf;
    if constexpr (CWM) {
        Dx = fs[3];
        Dy = fs[4];
        const float2 jxx = fs[5], jxy = fs[6], jyy = fs[7];
        X0 = add2(X0, Dx);
        X1 = add2(X1, Dy);
        const float2 txx = add2(one, jxx), tyy = add2(one, jyy);
        // n = (1 + Jxx, Jxy, eta_x) x (Jxy, 1 + Jyy, eta_y)
        nvx = fma2(jxy, sy, neg2(mul2(sx, tyy)));
        nvy = fma2(sx, jxy, neg2(mul2(txx, sy)));
        nvz = fma2(txx, tyy, neg2(mul2(jxy, jxy)));
        areaf = make_float2(fmaxf(nvz.x, 0.0f), fmaxf(nvz.y, 0.0f));
    }
    const float2 b2 = fma2(X0, X0, fma2(X1, X1, mul2(eta, eta)));
    float2 nn;
    if constexpr (CWM)
        nn = fma2(nvx, nvx, fma2(nvy, nvy, mul2(nvz, nvz)));
    else
        nn = fma2(sx, sx, fma2(sy, sy, one));
    const float2 inv_n = make_float2(rsqrtf(nn.x), rsqrtf(nn.y));

    // transmit leg (shared by the channels)
    const AntRec2 T = dup_rec(sm.tx[pi]);
    const float2 at = fma2(T.ux, X0, fma2(T.uy, X1, mul2(T.uz, eta)));
    const float2 st = fma2(neg2(at), at, b2);
    const float2 qt = mul2(st, fma2(neg2(at), T.inv2R2, T.inv2R));
    const float2 dt = add2(at, qt);
    const float2 et = mul2(dt, T.invR);
    const float2 rho_t = fma2(et, et, sub2(one, et));
    const float2 ut = mul2(add2(T.u0, fma2(X0, T.aRx, fma2(X1, T.aRy, mul2(eta, T.aRz)))), rho_t);
    const float2 vt = mul2(add2(T.v0, fma2(X0, T.eRx, fma2(X1, T.eRy, mul2(eta, T.eRz)))), rho_t);
    float2 gt, gti;
    if constexpr (LUT)
        pair_gain(sm, S, P, 0, A.tx_laz_l, A.tx_lel_l, ut, vt, gt, gti);
    else
        gt = mul2(sinc2_2(P, mul2(dup(A.tx_laz_l), ut)), sinc2_2(P, mul2(dup(A.tx_lel_l), vt)));
    const float2 rt0 = mul2(fma2(X0, T.invR, T.ux), rho_t);
    const float2 rt1 = mul2(fma2(X1, T.invR, T.uy), rho_t);
    const float2 rt2 = mul2(fma2(eta, T.invR, T.uz), rho_t);
    // with u-v grids the transmit gain stays out of the real amplitude
    const float2 ampt = LUT ? mul2(T.ampr, rho_t) : mul2(mul2(gt, T.ampr), rho_t);

    const AntRec *RX = sm.rx + pi * nc;
    const ChanRec *CH = sm.ch + pi * nc;
    float2 gr_prev = make_float2(0.0f, 0.0f), amps_prev = make_float2(0.0f, 0.0f);
    // with the six-channel layout known at compile time, channels 1, 2 and 4, 5 are
    // the second and third phase centres of the antenna of channels 0 and 3 (5 m
    // apart): they take that channel's second-order range term, R / r and product
    // of the common amplitude factors. Between phase centres the facet's direction
    // changes by ~separation / R ~ 6e-6 rad, which moves the second-order term by
    // ~1e-8 m (1.5e-6 rad of phase) and R / r by ~3e-10.
    float2 qr_prev = make_float2(0.0f, 0.0f), rho_prev = make_float2(0.0f, 0.0f);
    float2 ampc_prev = make_float2(0.0f, 0.0f);
#pragma unroll CU
    for (int ch = 0; ch < nc; ++ch) {
        const bool pc = SH3 && (ch % 3 != 0);  // a later phase centre of the antenna (compile time)
        const AntRec2 R = dup_rec(RX[ch]);
        const ChanRec2 Q = dup_chan(CH[ch]);
        const float2 ar = fma2(R.ux, X0, fma2(R.uy, X1, mul2(R.uz, eta)));
        float2 qr = qr_prev;
        if (!pc) {
            const float2 sr_ = fma2(neg2(ar), ar, b2);
            qr = mul2(sr_, fma2(neg2(ar), R.inv2R2, R.inv2R));
        }
        qr_prev = qr;
        const float2 dr = add2(ar, qr);
        // range bins first: the warp window of the reduction is planned here, its
        // warp-wide reductions overlapping the pattern, NRCS and phase arithmetic
        const float2 p = fma2(add2(dt, dr), dup(A.inv_dr), Q.pfrac);
        const float2 kf = make_float2(floorf(p.x), floorf(p.y));
        const float2 fr = sub2(p, kf);
        const int kba = Q.kbase + (int)kf.x - (TAPS == 1 ? 0 : 3);
        const int kbb = Q.kbase + (int)kf.y - (TAPS == 1 ? 0 : 3);
        sink.prepare(kba, kbb, G.va, G.vb);
        float2 rho_r = rho_prev;
        if (!pc) {
            const float2 er = mul2(dr, R.invR);
            rho_r = fma2(er, er, sub2(one, er));
        }
        rho_prev = rho_r;
        float2 gr, gri;
        if constexpr (LUT) {
            const float2 ur = mul2(add2(R.u0, fma2(X0, R.aRx, fma2(X1, R.aRy, mul2(eta, R.aRz)))), rho_r);
            const float2 vr = mul2(add2(R.v0, fma2(X0, R.eRx, fma2(X1, R.eRy, mul2(eta, R.eRz)))), rho_r);
            pair_gain(sm, S, P, 1 + ch, A.rx_laz_l[ch], A.rx_lel_l[ch], ur, vr, gr, gri);
        } else if (SH3 ? (ch % 3 != 0) : ((S.rx_share >> ch) & 1u)) {
            // phase centre of the same receive antenna as channel ch - 1: same gain
            gr = gr_prev;
        } else {
            const float2 ur = mul2(add2(R.u0, fma2(X0, R.aRx, fma2(X1, R.aRy, mul2(eta, R.aRz)))), rho_r);
            const float2 vr = mul2(add2(R.v0, fma2(X0, R.eRx, fma2(X1, R.eRy, mul2(eta, R.eRz)))), rho_r);
            gr = mul2(sinc2_2(P, mul2(dup(A.rx_laz_l[ch]), ur)), sinc2_2(P, mul2(dup(A.rx_lel_l[ch]), vr)));
        }
        gr_prev = gr;
        const float2 qx = neg2(fma2(fma2(X0, R.invR, R.ux), rho_r, rt0));
        const float2 qy = neg2(fma2(fma2(X1, R.invR, R.uy), rho_r, rt1));
        const float2 qz = neg2(fma2(fma2(eta, R.invR, R.uz), rho_r, rt2));
        // sqrt(sigma0 A) = X rsqrt(X Q_z), X = base A (1 + m cos phi) max(0, n.Q) / |n| (x n_z with the CWM)
        float2 amp_s = G.amp_static;
        if (SH3 ? (ch % 3 != 0) : ((S.rx_share >> ch) & 1u)) {
            // phase centre of the previous channel's antenna: its Q direction differs
            // by ~(separation / R) ~ 6e-6 rad, the NRCS by < 4e-6 relative
            amp_s = amps_prev;
        } else if (!S.static_surface) {
            const float2 qh2 = fma2(qx, qx, mul2(qy, qy));
            // 1 / |Q_H| (clamped: Q_H = 0 gives cos phi = 0)
            const float2 rq = make_float2(rsqrtf(fmaxf(qh2.x, 1e-30f)), rsqrtf(fmaxf(qh2.y, 1e-30f)));
            const float2 cphi = mul2(fma2(dup(A.wcos), qx, mul2(dup(A.wsin), qy)), rq);
            float2 nq;
            if constexpr (CWM)
                nq = fma2(nvx, qx, fma2(nvy, qy, mul2(nvz, qz)));
            else
                nq = fma2(neg2(sx), qx, fma2(neg2(sy), qy, qz));
            const float2 nqp = make_float2(fmaxf(nq.x, 0.0f), fmaxf(nq.y, 0.0f));
            float2 X = mul2(mul2(G.base_area, fma2(dup(A.wind_mod), cphi, one)), mul2(nqp, inv_n));
            if constexpr (CWM) X = mul2(X, areaf);
            // X >= 0 and Q_z > 0: X rsqrt(X Q_z), clamped so that X = 0 gives 0
            const float2 Xq = mul2(X, qz);
            amp_s = mul2(X, make_float2(rsqrtf(fmaxf(Xq.x, 1e-30f)), rsqrtf(fmaxf(Xq.y, 1e-30f))));
        } else if constexpr (CWM) {
            amp_s = mul2(amp_s, make_float2(sqrtf(areaf.x), sqrtf(areaf.y)));
        }
        amps_prev = amp_s;
        float2 amp;
        if constexpr (LUT) {
            amp = mul2(mul2(amp_s, ampt), mul2(R.ampr, rho_r));
        } else {
            // amp_s G_t G_r Rbar_t Rbar_r / (r_t r_r): everything but the channel's
            // own Rbar_r / R_r is common to the phase centres of one antenna
            const float2 ampc = pc ? ampc_prev : mul2(mul2(mul2(amp_s, ampt), gr), rho_r);
            ampc_prev = ampc;
            amp = mul2(ampc, R.ampr);
        }
        const float2 vc = neg2(fma2(G.cu, qx, mul2(G.cv, qy)));
        float2 phi = fma2(dup(fi), Q.ax, Q.psi);
        phi = fma2(G.fj, Q.ay, phi);
        phi = fma2(Q.gam, eta, phi);
        if constexpr (CWM) {
            phi = fma2(dup(Q.gx), Dx, phi);
            phi = fma2(dup(Q.gy), Dy, phi);
        }
        phi = fma2(dup(-A.k0), add2(qt, qr), phi);
        phi = fma2(dup(-PR.k0t), vc, phi);
        const float2 kk = make_float2(rintf(phi.x * 0.15915494309189535f), rintf(phi.y * 0.15915494309189535f));
        phi = fma2(neg2(kk), dup(6.28125f), phi);
        phi = fma2(neg2(kk), dup(1.9353071795864769e-3f), phi);
        float sa, ca, sb, cb;
        __sincosf(phi.x, &sa, &ca);
        __sincosf(phi.y, &sb, &cb);
        const float2 sp = make_float2(sa, sb), cp = make_float2(ca, cb);
        float2 zr = mul2(amp, G.zr), zi = mul2(amp, G.zi);
        if constexpr (LUT) {
            // times the complex field weight G_t G_r
            const float2 wr = fma2(gt, gr, neg2(mul2(gti, gri)));
            const float2 wi = fma2(gt, gri, mul2(gti, gr));
            const float2 nr = fma2(zr, wr, neg2(mul2(zi, wi)));
            zi = fma2(zr, wi, mul2(zi, wr));
            zr = nr;
        }
        const float2 vre = fma2(zr, cp, neg2(mul2(zi, sp)));
        const float2 vim = fma2(zr, sp, mul2(zi, cp));
        float ha[8], hb[8];
        if (TAPS == 1) {
            ha[0] = hb[0] = 1.0f;
#pragma unroll
            for (int j = 1; j < 8; ++j) ha[j] = hb[j] = 0.0f;
        } else {
            const float2 t = fma2(dup(2.0f), fr, dup(-1.0f));
            const float2 t2 = mul2(t, t);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 ev = P.tap_e[j][kTapEven - 1];
#pragma unroll
                for (int d = kTapEven - 2; d >= 0; --d) ev = fma2(ev, t2, P.tap_e[j][d]);
                float2 od = P.tap_o[j][kTapOdd - 1];
#pragma unroll
                for (int d = kTapOdd - 2; d >= 0; --d) od = fma2(od, t2, P.tap_o[j][d]);
                const float2 lo = fma2(od, t, ev), hi = fma2(neg2(od), t, ev);
                ha[j] = lo.x;
                hb[j] = lo.y;
                ha[7 - j] = hi.x;
                hb[7 - j] = hi.y;
            }
        }
        sink.put2(A, ch, Q.kbase, kba, kbb, ha, hb, vre, vim, qx, qy, PR.k0t, G.va, G.vb);
    }
}

__device__ void facet_setup(const MixedArgs &A, int ix, int iy, int jref, FacetGeo &G)
{
    const DevScene &S = A.S;
    G.valid = ix < S.nx && iy < S.ny;
    G.fj = (float)(iy - jref);
    G.xi_y = (float)((iy - jref) * S.dx);
    G.fid = (uint32_t)min(iy, S.ny - 1) * (uint32_t)S.nx + (uint32_t)min(ix, S.nx - 1);
    double base = S.sigma0_base, cu = S.cur_u, cv = S.cur_v;
    G.cell = -1;
    if (S.ncx > 0) {
        double x = (min(ix, S.nx - 1) + 0.5 - 0.5 * S.nx) * S.dx;
        double y = (min(iy, S.ny - 1) + 0.5 - 0.5 * S.ny) * S.dx;
        int cx = (int)floor((x + 0.5 * S.nx * S.dx) / S.cell);
        int cy = (int)floor((y + 0.5 * S.ny * S.dx) / S.cell);
        cx = min(max(cx, 0), S.ncx - 1);
        cy = min(max(cy, 0), S.ncy - 1);
        int ci = cy * S.ncx + cx;
        G.cell = ci;
        if (S.cell_sigma0) base = S.cell_sigma0[ci];
        if (S.cell_uv) {
            cu = S.cell_uv[2 * ci];
            cv = S.cell_uv[2 * ci + 1];
        }
    }
    G.base = (float)base;
    G.base_area = (float)(base * S.area);
    G.amp_static = (float)sqrt(base * S.area);
    G.cu = (float)cu;
    G.cv = (float)cv;
    G.epoch = -1;
    G.z = make_float2(0.f, 0.f);
}

// Tile geometry of one work item: 32 columns x ty rows (ty = 8 or 16) of the
// scene's facet grid; warp w handles rows w and (ty = 16) w + 8.
struct ItemGeo {
    int tx0, ty0, ty, pa, pe, batch;
};

__device__ __forceinline__ ItemGeo item_geo(const MixedArgs &A, int tile, int batch, int ty, int n0, int np)
{
    ItemGeo g;
    const int tiles_x = (A.S.nx + TX - 1) / TX;
    g.tx0 = (tile % tiles_x) * TX;
    g.ty0 = (tile / tiles_x) * ty;
    g.ty = ty;
    g.batch = batch;
    g.pa = max(n0, batch * A.nb);
    g.pe = min(n0 + np, (batch + 1) * A.nb);
    return g;
}

// FP32 copies of the scene's u-v grid descriptors in shared memory (the caller
// synchronises before they are read).
__device__ __forceinline__ void stage_luts(const Smem &sm, const DevScene &S)
{
    for (int i = threadIdx.x; i <= S.nc; i += NT) {
        PatLutF f{};
        if (S.lut_mask & (1u << i)) {
            const PatLut &L = S.luts[i];
            f.g = L.g32;
            f.nu = L.nu;
            f.nv = L.nv;
            f.u0 = (float)L.u0;
            f.inv_du = (float)L.inv_du;
            f.v0 = (float)L.v0;
            f.inv_dv = (float)L.inv_dv;
            f.umax = (float)(L.nu - 1);
            f.vmax = (float)(L.nv - 1);
        }
        sm.lut[i] = f;
    }
}

// Taylor coefficients of the item's two facets per thread, or zero for a static
// surface. UNROLL unrolls the component loop to overlap the shared-memory reads of
// consecutive components (measured best: 4, in the echo kernels and in the
// standalone generator at three CTAs per SM).
template <int NF, int UNROLL = 1>
__device__ __forceinline__ void item_coeffs(const Smem &sm, const MixedArgs &A, int batch, int tx0, int ty0, int ty,
                                            int ix, int iya, int iyb, float2 C[NF][kOrders])
{
    const DevScene &S = A.S;
    if (!S.static_surface && S.nw > 0) {
        const SetRange R = set_range(S, tx0, tx0 + TX - 1, ty0, ty0 + ty - 1);
        if (S.het_ncx > 0)
            taylor_coeffs<NF, true, UNROLL>(sm, A, batch, tx0, ty0, ix, iya, iyb, R, C);
        else
            taylor_coeffs<NF, false, UNROLL>(sm, A, batch, tx0, ty0, ix, iya, iyb, R, C);
    } else {
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int o = 0; o < kOrders; ++o) C[f][o] = make_float2(0.0f, 0.0f);
    }
}

// Keep the item's Taylor coefficients where the pulse loop reads them: a
// thread-private column of shared memory for the linear surface (frees 36
// registers for the per-channel arithmetic; two orders per 128-bit load),
// registers for the CWM.
template <int NF>
__device__ __forceinline__ void store_coeffs(const Smem &sm, const float2 C[NF][kOrders])
{
    if constexpr (NF == 3) {
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int q = 0; q < kOrders / 2; ++q)
                reinterpret_cast<float4 *>(sm.coef)[(f * (kOrders / 2) + q) * NT + threadIdx.x] =
                    make_float4(C[f][2 * q].x, C[f][2 * q].y, C[f][2 * q + 1].x, C[f][2 * q + 1].y);
    }
}

// State fields of the two facets at time offset tau (Horner in time).
template <int NF>
__device__ __forceinline__ void eval_state(const Smem &sm, const float2 C[NF][kOrders], float tau, float2 st[NF])
{
    const float2 t = dup(tau);
    if constexpr (NF == 3) {
        const float4 *cs = reinterpret_cast<const float4 *>(sm.coef) + threadIdx.x;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            float2 c[kOrders];
#pragma unroll
            for (int q = 0; q < kOrders / 2; ++q) {
                const float4 v = cs[(f * (kOrders / 2) + q) * NT];
                c[2 * q] = make_float2(v.x, v.y);
                c[2 * q + 1] = make_float2(v.z, v.w);
            }
            st[f] = horner2(c, t);
        }
    } else {
#pragma unroll
        for (int f = 0; f < NF; ++f) st[f] = horner2(C[f], t);
    }
}

// One forward work item (tile x pulse batch) of one scene. Every thread of the
// CTA calls it; it starts and ends with the CTA's range tiles all zero.
template <int TAPS, typename OutT, int V, int NCC = 0, bool SH3 = false, typename Sink = ScatterSink<OutT>>
__device__ void forward_item(const Smem &sm, const MixedArgs &A, const PolyArgs &P, const ItemGeo &I, int n0, int np,
                             OutT *iq, const ProbeOut *probe = nullptr)
{
    constexpr int NF = Var<V>::NF;
    const DevScene &S = A.S;
    const int nc = S.nc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool two = I.ty > NWARP;
    const int ix = I.tx0 + lane;
    const int iref = I.tx0 + TX / 2, jref = I.ty0 + I.ty / 2;
    const double xr = (iref + 0.5 - 0.5 * S.nx) * S.dx;
    const double yr = (jref + 0.5 - 0.5 * S.ny) * S.dx;
    const float xi_x = pin((float)((ix - iref) * S.dx));
    const float fi = pin((float)(ix - iref));

    FacetGeo ga, gb;
    // rows of the thread's two facets: adjacent rows 2w, 2w + 1 (16-row tiles; their
    // range bins differ by at most one, so the warp reduces both in one pass), or
    // row w alone (8-row tiles)
    const int iya = I.ty0 + (two ? 2 * warp : warp), iyb = iya + 1;
    facet_setup(A, ix, iya, jref, ga);
    facet_setup(A, ix, iyb, jref, gb);
    float2 C[NF][kOrders];
    item_coeffs<NF, 4>(sm, A, I.batch, I.tx0, I.ty0, I.ty, ix, iya, two ? iyb : iya, C);
    __syncthreads();
    // the warp buffers share memory with the wave-table chunk: clear them
    for (int i = threadIdx.x; i < NWARP * SBINS * SROW; i += NT) sm.stage[i] = 0.0f;
    if (Var<V>::LUT) stage_luts(sm, S);
    __syncthreads();

    Sink sink;
    sink.stage = sm.stage + warp * SBINS * SROW;
    sink.tiles = sm.tile;
    sink.iq = iq;
    sink.n0 = n0;
    sink.np = np;
    sink.cstride = 2 * (size_t)np * S.nr;
    if constexpr (Sink::kProbe) {
        sink.out = *probe;
        sink.ix = ix;
        sink.iya = iya;
        sink.iyb = two ? iyb : -1;
        if (ga.valid) probe->cells[(size_t)iya * S.nx + ix] = ga.cell;
        if (two && gb.valid) probe->cells[(size_t)iyb * S.nx + ix] = gb.cell;
    }
    // pack the two facets: .x = row w, .y = row w + 8 (a copy of .x, masked off, for 8-row tiles)
    PairGeo G;
    const FacetGeo &gq = two ? gb : ga;
    G.xi_y = pin(make_float2(ga.xi_y, gq.xi_y));
    G.fj = pin(make_float2(ga.fj, gq.fj));
    G.base_area = pin(make_float2(ga.base_area, gq.base_area));
    G.amp_static = pin(make_float2(ga.amp_static, gq.amp_static));
    G.cu = pin(make_float2(ga.cu, gq.cu));
    G.cv = pin(make_float2(ga.cv, gq.cv));
    G.va = ga.valid;
    G.vb = two && gb.valid;
    store_coeffs<NF>(sm, C);
    for (int c0 = I.pa; c0 < I.pe; c0 += NBR) {
        const int ce = min(c0 + NBR, I.pe);
        __syncthreads();  // the previous chunk's flush is done with the records
        build_refs<false>(sm, A, c0, ce, xr, yr);
        __syncthreads();
        for (int n = c0; n < ce;) {
            // speckle of the epoch of pulse n, then the chunk's pulses of that epoch
            const int e = sm.pr[n - c0].epoch;
            const int ne = S.epoch_pulses > 0 ? min(ce, (e + 1) * S.epoch_pulses) : ce;
            if (e != ga.epoch) {
                ga.z = speckle_epoch(S, ga.fid, e, ga.epoch, ga.z);
                ga.epoch = e;
            }
            if (two && e != gb.epoch) {
                gb.z = speckle_epoch(S, gb.fid, e, gb.epoch, gb.z);
                gb.epoch = e;
            }
            G.zr = make_float2(ga.z.x, two ? gb.z.x : 0.0f);
            G.zi = make_float2(ga.z.y, two ? gb.z.y : 0.0f);
            if constexpr (Sink::kProbe) {
                sink.epoch = e;
                sink.za = ga.z;
                sink.zb = gb.z;
            }
            for (; n < ne; ++n) {
                const int pi = n - c0;
                sink.set_pulse(A, n, n & (kTileBufs - 1));
                float2 st[NF];
                eval_state<NF>(sm, C, sm.pr[pi].tau, st);
                facet_pulse2<TAPS, V, (SH3 ? (Var<V>::CWM ? 3 : 6) : Var<V>::FWD_CU), NCC, SH3>(sm, A, P, G, st, pi, xi_x, fi, sink);
                // flush the range tiles of pulse pairs (one barrier per two pulses;
                // a tile is reused four pulses later, after at least one more barrier)
                if ((pi & 1) || n == ce - 1) {
                    __syncthreads();
                    for (int p = (pi & 1) ? n - 1 : n; p <= n; ++p) {
                        const int pp = p - c0, pb = p & (kTileBufs - 1);
                        for (int i = threadIdx.x; i < nc * WT; i += NT) {
                            int ch = i / WT, w = i % WT;
                            float2 *slot = sm.tile + (pb * nc + ch) * WT + w;
                            float2 v = *slot;
                            *slot = make_float2(0.f, 0.f);
                            int k = sm.ch[pp * nc + ch].kbase - WT_LO + w;
                            if ((v.x != 0.0f || v.y != 0.0f) && k >= 0 && k < S.nr)
                                gadd<OutT>(iq + 2 * ((size_t)ch * np + (p - n0)) * S.nr, (size_t)k, v.x, v.y);
                        }
                    }
                }
            }
        }
    }
    // every tile has been flushed; make sure every thread is done with the tiles
    // and the records before they are reused
    __syncthreads();
}

__device__ __forceinline__ void clear_smem(const Smem &sm, int nc)
{
    for (int i = threadIdx.x; i < kTileBufs * nc * WT; i += NT) sm.tile[i] = make_float2(0.f, 0.f);
    for (int i = threadIdx.x; i < NWARP * SBINS * SROW; i += NT) sm.stage[i] = 0.0f;
}

template <int TAPS, typename OutT, int V, int NCC, bool SH3>
__global__ void __launch_bounds__(NT, Var<V>::MIN_BLOCKS)
    accumulate_mixed_kernel(MixedArgs A, PolyArgs P, int n0, int np, int b0, int ty, OutT *iq)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem sm = carve(smem_raw, A.S.nc, Var<V>::NF);
    const ItemGeo I = item_geo(A, blockIdx.x, b0 + blockIdx.y, ty, n0, np);
    if (I.pa >= I.pe) return;
    clear_smem(sm, A.S.nc);
    forward_item<TAPS, OutT, V, NCC, SH3>(sm, A, P, I, n0, np, iq);
}

// Index probe: the accumulator's work items with the probe sink (no output is
// accumulated; see ProbeSink).
template <int TAPS, int V, int NCC, bool SH3>
__global__ void __launch_bounds__(NT, Var<V>::MIN_BLOCKS)
    probe_mixed_kernel(MixedArgs A, PolyArgs P, int n0, int np, int b0, ProbeOut out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem sm = carve(smem_raw, A.S.nc, Var<V>::NF);
    const ItemGeo I = item_geo(A, blockIdx.x, b0 + blockIdx.y, TY, n0, np);
    if (I.pa >= I.pe) return;
    clear_smem(sm, A.S.nc);
    forward_item<TAPS, float, V, NCC, SH3, ProbeSink>(sm, A, P, I, n0, np, nullptr, &out);
}

// Work list of a batched launch: scene s owns items [start[s], start[s + 1]);
// item i of scene s is (batch = i / tiles[s], tile = i % tiles[s]) so that
// consecutive items share the pulse batch (IQ rows stay in L2).
struct BatchItems {
    const MixedArgs *args;  // [n] per-scene arguments (device)
    const int *start;       // [n + 1] prefix sums of items
    const int *tiles;       // [n] tiles per batch
    const int *ty;          // [n] tile height (8 or 16), chosen by the autotuner
    const int *order;       // [n] processing order of the scenes (largest first)
    float *const *iq;       // [n] IQ outputs (complex64)
    int n;
    int total;
};

// Persistent batched forward launch: a fixed pool of CTAs pulls work items from
// a global counter until the list is exhausted (no waiting on other CTAs). The
// scene arguments of the current item are copied to shared memory.
template <int TAPS, int V, int NCC, bool SH3 = false>
__global__ void __launch_bounds__(NT, Var<V>::MIN_BLOCKS)
    batch_mixed_kernel(BatchItems B, PolyArgs P, unsigned int *counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ MixedArgs args;
    __shared__ int s_item, s_scene;
    const int nc_max = B.args[0].S.nc;  // layout sized for the first scene's channels (all equal)
    const Smem sm = carve(smem_raw, nc_max, Var<V>::NF);
    int cur_scene = -1;
    clear_smem(sm, nc_max);
    for (;;) {
        if (threadIdx.x == 0) {
            int it = (int)atomicAdd(counter, 1u);
            s_item = it;
            int sc = -1;
            if (it < B.total) {
                // scenes are laid out in processing order: find k with start[k] <= it < start[k+1]
                int lo = 0, hi = B.n - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (B.start[mid] <= it)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                sc = lo;
            }
            s_scene = sc;
        }
        __syncthreads();
        const int it = s_item, k = s_scene;
        if (it >= B.total) break;
        const int scene = B.order[k];
        if (scene != cur_scene) {
            const int *src = reinterpret_cast<const int *>(B.args + scene);
            int *dst = reinterpret_cast<int *>(&args);
            for (int i = threadIdx.x; i < (int)(sizeof(MixedArgs) / 4); i += NT) dst[i] = src[i];
            cur_scene = scene;
        }
        __syncthreads();
        const int local = it - B.start[k];
        const int tiles = B.tiles[scene];
        const ItemGeo I = item_geo(args, local % tiles, local / tiles, B.ty[scene], 0, args.S.np_total);
        if (I.pa < I.pe) forward_item<TAPS, float, V, NCC, SH3>(sm, args, P, I, 0, args.S.np_total, B.iq[scene]);
        __syncthreads();
    }
}

// Per-cell gradient of one facet, reduced over the warp's lanes of the same cell
// (lanes along x: cells form contiguous lane segments) and added by the segment
// head with FP64 atomics.
__device__ __forceinline__ void add_cell_grads(const FacetGeo &G, float as, float au, float av, double *g_sigma,
                                               double *g_uv)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool ok = G.valid && G.cell >= 0;
    const int cell = ok ? G.cell : -1;
    double vs = (ok && G.base > 0.0f) ? (double)as / (double)G.base : 0.0;
    double vu = ok ? 2.0 * (double)au : 0.0;
    double vv = ok ? 2.0 * (double)av : 0.0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        double ts = __shfl_down_sync(FULL, vs, d);
        double tu = __shfl_down_sync(FULL, vu, d);
        double tv = __shfl_down_sync(FULL, vv, d);
        int tc = __shfl_down_sync(FULL, cell, d);
        if (lane + d < 32 && tc == cell) {
            vs += ts;
            vu += tu;
            vv += tv;
        }
    }
    const int prev = __shfl_up_sync(FULL, cell, 1);
    const bool head = (lane == 0 || prev != cell);
    if (head && cell >= 0) {
        if (g_sigma) atomicAdd(g_sigma + cell, vs);
        if (g_uv) {
            atomicAdd(g_uv + 2 * cell, vu);
            atomicAdd(g_uv + 2 * cell + 1, vv);
        }
    }
}

template <int TAPS, typename InT, int V, int NCC, bool SH3>
__global__ void __launch_bounds__(NT, Var<V>::MIN_BLOCKS)
    adjoint_mixed_kernel(MixedArgs A, PolyArgs P, int n0, int np, int b0, const InT *resid, double *g_sigma,
                         double *g_uv)
{
    constexpr int NF = Var<V>::NF;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DevScene &S = A.S;
    const int nc = S.nc;
    const Smem sm = carve(smem_raw, nc, NF);
    const int tiles_x = (S.nx + TX - 1) / TX;
    const int tx0 = (blockIdx.x % tiles_x) * TX;
    const int ty0 = (blockIdx.x / tiles_x) * TY;
    const int batch = b0 + blockIdx.y;
    const int pa = max(n0, batch * A.nb);
    const int pe = min(n0 + np, (batch + 1) * A.nb);
    if (pa >= pe) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ix = tx0 + lane;
    const int iref = tx0 + TX / 2, jref = ty0 + TY / 2;
    const double xr = (iref + 0.5 - 0.5 * S.nx) * S.dx;
    const double yr = (jref + 0.5 - 0.5 * S.ny) * S.dx;
    const float xi_x = pin((float)((ix - iref) * S.dx));
    const float fi = pin((float)(ix - iref));

    FacetGeo ga, gb;
    const int iya = ty0 + 2 * warp, iyb = iya + 1;  // the forward path's facet rows
    facet_setup(A, ix, iya, jref, ga);
    facet_setup(A, ix, iyb, jref, gb);
    float2 C[NF][kOrders];
    item_coeffs<NF, 4>(sm, A, batch, tx0, ty0, TY, ix, iya, iyb, C);
    if (Var<V>::LUT) {
        __syncthreads();
        stage_luts(sm, S);
    }
    PairGeo G;
    G.xi_y = pin(make_float2(ga.xi_y, gb.xi_y));
    G.fj = pin(make_float2(ga.fj, gb.fj));
    G.base_area = pin(make_float2(ga.base_area, gb.base_area));
    G.amp_static = pin(make_float2(ga.amp_static, gb.amp_static));
    G.cu = pin(make_float2(ga.cu, gb.cu));
    G.cv = pin(make_float2(ga.cv, gb.cv));
    G.va = ga.valid;
    G.vb = gb.valid;
    store_coeffs<NF>(sm, C);
    GatherSink2<InT> sink;
    sink.win = sm.tile;
    sink.resid = resid;
    sink.n0 = n0;
    sink.np = np;
    sink.as = sink.au = sink.av = make_float2(0.0f, 0.0f);
    for (int c0 = pa; c0 < pe; c0 += NBR) {
        const int ce = min(c0 + NBR, pe);
        __syncthreads();  // the previous chunk is done with the records
        build_refs<true>(sm, A, c0, ce, xr, yr);
        for (int n = c0; n < ce;) {
            __syncthreads();
            // speckle of the epoch of pulse n, then the chunk's pulses of that epoch
            const int e = sm.pr[n - c0].epoch;
            const int ne = S.epoch_pulses > 0 ? min(ce, (e + 1) * S.epoch_pulses) : ce;
            if (e != ga.epoch) {
                ga.z = speckle_epoch(S, ga.fid, e, ga.epoch, ga.z);
                ga.epoch = e;
            }
            if (e != gb.epoch) {
                gb.z = speckle_epoch(S, gb.fid, e, gb.epoch, gb.z);
                gb.epoch = e;
            }
            G.zr = make_float2(ga.z.x, gb.z.x);
            G.zi = make_float2(ga.z.y, gb.z.y);
            for (; n < ne; ++n) {
                const int pi = n - c0;
                __syncthreads();  // the previous pulse is done with the residual window
                // residual window of this pulse, every channel
                for (int i = threadIdx.x; i < nc * WA; i += NT) {
                    int ch = i / WA, w = i % WA;
                    int k = sm.ch[pi * nc + ch].kbase - WA_LO + w;
                    float2 v = make_float2(0.f, 0.f);
                    if (k >= 0 && k < S.nr) {
                        const InT *r = resid + 2 * (((size_t)ch * np + (n - n0)) * S.nr + k);
                        v = make_float2((float)r[0], (float)r[1]);
                    }
                    sm.tile[i] = v;
                }
                __syncthreads();
                sink.n = n;
                float2 st[NF];
                eval_state<NF>(sm, C, sm.pr[pi].tau, st);
                facet_pulse2<TAPS, V, (NCC > 0 ? NCC : 1), NCC, SH3>(sm, A, P, G, st, pi, xi_x, fi, sink);
            }
        }
    }
    add_cell_grads(ga, sink.as.x, sink.au.x, sink.av.x, g_sigma, g_uv);
    add_cell_grads(gb, sink.as.y, sink.au.y, sink.av.y, g_sigma, g_uv);
}

// Facet generator of the mixed path: same Taylor expansion, states written out
// ([np][NF][n_facets]).
template <int V>
__global__ void __launch_bounds__(NT, Var<V>::CWM ? 1 : 3)
    generate_mixed_kernel(MixedArgs A, int n0, int np, int b0, float *state)
{
    constexpr int NF = Var<V>::NF;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DevScene &S = A.S;
    const Smem sm = carve(smem_raw, S.nc, NF);
    const int tiles_x = (S.nx + TX - 1) / TX;
    const int tx0 = (blockIdx.x % tiles_x) * TX;
    const int ty0 = (blockIdx.x / tiles_x) * TY;
    const int batch = b0 + blockIdx.y;
    const int pa = max(n0, batch * A.nb);
    const int pe = min(n0 + np, (batch + 1) * A.nb);
    if (pa >= pe) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ix = tx0 + lane;
    const int iya = ty0 + 2 * warp, iyb = iya + 1;
    const bool va = ix < S.nx && iya < S.ny, vb = ix < S.nx && iyb < S.ny;
    float2 C[NF][kOrders];
    item_coeffs<NF, 4>(sm, A, batch, tx0, ty0, TY, ix, iya, iyb, C);
    // the window's pulse times, staged in the (now free) chunk region
    float *tau_s = reinterpret_cast<float *>(sm.w);
    __syncthreads();
    for (int i = threadIdx.x; i < pe - pa; i += NT) tau_s[i] = A.tau[pa + i];
    __syncthreads();
    const int64_t nf = (int64_t)S.nx * S.ny;
    const int64_t fa = (int64_t)iya * S.nx + ix, fb = (int64_t)iyb * S.nx + ix;
    // states are written once and not read back here: streaming stores (pulse
    // loop unrolled by 8: 1 % faster than 4 at a full 256-pulse window)
#pragma unroll 8
    for (int n = pa; n < pe; ++n) {
        const float2 t = dup(tau_s[n - pa]);
        float *o = state + (size_t)(n - n0) * NF * nf;
        float2 st[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) st[q] = horner2(C[q], t);
        if (va) {
#pragma unroll
            for (int q = 0; q < NF; ++q) __stcs(o + q * nf + fa, st[q].x);
        }
        if (vb) {
#pragma unroll
            for (int q = 0; q < NF; ++q) __stcs(o + q * nf + fb, st[q].y);
        }
    }
}

// Facet generator with tensor-memory-accelerator stores (three-field states,
// nx % 4 == 0): the same contraction and Horner evaluation as
// generate_mixed_kernel, but each pulse's [3][TY][TX] box of states is written to
// shared memory and sent to the state array by one bulk tensor store, so the
// threads issue no global stores and no 64-bit address arithmetic. Groups of
// kGenGroup pulses rotate through three staging slots: before the barrier that
// closes group g the issuing thread waits until the stores of group g - 2 have
// read their slot, which group g + 1 reuses. The tensor map clips the box at the
// scene's edges; the wave-table chunk of the contraction shares the staging
// region (it is dead by then).
constexpr int kGenGroup = 4;          // pulses per staging slot
constexpr int kGenBox = 3 * TY * TX;  // floats of one pulse's box
constexpr int kGenSlots = 3;

// staging slots (128-byte aligned inside the region) and the window's pulse times
__host__ __device__ constexpr int gen_tma_bytes()
{
    return 128 + kGenSlots * kGenGroup * kGenBox * 4 + NBG * 4 > wave_chunk_bytes(3)
               ? 128 + kGenSlots * kGenGroup * kGenBox * 4 + NBG * 4
               : wave_chunk_bytes(3);
}

// the threads' shared-memory writes become visible to the bulk copies
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, const float *src, int x, int y, int z, int w)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(src));
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(s), "r"(x), "r"(y), "r"(z), "r"(w)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// every committed group but the newest has finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all_but_one()
{
    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}

// every committed group is complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(NT, 3)
    generate_tma_kernel(const __grid_constant__ CUtensorMap map, MixedArgs A, int n0, int np, int b0)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const DevScene &S = A.S;
    const Smem sm = carve(smem_raw, S.nc, 3);
    const int tiles_x = (S.nx + TX - 1) / TX;
    const int tx0 = (blockIdx.x % tiles_x) * TX;
    const int ty0 = (blockIdx.x / tiles_x) * TY;
    const int batch = b0 + blockIdx.y;
    const int pa = max(n0, batch * A.nb);
    const int pe = min(n0 + np, (batch + 1) * A.nb);
    if (pa >= pe) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ix = tx0 + lane;
    const int iya = ty0 + 2 * warp, iyb = iya + 1;
    float2 C[3][kOrders];
    item_coeffs<3, 4>(sm, A, batch, tx0, ty0, TY, ix, iya, iyb, C);
    const unsigned raw_s = static_cast<unsigned>(__cvta_generic_to_shared(smem_raw));
    float *slots = reinterpret_cast<float *>(smem_raw + ((128 - (raw_s & 127)) & 127));
    float *tau_s = slots + kGenSlots * kGenGroup * kGenBox;
    __syncthreads();  // the chunk region is dead
    for (int i = threadIdx.x; i < pe - pa; i += NT) tau_s[i] = A.tau[pa + i];
    __syncthreads();
    const int at = 2 * warp * TX + lane;  // facet a in the box; facet b one row below
    int slot = 0;
    for (int n = pa; n < pe; n += kGenGroup) {
        const int cnt = min(kGenGroup, pe - n);
        float *bx = slots + slot * kGenGroup * kGenBox;
#pragma unroll
        for (int p = 0; p < kGenGroup; ++p) {
            if (p < cnt) {
                const float2 t = dup(tau_s[n - pa + p]);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float2 v = horner2(C[q], t);
                    bx[p * kGenBox + q * TX * TY + at] = v.x;
                    bx[p * kGenBox + q * TX * TY + at + TX] = v.y;
                }
            }
        }
        fence_async_shared();
        if (threadIdx.x == 0) bulk_wait_read_all_but_one();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int p = 0; p < cnt; ++p) tma_store_4d(&map, bx + p * kGenBox, tx0, ty0, 0, n + p - n0);
            bulk_commit();
        }
        slot = slot == kGenSlots - 1 ? 0 : slot + 1;
    }
    if (threadIdx.x == 0) bulk_wait_all();
}

MixedArgs make_args(const DevScene &S, const MixedTables &M)
{
    MixedArgs A;
    A.S = S;
    A.ex = M.ex;
    A.ey = M.ey;
    A.tc = M.tc;
    A.cr = M.cr;
    A.tau = M.tau;
    A.nb = M.nb;
    A.n_batches = M.n_batches;
    A.tx_laz_l = (float)(S.tx_laz * S.inv_lambda);
    A.tx_lel_l = (float)(S.tx_lel * S.inv_lambda);
    for (int c = 0; c < kMaxCh; ++c) {
        A.rx_laz_l[c] = c < S.nc ? (float)(S.rx_laz[c] * S.inv_lambda) : 0.0f;
        A.rx_lel_l[c] = c < S.nc ? (float)(S.rx_lel[c] * S.inv_lambda) : 0.0f;
    }
    A.wcos = (float)S.wcos;
    A.wsin = (float)S.wsin;
    A.wind_mod = (float)S.wind_mod;
    A.area = (float)S.area;
    A.k0 = (float)S.k0;
    A.inv_dr = (float)S.inv_dr;
    return A;
}

PolyArgs make_poly(const MixedTables &M)
{
    PolyArgs P;
    // even / odd parts of taps j and 7 - j, averaged so that the symmetry is exact
    for (int j = 0; j < 4; ++j) {
        for (int k = 0; k < kTapEven; ++k) {
            const float c = 0.5f * (M.tap[j][2 * k] + M.tap[7 - j][2 * k]);
            P.tap_e[j][k] = make_float2(c, c);
        }
        for (int k = 0; k < kTapOdd; ++k) {
            const float c = 0.5f * (M.tap[j][2 * k + 1] - M.tap[7 - j][2 * k + 1]);
            P.tap_o[j][k] = make_float2(c, c);
        }
    }
    for (int d = 0; d <= kSincDeg; ++d) P.sinc2[d] = make_float2(M.sinc2[d], M.sinc2[d]);
    return P;
}

template <typename K>
cudaError_t prep(K kernel, int bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Grid of a launch over pulses [n0, n0 + np): (tiles, pulse batches), split into
// launches of at most 65535 batches; f(bb, grid) issues one launch.
template <typename F>
cudaError_t over_batches(const DevScene &S, const MixedTables &M, int ty, int n0, int np, F f)
{
    const int tiles = ((S.nx + TX - 1) / TX) * ((S.ny + ty - 1) / ty);
    const int b0 = n0 / M.nb, b1 = (n0 + np - 1) / M.nb;
    for (int bb = b0; bb <= b1; bb += 65535) {
        const int cnt = min(65535, b1 - bb + 1);
        cudaError_t e = f(bb, dim3(tiles, cnt));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int TAPS, typename OutT, int V, int NCC, bool SH3 = false>
cudaError_t accumulate_nc(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np, OutT *iq)
{
    const MixedArgs A = make_args(S, M);
    const PolyArgs P = make_poly(M);
    const int bytes = layout(S.nc, Var<V>::NF).total;
    cudaError_t e = prep(accumulate_mixed_kernel<TAPS, OutT, V, NCC, SH3>, bytes);
    if (e != cudaSuccess) return e;
    return over_batches(S, M, TY, n0, np, [&](int bb, dim3 grid) {
        accumulate_mixed_kernel<TAPS, OutT, V, NCC, SH3><<<grid, NT, bytes, st>>>(A, P, n0, np, bb, TY, iq);
        return cudaGetLastError();
    });
}

// Six channels (two receive antennas of three phase centres) get their own
// instantiation with a compile-time channel count (0.7 % faster than the loop
// over the scene's count); other counts and the box taps use the general one.
template <int TAPS, typename OutT, int V>
cudaError_t accumulate_t(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np, OutT *iq)
{
    if constexpr (TAPS == 8) {
        if (S.nc == 6 && S.rx_share == 0x36u) return accumulate_nc<TAPS, OutT, V, 6, true>(S, M, st, n0, np, iq);
        if (S.nc == 6) return accumulate_nc<TAPS, OutT, V, 6>(S, M, st, n0, np, iq);
    }
    return accumulate_nc<TAPS, OutT, V, 0>(S, M, st, n0, np, iq);
}

template <int TAPS, int V, int NCC, bool SH3 = false>
cudaError_t probe_nc(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np, const ProbeOut &out)
{
    const MixedArgs A = make_args(S, M);
    const PolyArgs P = make_poly(M);
    const int bytes = layout(S.nc, Var<V>::NF).total;
    cudaError_t e = prep(probe_mixed_kernel<TAPS, V, NCC, SH3>, bytes);
    if (e != cudaSuccess) return e;
    return over_batches(S, M, TY, n0, np, [&](int bb, dim3 grid) {
        probe_mixed_kernel<TAPS, V, NCC, SH3><<<grid, NT, bytes, st>>>(A, P, n0, np, bb, out);
        return cudaGetLastError();
    });
}

// Same instantiation choice as accumulate_t, so that the probe runs the code of
// the accumulator the scene uses.
template <int TAPS, int V>
cudaError_t probe_t(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np, const ProbeOut &out)
{
    if constexpr (TAPS == 8) {
        if (S.nc == 6 && S.rx_share == 0x36u) return probe_nc<TAPS, V, 6, true>(S, M, st, n0, np, out);
        if (S.nc == 6) return probe_nc<TAPS, V, 6>(S, M, st, n0, np, out);
    }
    return probe_nc<TAPS, V, 0>(S, M, st, n0, np, out);
}

template <int TAPS, typename InT, int V, int NCC, bool SH3 = false>
cudaError_t adjoint_nc(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np, const InT *resid,
                       double *g_sigma, double *g_uv)
{
    const MixedArgs A = make_args(S, M);
    const PolyArgs P = make_poly(M);
    const int bytes = layout(S.nc, Var<V>::NF).total;
    cudaError_t e = prep(adjoint_mixed_kernel<TAPS, InT, V, NCC, SH3>, bytes);
    if (e != cudaSuccess) return e;
    return over_batches(S, M, TY, n0, np, [&](int bb, dim3 grid) {
        adjoint_mixed_kernel<TAPS, InT, V, NCC, SH3><<<grid, NT, bytes, st>>>(A, P, n0, np, bb, resid, g_sigma, g_uv);
        return cudaGetLastError();
    });
}

// The adjoint's channel loop runs fully unrolled for six channels (two antennas
// of three phase centres, 4 % faster), otherwise over the scene's channel count.
template <int TAPS, typename InT, int V>
cudaError_t adjoint_t(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np, const InT *resid,
                      double *g_sigma, double *g_uv)
{
    if constexpr (TAPS == 8) {
        if (S.nc == 6 && S.rx_share == 0x36u) return adjoint_nc<TAPS, InT, V, 6, true>(S, M, st, n0, np, resid, g_sigma, g_uv);
        if (S.nc == 6) return adjoint_nc<TAPS, InT, V, 6>(S, M, st, n0, np, resid, g_sigma, g_uv);
    }
    return adjoint_nc<TAPS, InT, V, 0>(S, M, st, n0, np, resid, g_sigma, g_uv);
}

// Launchers of one variant V.
template <int V>
struct MixedLaunch {
    static cudaError_t generate(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                                float *state)
    {
        const MixedArgs A = make_args(S, M);
        if constexpr (Var<V>::NF == 3) {
            alignas(64) CUtensorMap map;
            if (np > 0 && M.nb <= NBG && S.nx % 4 == 0 && reinterpret_cast<uintptr_t>(state) % 16 == 0 &&
                encode_state_map(&map, state, S.nx, S.ny, 3, np, TX, TY) == cudaSuccess) {
                const int bytes = gen_tma_bytes();
                cudaError_t e = prep(generate_tma_kernel, bytes);
                if (e != cudaSuccess) return e;
                return over_batches(S, M, TY, n0, np, [&](int bb, dim3 grid) {
                    generate_tma_kernel<<<grid, NT, bytes, st>>>(map, A, n0, np, bb);
                    return cudaGetLastError();
                });
            }
        }
        // the kernel uses only the wave-table chunk: the rest of the SM's shared
        // memory stays L1 for the wave phasor tables it reads
        const int bytes = layout(S.nc, Var<V>::NF).w + wave_chunk_bytes(Var<V>::NF);
        cudaError_t e = prep(generate_mixed_kernel<V>, bytes);
        if (e != cudaSuccess) return e;
        return over_batches(S, M, TY, n0, np, [&](int bb, dim3 grid) {
            generate_mixed_kernel<V><<<grid, NT, bytes, st>>>(A, n0, np, bb, state);
            return cudaGetLastError();
        });
    }

    static cudaError_t accumulate(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np, void *iq,
                                  harm_dtype dtype)
    {
        if (dtype == HARM_C64)
            return S.taps == 1 ? accumulate_t<1, float, V>(S, M, st, n0, np, (float *)iq)
                               : accumulate_t<8, float, V>(S, M, st, n0, np, (float *)iq);
        return S.taps == 1 ? accumulate_t<1, double, V>(S, M, st, n0, np, (double *)iq)
                           : accumulate_t<8, double, V>(S, M, st, n0, np, (double *)iq);
    }

    static cudaError_t probe(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                             const ProbeOut &out)
    {
        return S.taps == 1 ? probe_t<1, V>(S, M, st, n0, np, out) : probe_t<8, V>(S, M, st, n0, np, out);
    }

    static cudaError_t adjoint(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                               const void *resid, harm_dtype dtype, double *g_sigma, double *g_uv)
    {
        if (dtype == HARM_C64)
            return S.taps == 1 ? adjoint_t<1, float, V>(S, M, st, n0, np, (const float *)resid, g_sigma, g_uv)
                               : adjoint_t<8, float, V>(S, M, st, n0, np, (const float *)resid, g_sigma, g_uv);
        return S.taps == 1 ? adjoint_t<1, double, V>(S, M, st, n0, np, (const double *)resid, g_sigma, g_uv)
                           : adjoint_t<8, double, V>(S, M, st, n0, np, (const double *)resid, g_sigma, g_uv);
    }

    static cudaError_t batch(const BatchLaunch &L, cudaStream_t st)
    {
        BatchItems B;
        B.args = reinterpret_cast<const MixedArgs *>(L.args);
        B.start = L.start;
        B.tiles = L.tiles;
        B.ty = L.ty;
        B.order = L.order;
        B.iq = L.iq;
        B.n = L.n;
        B.total = L.total;
        const PolyArgs P = make_poly(*L.poly);
        const int bytes = layout(L.nc, Var<V>::NF).total;
        cudaError_t e;
        if (L.taps == 1) {
            if ((e = prep(batch_mixed_kernel<1, V, 0>, bytes)) != cudaSuccess) return e;
            batch_mixed_kernel<1, V, 0><<<L.ctas, NT, bytes, st>>>(B, P, L.counter);
        } else if (L.nc == 6 && L.share3) {  // compile-time channel layout, as for single scenes
            if ((e = prep(batch_mixed_kernel<8, V, 6, true>, bytes)) != cudaSuccess) return e;
            batch_mixed_kernel<8, V, 6, true><<<L.ctas, NT, bytes, st>>>(B, P, L.counter);
        } else if (L.nc == 6) {
            if ((e = prep(batch_mixed_kernel<8, V, 6>, bytes)) != cudaSuccess) return e;
            batch_mixed_kernel<8, V, 6><<<L.ctas, NT, bytes, st>>>(B, P, L.counter);
        } else {
            if ((e = prep(batch_mixed_kernel<8, V, 0>, bytes)) != cudaSuccess) return e;
            batch_mixed_kernel<8, V, 0><<<L.ctas, NT, bytes, st>>>(B, P, L.counter);
        }
        return cudaGetLastError();
    }
};

}  // namespace

// The translation unit that includes this file with HARM_MIXED_VARIANT defined
// exports the launchers of that variant under names ending in _v<V>.
#ifdef HARM_MIXED_VARIANT
#define HARM_CAT2(a, b) a##b
#define HARM_CAT(a, b) HARM_CAT2(a, b)
cudaError_t HARM_CAT(mixed_generate_v, HARM_MIXED_VARIANT)(const DevScene &S, const MixedTables &M, cudaStream_t st,
                                                           int n0, int np, float *state)
{
    return MixedLaunch<HARM_MIXED_VARIANT>::generate(S, M, st, n0, np, state);
}
cudaError_t HARM_CAT(mixed_accumulate_v, HARM_MIXED_VARIANT)(const DevScene &S, const MixedTables &M,
                                                             cudaStream_t st, int n0, int np, void *iq,
                                                             harm_dtype dtype)
{
    return MixedLaunch<HARM_MIXED_VARIANT>::accumulate(S, M, st, n0, np, iq, dtype);
}
cudaError_t HARM_CAT(mixed_adjoint_v, HARM_MIXED_VARIANT)(const DevScene &S, const MixedTables &M, cudaStream_t st,
                                                          int n0, int np, const void *resid, harm_dtype dtype,
                                                          double *g_sigma, double *g_uv)
{
    return MixedLaunch<HARM_MIXED_VARIANT>::adjoint(S, M, st, n0, np, resid, dtype, g_sigma, g_uv);
}
cudaError_t HARM_CAT(mixed_batch_v, HARM_MIXED_VARIANT)(const BatchLaunch &L, cudaStream_t st)
{
    return MixedLaunch<HARM_MIXED_VARIANT>::batch(L, st);
}
cudaError_t HARM_CAT(mixed_probe_v, HARM_MIXED_VARIANT)(const DevScene &S, const MixedTables &M, cudaStream_t st,
                                                        int n0, int np, int *bins, void *speckle, void *words,
                                                        int *cells)
{
    ProbeOut out;
    out.bins = bins;
    out.speckle = reinterpret_cast<float2 *>(speckle);
    out.words = reinterpret_cast<uint4 *>(words);
    out.cells = cells;
    return MixedLaunch<HARM_MIXED_VARIANT>::probe(S, M, st, n0, np, out);
}
#endif

}  // namespace harm
