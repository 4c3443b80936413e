// Mixed-precision echo path: FP64 only for per-pulse platform state, the
// reference bistatic range and each tile's range offset; FP32 for the per-facet
// geometry, antenna patterns, NRCS, phase, interpolation taps and accumulation.
//
// Work decomposition (one CTA = a 32 x 16 facet tile x a 128-pulse batch):
//  1. Facet generator: the surface of the tile over the batch is expanded in time
//     about the batch centre, eta(t_c + tau) = sum_m eta_m tau^m (m <= 5), with
//     the Taylor coefficients eta_m = Re sum_w Q_w E_{w,m} accumulated over the
//     wave components (register-blocked FP32 contraction, separable phasors Q).
//  2. FP64 tile references, per 32-pulse chunk: for every pulse and antenna, the
//     range R from the antenna to the tile's reference point on the mean surface,
//     its unit vector and the tile's reduced reference phase and range-bin offset.
//     Per facet, r - R is a small offset that FP32 carries to ~1e-8 m:
//        r - R = a + (b - a^2) / (2R) + (a^3 - a b) / (2R^2),  a = u.xi, b = |xi|^2
//     for the facet offset xi from the reference point; the linear phase term
//     K0 (u_t + u_r).xi is split into exactly-reduced lattice steps.
//  3. For each pulse: each thread evaluates its two facets (rows w and w + 8 of
//     the tile) together in packed FP32x2 arithmetic: Horner in time, then per
//     channel the contribution (Eq. 3, 4, 16) and its 8 Kaiser-sinc taps
//     (polynomials in the fractional bin). The warp pre-reduces its 32 lanes'
//     taps: each lane writes its taps into its own (row-rotated) column of a
//     per-warp [16 bin x 32 lane] shared buffer at the rows of its bins, then each
//     lane sums one bin-row half with vector loads; one shared atomic per
//     (bin, component) adds the warp's window to the CTA range tile, which is
//     flushed to the IQ with one vector atomic per bin and channel.
//  The adjoint runs the same per-pulse arithmetic and gathers the residual
//  through the same taps instead of scattering.
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
constexpr int NBR = 32;       // pulses per chunk of FP64 tile references
constexpr int NBG = 128;      // pulses per work item (time-Taylor window of the generator)
constexpr int WCH = 128;      // wave components per shared-memory chunk
constexpr int SROW = 72;      // floats per bin row of the warp buffer (2 halves of 32 + pad)
constexpr int SHALF = 36;     // float offset of lanes 16..31 in a row
constexpr int SBINS = 16;     // bins per warp window
constexpr float kPiF = 3.14159265358979f;

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
    float pad0, pad1;
};

struct __align__(16) PulseRec {
    float tau, k0t;
    int epoch;
    int pad;
};

// The same references with every value duplicated into a pair (v, v): the
// forward path evaluates two facets per thread with packed FP32x2 arithmetic and
// reads each reference as one 64-bit operand.
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
    int pad0;
    float2 pad1;
};

struct MixedArgs {
    DevScene S;
    const float2 *ex, *ey, *wt;
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
struct PolyArgs {
    float2 tap[8][kTapDeg + 1];
    float2 sinc2[kSincDeg + 1];
};

// Shared-memory layout (bytes), sized for nc channels.
struct Layout {
    int w, tile, tx, rx, ch, pr, txd, stage, total;
};

// The wave-table chunk (generator phase) and the warp buffers (pulse loop) are
// never live at the same time and share one region; the warp buffers are
// cleared after the generator phase.
__host__ __device__ inline Layout layout(int nc, bool dup)
{
    Layout L;
    int o = 0;
    const int wbytes = WCH * 3 * kOrders * 8;
    const int sbytes = NWARP * SBINS * SROW * 4;
    L.w = o;
    L.stage = o;
    o += wbytes > sbytes ? wbytes : sbytes;
    L.tile = o;  o += 2 * nc * WT * 8;
    L.tx = o;    o += NBR * (int)(dup ? sizeof(AntRec2) : sizeof(AntRec));
    L.rx = o;    o += NBR * nc * (int)(dup ? sizeof(AntRec2) : sizeof(AntRec));
    L.ch = o;    o += NBR * nc * (int)(dup ? sizeof(ChanRec2) : sizeof(ChanRec));
    L.pr = o;    o += NBR * (int)sizeof(PulseRec);
    L.txd = o;   o += NBR * 4 * 8;
    L.total = o;
    return L;
}

struct Smem {
    float2 *w;       // [WCH][3][kOrders]
    float2 *tile;    // [2][nc][WT]
    AntRec *tx;      // [NBR]          (scalar layout: adjoint)
    AntRec *rx;      // [NBR][nc]
    ChanRec *ch;     // [NBR][nc]
    AntRec2 *tx2;    // [NBR]          (pair layout: forward, same memory)
    AntRec2 *rx2;    // [NBR][nc]
    ChanRec2 *ch2;   // [NBR][nc]
    PulseRec *pr;    // [NBR]
    double *txd;     // [NBR][4]
    float *stage;    // [NWARP][SBINS][SROW]
};

__device__ __forceinline__ Smem carve(unsigned char *raw, int nc, bool dup)
{
    Layout L = layout(nc, dup);
    Smem s;
    s.w = reinterpret_cast<float2 *>(raw + L.w);
    s.tile = reinterpret_cast<float2 *>(raw + L.tile);
    s.tx = reinterpret_cast<AntRec *>(raw + L.tx);
    s.rx = reinterpret_cast<AntRec *>(raw + L.rx);
    s.ch = reinterpret_cast<ChanRec *>(raw + L.ch);
    s.tx2 = reinterpret_cast<AntRec2 *>(raw + L.tx);
    s.rx2 = reinterpret_cast<AntRec2 *>(raw + L.rx);
    s.ch2 = reinterpret_cast<ChanRec2 *>(raw + L.ch);
    s.pr = reinterpret_cast<PulseRec *>(raw + L.pr);
    s.txd = reinterpret_cast<double *>(raw + L.txd);
    s.stage = reinterpret_cast<float *>(raw + L.stage);
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

// Reduce an FP32 phase to [-pi, pi] with a two-part 2 pi (Cody-Waite).
__device__ __forceinline__ float reduce_phase(float a)
{
    float k = rintf(a * 0.15915494309189535f);
    a = fmaf(-k, 6.28125f, a);
    a = fmaf(-k, 1.9353071795864769e-3f, a);
    return a;
}

// FP64 tile reference of one antenna (state A) for the tile reference point
// X = (xr, yr, 0): D = X - p, R = |D|, u = D / R, and the stable offset
// R - |p| = (|X|^2 - 2 p.X) / (R + |p|).
__device__ void tile_ref(const AntState &A, double xr, double yr, double u[3], double &dref, AntRec &o)
{
    double D[3] = {xr - A.p[0], yr - A.p[1], -A.p[2]};
    double R = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    double iR = 1.0 / R;
    for (int i = 0; i < 3; ++i) u[i] = D[i] * iR;
    double xx = xr * xr + yr * yr;
    dref = (xx - 2.0 * (A.p[0] * xr + A.p[1] * yr)) / (R + A.rref);
    o.ux = (float)u[0];
    o.uy = (float)u[1];
    o.uz = (float)u[2];
    o.invR = (float)iR;
    o.inv2R = (float)(0.5 * iR);
    o.inv2R2 = (float)(0.5 * iR * iR);
    o.u0 = (float)(u[0] * A.a[0] + u[1] * A.a[1] + u[2] * A.a[2]);
    o.v0 = (float)(u[0] * A.e[0] + u[1] * A.e[1] + u[2] * A.e[2]);
    o.aRx = (float)(A.a[0] * iR);
    o.aRy = (float)(A.a[1] * iR);
    o.aRz = (float)(A.a[2] * iR);
    o.ampr = (float)(A.rref * iR);
    o.eRx = (float)(A.e[0] * iR);
    o.eRy = (float)(A.e[1] * iR);
    o.eRz = (float)(A.e[2] * iR);
    o.pad = 0.0f;
}

__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }

__device__ __forceinline__ AntRec2 dup_rec(const AntRec &r)
{
    AntRec2 o;
    o.ux = dup(r.ux); o.uy = dup(r.uy); o.uz = dup(r.uz); o.invR = dup(r.invR);
    o.inv2R = dup(r.inv2R); o.inv2R2 = dup(r.inv2R2); o.u0 = dup(r.u0); o.v0 = dup(r.v0);
    o.aRx = dup(r.aRx); o.aRy = dup(r.aRy); o.aRz = dup(r.aRz); o.ampr = dup(r.ampr);
    o.eRx = dup(r.eRx); o.eRy = dup(r.eRy); o.eRz = dup(r.eRz); o.pad = dup(0.0f);
    return o;
}

// FP64 references of the batch's pulses [pa, pe) for the tile reference point
// (xr, yr); thread-parallel over (pulse, antenna), one barrier between the
// transmit and receive stages. DUP selects the pair layout of the forward path.
template <bool DUP>
__device__ void build_refs(const Smem &sm, const MixedArgs &A, int pa, int pe, double xr, double yr)
{
    const DevScene &S = A.S;
    const int npb = pe - pa;
    for (int t = threadIdx.x; t < npb; t += NT) {
        int n = pa + t;
        const PulseState &P = S.pulses[n];
        double u[3], dref;
        AntRec r;
        tile_ref(P.tx, xr, yr, u, dref, r);
        if (DUP)
            sm.tx2[t] = dup_rec(r);
        else
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
    __syncthreads();
    for (int t = threadIdx.x; t < npb * S.nc; t += NT) {
        int pi = t / S.nc, c = t % S.nc;
        int n = pa + pi;
        const RxState &Rs = S.rx[(size_t)n * S.nc + c];
        double u[3], dref;
        AntRec r;
        tile_ref(Rs.rx, xr, yr, u, dref, r);
        const double *td = sm.txd + 4 * pi;
        double off = td[3] + dref;  // (R_t + R_r) - (Rbar_t + Rbar_r)
        ChanRec q;
        q.psi = (float)wrap_pi(Rs.psi - S.k0 * off);
        q.ax = (float)wrap_pi(-S.k0 * (td[0] + u[0]) * S.dx);
        q.ay = (float)wrap_pi(-S.k0 * (td[1] + u[1]) * S.dx);
        q.gam = (float)(-S.k0 * (td[2] + u[2]));
        double p = Rs.p_ref + off * S.inv_dr;
        double kb = floor(p);
        q.kbase = (int)kb;
        q.pfrac = (float)(p - kb);
        q.pad0 = q.pad1 = 0.0f;
        if (DUP) {
            sm.rx2[t] = dup_rec(r);
            ChanRec2 q2;
            q2.psi = dup(q.psi);
            q2.ax = dup(q.ax);
            q2.ay = dup(q.ay);
            q2.gam = dup(q.gam);
            q2.pfrac = dup(q.pfrac);
            q2.kbase = q.kbase;
            q2.pad0 = 0;
            q2.pad1 = dup(0.0f);
            sm.ch2[t] = q2;
        } else {
            sm.rx[t] = r;
            sm.ch[t] = q;
        }
    }
}

// Taylor coefficients of (eta, eta_x, eta_y) in time for two facets (column ix,
// rows iya / iyb), accumulated over the wave components in shared-memory chunks.
__device__ void taylor_coeffs(const Smem &sm, const MixedArgs &A, int batch, int ix, int iya, int iyb, bool two,
                              float ca[3][kOrders], float cb[3][kOrders])
{
    const DevScene &S = A.S;
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int o = 0; o < kOrders; ++o) ca[f][o] = cb[f][o] = 0.0f;
    const int nw = S.nw;
    const int ixc = min(ix, S.nx - 1), iyac = min(iya, S.ny - 1), iybc = min(iyb, S.ny - 1);
    for (int m0 = 0; m0 < nw; m0 += WCH) {
        const int cnt = min(WCH, nw - m0);
        __syncthreads();
        const float2 *src = A.wt + ((size_t)batch * nw + m0) * 3 * kOrders;
        for (int i = threadIdx.x; i < cnt * 3 * kOrders; i += NT) sm.w[i] = src[i];
        __syncthreads();
        for (int m = 0; m < cnt; ++m) {
            float2 e = __ldg(A.ex + (size_t)(m0 + m) * S.nx + ixc);
            float2 ya = __ldg(A.ey + (size_t)(m0 + m) * S.ny + iyac);
            float2 yb = __ldg(A.ey + (size_t)(m0 + m) * S.ny + iybc);
            float qar = e.x * ya.x - e.y * ya.y, qai = e.x * ya.y + e.y * ya.x;
            float qbr = e.x * yb.x - e.y * yb.y, qbi = e.x * yb.y + e.y * yb.x;
            const float2 *wm = sm.w + m * 3 * kOrders;
            if (two) {
#pragma unroll
                for (int f = 0; f < 3; ++f)
#pragma unroll
                    for (int o = 0; o < kOrders; ++o) {
                        float2 w = wm[f * kOrders + o];
                        ca[f][o] = fmaf(qar, w.x, fmaf(-qai, w.y, ca[f][o]));
                        cb[f][o] = fmaf(qbr, w.x, fmaf(-qbi, w.y, cb[f][o]));
                    }
            } else {
#pragma unroll
                for (int f = 0; f < 3; ++f)
#pragma unroll
                    for (int o = 0; o < kOrders; ++o) {
                        float2 w = wm[f * kOrders + o];
                        ca[f][o] = fmaf(qar, w.x, fmaf(-qai, w.y, ca[f][o]));
                    }
            }
        }
    }
}

__device__ __forceinline__ float horner(const float c[kOrders], float t)
{
    float r = c[kOrders - 1];
#pragma unroll
    for (int o = kOrders - 2; o >= 0; --o) r = fmaf(r, t, c[o]);
    return r;
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
    float *stage;
    float2 *tiles;  // [2][nc][WT]
    OutT *iq;
    int n, n0, np, buf;
    // two facets (packed path): one warp reduction each
    __device__ __forceinline__ void put2(const MixedArgs &A, int ch, int kbase, int kba, int kbb, const float ha[8],
                                         const float hb[8], float2 vre, float2 vim, float2, float2, float, bool va,
                                         bool vb)
    {
        float2 *tile_c = tiles + (buf * A.S.nc + ch) * WT;
        const int tile_base = kbase - WT_LO;
        OutT *grow = iq + 2 * ((size_t)ch * np + (n - n0)) * A.S.nr;
        warp_scatter<OutT>(stage, tile_c, tile_base, kba, va, ha, vre.x, vim.x, A.S.nr, grow, A.S.flags);
        warp_scatter<OutT>(stage, tile_c, tile_base, kbb, vb, hb, vre.y, vim.y, A.S.nr, grow, A.S.flags);
    }
};

// Adjoint sink of the packed path: the gathers of the two facets, then the
// chain-rule terms accumulated as pairs.
template <typename InT>
struct GatherSink2 {
    const float2 *win;  // [nc][WT] residual window of the pulse
    const InT *resid;
    int n, n0, np;
    float2 as, au, av;  // per-facet accumulators, facet a in .x, facet b in .y
    __device__ __forceinline__ float2 gather(const MixedArgs &A, const float2 *wc, int tb, const InT *grow, int kb,
                                             const float h[8]) const
    {
        float gr = 0.0f, gi = 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = kb + j;
            const int w = k - tb;
            float2 v;
            if ((unsigned)w < (unsigned)WT)
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
        const float2 *wc = win + ch * WT;
        const int tb = kbase - WT_LO;
        const InT *grow = resid + 2 * ((size_t)ch * np + (n - n0)) * A.S.nr;
        const float2 ga = gather(A, wc, tb, grow, kba, ha);
        const float2 gb = gather(A, wc, tb, grow, kbb, hb);
        const float2 GR = make_float2(ga.x, gb.x), GI = make_float2(ga.y, gb.y);
        const float2 re_gs = fma2(GR, vre, mul2(GI, vim));
        const float2 im_gs = fma2(GR, vim, neg2(mul2(GI, vre)));
        as = add2(as, re_gs);
        const float2 mk = dup(-k0t);
        au = fma2(mul2(mk, qx), im_gs, au);
        av = fma2(mul2(mk, qy), im_gs, av);
    }
};

// Per-thread pair of facets (same column, rows w and w + 8) for the packed path.
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

// Forward contribution of the thread's two facets for pulse pi (chunk index),
// every channel: the same arithmetic as facet_pulse, on FP32x2 pairs (facet a in
// .x, facet b in .y); transcendentals and integer work per element.
template <int TAPS, typename Sink>
__device__ __forceinline__ void facet_pulse2(const Smem &sm, const MixedArgs &A, const PolyArgs &P, const PairGeo &G,
                                             const float2 C[3][kOrders], int pi, float xi_x, float fi, Sink &sink)
{
    const DevScene &S = A.S;
    const int nc = S.nc;
    const float2 one = make_float2(1.0f, 1.0f);
    const PulseRec PR = sm.pr[pi];
    const float2 tau = dup(PR.tau);
    const float2 eta = horner2(C[0], tau);
    const float2 sx = horner2(C[1], tau);
    const float2 sy = horner2(C[2], tau);
    const float2 X0 = dup(xi_x), X1 = G.xi_y;
    const float2 b2 = fma2(X0, X0, fma2(X1, X1, mul2(eta, eta)));
    const float2 nn = fma2(sx, sx, fma2(sy, sy, one));
    const float2 inv_n = make_float2(rsqrtf(nn.x), rsqrtf(nn.y));

    // transmit leg (shared by the channels)
    const AntRec2 T = sm.tx2[pi];
    const float2 at = fma2(T.ux, X0, fma2(T.uy, X1, mul2(T.uz, eta)));
    const float2 st = fma2(neg2(at), at, b2);
    const float2 qt = mul2(st, fma2(neg2(at), T.inv2R2, T.inv2R));
    const float2 dt = add2(at, qt);
    const float2 et = mul2(dt, T.invR);
    const float2 rho_t = fma2(et, et, sub2(one, et));
    const float2 ut = mul2(add2(T.u0, fma2(X0, T.aRx, fma2(X1, T.aRy, mul2(eta, T.aRz)))), rho_t);
    const float2 vt = mul2(add2(T.v0, fma2(X0, T.eRx, fma2(X1, T.eRy, mul2(eta, T.eRz)))), rho_t);
    const float2 gt = mul2(sinc2_2(P, mul2(dup(A.tx_laz_l), ut)), sinc2_2(P, mul2(dup(A.tx_lel_l), vt)));
    const float2 rt0 = mul2(fma2(X0, T.invR, T.ux), rho_t);
    const float2 rt1 = mul2(fma2(X1, T.invR, T.uy), rho_t);
    const float2 rt2 = mul2(fma2(eta, T.invR, T.uz), rho_t);
    const float2 ampt = mul2(mul2(gt, T.ampr), rho_t);

    const AntRec2 *RX = sm.rx2 + pi * nc;
    const ChanRec2 *CH = sm.ch2 + pi * nc;
    for (int ch = 0; ch < nc; ++ch) {
        const AntRec2 R = RX[ch];
        const ChanRec2 Q = CH[ch];
        const float2 ar = fma2(R.ux, X0, fma2(R.uy, X1, mul2(R.uz, eta)));
        const float2 sr_ = fma2(neg2(ar), ar, b2);
        const float2 qr = mul2(sr_, fma2(neg2(ar), R.inv2R2, R.inv2R));
        const float2 dr = add2(ar, qr);
        const float2 er = mul2(dr, R.invR);
        const float2 rho_r = fma2(er, er, sub2(one, er));
        const float2 ur = mul2(add2(R.u0, fma2(X0, R.aRx, fma2(X1, R.aRy, mul2(eta, R.aRz)))), rho_r);
        const float2 vr = mul2(add2(R.v0, fma2(X0, R.eRx, fma2(X1, R.eRy, mul2(eta, R.eRz)))), rho_r);
        const float2 gr = mul2(sinc2_2(P, mul2(dup(A.rx_laz_l[ch]), ur)), sinc2_2(P, mul2(dup(A.rx_lel_l[ch]), vr)));
        const float2 qx = neg2(fma2(fma2(X0, R.invR, R.ux), rho_r, rt0));
        const float2 qy = neg2(fma2(fma2(X1, R.invR, R.uy), rho_r, rt1));
        const float2 qz = neg2(fma2(fma2(eta, R.invR, R.uz), rho_r, rt2));
        // sqrt(sigma0 A) = X rsqrt(X Q_z), X = base A (1 + m cos phi) max(0, n.Q) / |n|
        float2 amp_s = G.amp_static;
        if (!S.static_surface) {
            const float2 qh2 = fma2(qx, qx, mul2(qy, qy));
            const float2 rq = make_float2(qh2.x > 0.0f ? rsqrtf(qh2.x) : 0.0f, qh2.y > 0.0f ? rsqrtf(qh2.y) : 0.0f);
            const float2 cphi = mul2(fma2(dup(A.wcos), qx, mul2(dup(A.wsin), qy)), rq);
            const float2 nq = fma2(neg2(sx), qx, fma2(neg2(sy), qy, qz));
            const float2 nqp = make_float2(fmaxf(nq.x, 0.0f), fmaxf(nq.y, 0.0f));
            const float2 X = mul2(mul2(G.base_area, fma2(dup(A.wind_mod), cphi, one)), mul2(nqp, inv_n));
            const float2 Xq = mul2(X, qz);
            amp_s = make_float2(X.x > 0.0f ? X.x * rsqrtf(Xq.x) : 0.0f, X.y > 0.0f ? X.y * rsqrtf(Xq.y) : 0.0f);
        }
        const float2 amp = mul2(mul2(mul2(amp_s, ampt), mul2(gr, R.ampr)), rho_r);
        const float2 vc = neg2(fma2(G.cu, qx, mul2(G.cv, qy)));
        float2 phi = fma2(dup(fi), Q.ax, Q.psi);
        phi = fma2(G.fj, Q.ay, phi);
        phi = fma2(Q.gam, eta, phi);
        phi = fma2(dup(-A.k0), add2(qt, qr), phi);
        phi = fma2(dup(-PR.k0t), vc, phi);
        const float2 kk = make_float2(rintf(phi.x * 0.15915494309189535f), rintf(phi.y * 0.15915494309189535f));
        phi = fma2(neg2(kk), dup(6.28125f), phi);
        phi = fma2(neg2(kk), dup(1.9353071795864769e-3f), phi);
        float sa, ca, sb, cb;
        __sincosf(phi.x, &sa, &ca);
        __sincosf(phi.y, &sb, &cb);
        const float2 sp = make_float2(sa, sb), cp = make_float2(ca, cb);
        const float2 zr = mul2(amp, G.zr), zi = mul2(amp, G.zi);
        const float2 vre = fma2(zr, cp, neg2(mul2(zi, sp)));
        const float2 vim = fma2(zr, sp, mul2(zi, cp));
        const float2 p = fma2(add2(dt, dr), dup(A.inv_dr), Q.pfrac);
        const float2 kf = make_float2(floorf(p.x), floorf(p.y));
        const float2 fr = sub2(p, kf);
        int kba, kbb;
        float ha[8], hb[8];
        if (TAPS == 1) {
            kba = Q.kbase + (int)kf.x;
            kbb = Q.kbase + (int)kf.y;
            ha[0] = hb[0] = 1.0f;
#pragma unroll
            for (int j = 1; j < 8; ++j) ha[j] = hb[j] = 0.0f;
        } else {
            kba = Q.kbase + (int)kf.x - 3;
            kbb = Q.kbase + (int)kf.y - 3;
            const float2 t = fma2(dup(2.0f), fr, dup(-1.0f));
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float2 v = P.tap[j][kTapDeg];
#pragma unroll
                for (int d = kTapDeg - 1; d >= 0; --d) v = fma2(v, t, P.tap[j][d]);
                ha[j] = v.x;
                hb[j] = v.y;
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

// One forward work item (tile x pulse batch) of one scene. Every thread of the
// CTA calls it; it starts and ends with the CTA's range tiles all zero.
template <int TAPS, typename OutT>
__device__ void forward_item(const Smem &sm, const MixedArgs &A, const PolyArgs &P, const ItemGeo &I, int n0, int np,
                             OutT *iq)
{
    const DevScene &S = A.S;
    const int nc = S.nc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool two = I.ty > NWARP;
    const int ix = I.tx0 + lane;
    const int iref = I.tx0 + TX / 2, jref = I.ty0 + I.ty / 2;
    const double xr = (iref + 0.5 - 0.5 * S.nx) * S.dx;
    const double yr = (jref + 0.5 - 0.5 * S.ny) * S.dx;
    const float xi_x = (float)((ix - iref) * S.dx);
    const float fi = (float)(ix - iref);

    FacetGeo ga, gb;
    facet_setup(A, ix, I.ty0 + warp, jref, ga);
    facet_setup(A, ix, I.ty0 + warp + NWARP, jref, gb);
    float ca[3][kOrders], cb[3][kOrders];
    if (!S.static_surface && S.nw > 0) {
        taylor_coeffs(sm, A, I.batch, ix, I.ty0 + warp, I.ty0 + warp + NWARP, two, ca, cb);
    } else {
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int o = 0; o < kOrders; ++o) ca[f][o] = cb[f][o] = 0.0f;
    }
    __syncthreads();
    // the warp buffers share memory with the wave-table chunk: clear them
    for (int i = threadIdx.x; i < NWARP * SBINS * SROW; i += NT) sm.stage[i] = 0.0f;
    __syncthreads();

    ScatterSink<OutT> sink;
    sink.stage = sm.stage + warp * SBINS * SROW;
    sink.tiles = sm.tile;
    sink.iq = iq;
    sink.n0 = n0;
    sink.np = np;
    // pack the two facets: .x = row w, .y = row w + 8 (a copy of .x, masked off, for 8-row tiles)
    PairGeo G;
    const FacetGeo &gq = two ? gb : ga;
    G.xi_y = make_float2(ga.xi_y, gq.xi_y);
    G.fj = make_float2(ga.fj, gq.fj);
    G.base_area = make_float2(ga.base_area, gq.base_area);
    G.amp_static = make_float2(ga.amp_static, gq.amp_static);
    G.cu = make_float2(ga.cu, gq.cu);
    G.cv = make_float2(ga.cv, gq.cv);
    G.va = ga.valid;
    G.vb = two && gb.valid;
    float2 C[3][kOrders];
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int o = 0; o < kOrders; ++o) C[f][o] = make_float2(ca[f][o], two ? cb[f][o] : ca[f][o]);
    for (int c0 = I.pa; c0 < I.pe; c0 += NBR) {
        const int ce = min(c0 + NBR, I.pe);
        __syncthreads();  // the previous chunk's flush is done with the records
        build_refs<true>(sm, A, c0, ce, xr, yr);
        __syncthreads();
        for (int n = c0; n < ce; ++n) {
            const int pi = n - c0;
            const int buf = n & 1;
            const int e = sm.pr[pi].epoch;
            if (e != ga.epoch) {
                ga.z = speckle_f(S.speckle_seed, ga.fid, (uint32_t)e);
                ga.epoch = e;
            }
            if (two && e != gb.epoch) {
                gb.z = speckle_f(S.speckle_seed, gb.fid, (uint32_t)e);
                gb.epoch = e;
            }
            G.zr = make_float2(ga.z.x, two ? gb.z.x : 0.0f);
            G.zi = make_float2(ga.z.y, two ? gb.z.y : 0.0f);
            sink.n = n;
            sink.buf = buf;
            facet_pulse2<TAPS>(sm, A, P, G, C, pi, xi_x, fi, sink);
            __syncthreads();
            for (int i = threadIdx.x; i < nc * WT; i += NT) {
                int ch = i / WT, w = i % WT;
                float2 *slot = sm.tile + (buf * nc + ch) * WT + w;
                float2 v = *slot;
                *slot = make_float2(0.f, 0.f);
                int k = sm.ch2[pi * nc + ch].kbase - WT_LO + w;
                if ((v.x != 0.0f || v.y != 0.0f) && k >= 0 && k < S.nr)
                    gadd<OutT>(iq + 2 * ((size_t)ch * np + (n - n0)) * S.nr, (size_t)k, v.x, v.y);
            }
        }
    }
    // the other buffer was flushed one pulse earlier; make sure every thread is
    // done with the tiles and the records before they are reused
    __syncthreads();
}

__device__ __forceinline__ void clear_smem(const Smem &sm, int nc)
{
    for (int i = threadIdx.x; i < 2 * nc * WT; i += NT) sm.tile[i] = make_float2(0.f, 0.f);
    for (int i = threadIdx.x; i < NWARP * SBINS * SROW; i += NT) sm.stage[i] = 0.0f;
}

template <int TAPS, typename OutT>
__global__ void __launch_bounds__(NT, 2)
    accumulate_mixed_kernel(MixedArgs A, PolyArgs P, int n0, int np, int b0, int ty, OutT *iq)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem sm = carve(smem_raw, A.S.nc, true);
    const ItemGeo I = item_geo(A, blockIdx.x, b0 + blockIdx.y, ty, n0, np);
    if (I.pa >= I.pe) return;
    clear_smem(sm, A.S.nc);
    forward_item<TAPS, OutT>(sm, A, P, I, n0, np, iq);
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
template <int TAPS>
__global__ void __launch_bounds__(NT, 2) batch_mixed_kernel(BatchItems B, PolyArgs P, unsigned int *counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ MixedArgs args;
    __shared__ int s_item, s_scene;
    const int nc_max = B.args[0].S.nc;  // layout sized for the first scene's channels (all equal)
    const Smem sm = carve(smem_raw, nc_max, true);
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
        if (I.pa < I.pe) forward_item<TAPS, float>(sm, args, P, I, 0, args.S.np_total, B.iq[scene]);
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

template <int TAPS, typename InT>
__global__ void __launch_bounds__(NT, 2)
    adjoint_mixed_kernel(MixedArgs A, PolyArgs P, int n0, int np, int b0, const InT *resid, double *g_sigma,
                         double *g_uv)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DevScene &S = A.S;
    const int nc = S.nc;
    const Smem sm = carve(smem_raw, nc, true);
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
    const float xi_x = (float)((ix - iref) * S.dx);
    const float fi = (float)(ix - iref);

    FacetGeo ga, gb;
    facet_setup(A, ix, ty0 + warp, jref, ga);
    facet_setup(A, ix, ty0 + warp + NWARP, jref, gb);
    float ca[3][kOrders], cb[3][kOrders];
    if (!S.static_surface && S.nw > 0) {
        taylor_coeffs(sm, A, batch, ix, ty0 + warp, ty0 + warp + NWARP, true, ca, cb);
    } else {
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int o = 0; o < kOrders; ++o) ca[f][o] = cb[f][o] = 0.0f;
    }
    PairGeo G;
    G.xi_y = make_float2(ga.xi_y, gb.xi_y);
    G.fj = make_float2(ga.fj, gb.fj);
    G.base_area = make_float2(ga.base_area, gb.base_area);
    G.amp_static = make_float2(ga.amp_static, gb.amp_static);
    G.cu = make_float2(ga.cu, gb.cu);
    G.cv = make_float2(ga.cv, gb.cv);
    G.va = ga.valid;
    G.vb = gb.valid;
    float2 C[3][kOrders];
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int o = 0; o < kOrders; ++o) C[f][o] = make_float2(ca[f][o], cb[f][o]);
    GatherSink2<InT> sink;
    sink.win = sm.tile;
    sink.resid = resid;
    sink.n0 = n0;
    sink.np = np;
    sink.as = sink.au = sink.av = make_float2(0.0f, 0.0f);
    for (int n = pa; n < pe; ++n) {
        const int pi = (n - pa) % NBR;
        if (pi == 0) {
            __syncthreads();  // the previous chunk is done with the records
            build_refs<true>(sm, A, n, min(n + NBR, pe), xr, yr);
        }
        __syncthreads();
        // residual window of this pulse, every channel
        for (int i = threadIdx.x; i < nc * WT; i += NT) {
            int ch = i / WT, w = i % WT;
            int k = sm.ch2[pi * nc + ch].kbase - WT_LO + w;
            float2 v = make_float2(0.f, 0.f);
            if (k >= 0 && k < S.nr) {
                const InT *r = resid + 2 * (((size_t)ch * np + (n - n0)) * S.nr + k);
                v = make_float2((float)r[0], (float)r[1]);
            }
            sm.tile[i] = v;
        }
        __syncthreads();
        const int e = sm.pr[pi].epoch;
        if (e != ga.epoch) {
            ga.z = speckle_f(S.speckle_seed, ga.fid, (uint32_t)e);
            ga.epoch = e;
        }
        if (e != gb.epoch) {
            gb.z = speckle_f(S.speckle_seed, gb.fid, (uint32_t)e);
            gb.epoch = e;
        }
        G.zr = make_float2(ga.z.x, gb.z.x);
        G.zi = make_float2(ga.z.y, gb.z.y);
        sink.n = n;
        facet_pulse2<TAPS>(sm, A, P, G, C, pi, xi_x, fi, sink);
    }
    add_cell_grads(ga, sink.as.x, sink.au.x, sink.av.x, g_sigma, g_uv);
    add_cell_grads(gb, sink.as.y, sink.au.y, sink.av.y, g_sigma, g_uv);
}

// Facet generator of the mixed path: same Taylor expansion, states written out.
__global__ void __launch_bounds__(NT, 2) generate_mixed_kernel(MixedArgs A, int n0, int np, int b0, float *state)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DevScene &S = A.S;
    const Smem sm = carve(smem_raw, S.nc, false);
    const int tiles_x = (S.nx + TX - 1) / TX;
    const int tx0 = (blockIdx.x % tiles_x) * TX;
    const int ty0 = (blockIdx.x / tiles_x) * TY;
    const int batch = b0 + blockIdx.y;
    const int pa = max(n0, batch * A.nb);
    const int pe = min(n0 + np, (batch + 1) * A.nb);
    if (pa >= pe) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ix = tx0 + lane;
    const int iya = ty0 + warp, iyb = ty0 + warp + NWARP;
    const bool va = ix < S.nx && iya < S.ny, vb = ix < S.nx && iyb < S.ny;
    float ca[3][kOrders], cb[3][kOrders];
    if (!S.static_surface && S.nw > 0) {
        taylor_coeffs(sm, A, batch, ix, iya, iyb, true, ca, cb);
    } else {
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int o = 0; o < kOrders; ++o) ca[f][o] = cb[f][o] = 0.0f;
    }
    const int64_t nf = (int64_t)S.nx * S.ny;
    for (int n = pa; n < pe; ++n) {
        float tau = A.tau[n];
        float *o = state + (size_t)(n - n0) * 3 * nf;
        if (va) {
            int64_t f = (int64_t)iya * S.nx + ix;
            o[f] = horner(ca[0], tau);
            o[nf + f] = horner(ca[1], tau);
            o[2 * nf + f] = horner(ca[2], tau);
        }
        if (vb) {
            int64_t f = (int64_t)iyb * S.nx + ix;
            o[f] = horner(cb[0], tau);
            o[nf + f] = horner(cb[1], tau);
            o[2 * nf + f] = horner(cb[2], tau);
        }
    }
}

MixedArgs make_args(const DevScene &S, const MixedTables &M)
{
    MixedArgs A;
    A.S = S;
    A.ex = M.ex;
    A.ey = M.ey;
    A.wt = M.wt;
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
    for (int j = 0; j < 8; ++j)
        for (int d = 0; d <= kTapDeg; ++d) P.tap[j][d] = make_float2(M.tap[j][d], M.tap[j][d]);
    for (int d = 0; d <= kSincDeg; ++d) P.sinc2[d] = make_float2(M.sinc2[d], M.sinc2[d]);
    return P;
}

template <typename K>
cudaError_t prep(K kernel, int bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace

int mixed_smem_bytes(int nc) { return layout(nc, true).total; }

cudaError_t launch_generate_mixed(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                                  float *state)
{
    MixedArgs A = make_args(S, M);
    const int bytes = layout(S.nc, false).total;
    cudaError_t e = prep(generate_mixed_kernel, bytes);
    if (e != cudaSuccess) return e;
    int tiles = ((S.nx + TX - 1) / TX) * ((S.ny + TY - 1) / TY);
    int b0 = n0 / M.nb, b1 = (n0 + np - 1) / M.nb;
    for (int bb = b0; bb <= b1; bb += 65535) {
        int cnt = min(65535, b1 - bb + 1);
        generate_mixed_kernel<<<dim3(tiles, cnt), NT, bytes, st>>>(A, n0, np, bb, state);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_accumulate_mixed(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                                    void *iq, harm_dtype dtype)
{
    MixedArgs A = make_args(S, M);
    PolyArgs P = make_poly(M);
    const int bytes = layout(S.nc, true).total;
    const int ty = TY;
    int tiles = ((S.nx + TX - 1) / TX) * ((S.ny + ty - 1) / ty);
    int b0 = n0 / M.nb, b1 = (n0 + np - 1) / M.nb;
    cudaError_t e;
    for (int bb = b0; bb <= b1; bb += 65535) {
        int cnt = min(65535, b1 - bb + 1);
        dim3 grid(tiles, cnt);
        if (dtype == HARM_C64) {
            if (S.taps == 1) {
                if ((e = prep(accumulate_mixed_kernel<1, float>, bytes)) != cudaSuccess) return e;
                accumulate_mixed_kernel<1, float><<<grid, NT, bytes, st>>>(A, P, n0, np, bb, ty, (float *)iq);
            } else {
                if ((e = prep(accumulate_mixed_kernel<8, float>, bytes)) != cudaSuccess) return e;
                accumulate_mixed_kernel<8, float><<<grid, NT, bytes, st>>>(A, P, n0, np, bb, ty, (float *)iq);
            }
        } else {
            if (S.taps == 1) {
                if ((e = prep(accumulate_mixed_kernel<1, double>, bytes)) != cudaSuccess) return e;
                accumulate_mixed_kernel<1, double><<<grid, NT, bytes, st>>>(A, P, n0, np, bb, ty, (double *)iq);
            } else {
                if ((e = prep(accumulate_mixed_kernel<8, double>, bytes)) != cudaSuccess) return e;
                accumulate_mixed_kernel<8, double><<<grid, NT, bytes, st>>>(A, P, n0, np, bb, ty, (double *)iq);
            }
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_adjoint_mixed(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                                 const void *resid, harm_dtype dtype, double *g_sigma, double *g_uv)
{
    MixedArgs A = make_args(S, M);
    PolyArgs P = make_poly(M);
    const int bytes = layout(S.nc, true).total;
    int tiles = ((S.nx + TX - 1) / TX) * ((S.ny + TY - 1) / TY);
    int b0 = n0 / M.nb, b1 = (n0 + np - 1) / M.nb;
    cudaError_t e;
    for (int bb = b0; bb <= b1; bb += 65535) {
        int cnt = min(65535, b1 - bb + 1);
        dim3 grid(tiles, cnt);
        if (dtype == HARM_C64) {
            if (S.taps == 1) {
                if ((e = prep(adjoint_mixed_kernel<1, float>, bytes)) != cudaSuccess) return e;
                adjoint_mixed_kernel<1, float><<<grid, NT, bytes, st>>>(A, P, n0, np, bb, (const float *)resid,
                                                                         g_sigma, g_uv);
            } else {
                if ((e = prep(adjoint_mixed_kernel<8, float>, bytes)) != cudaSuccess) return e;
                adjoint_mixed_kernel<8, float><<<grid, NT, bytes, st>>>(A, P, n0, np, bb, (const float *)resid,
                                                                         g_sigma, g_uv);
            }
        } else {
            if (S.taps == 1) {
                if ((e = prep(adjoint_mixed_kernel<1, double>, bytes)) != cudaSuccess) return e;
                adjoint_mixed_kernel<1, double><<<grid, NT, bytes, st>>>(A, P, n0, np, bb, (const double *)resid,
                                                                          g_sigma, g_uv);
            } else {
                if ((e = prep(adjoint_mixed_kernel<8, double>, bytes)) != cudaSuccess) return e;
                adjoint_mixed_kernel<8, double><<<grid, NT, bytes, st>>>(A, P, n0, np, bb, (const double *)resid,
                                                                          g_sigma, g_uv);
            }
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int mixed_batch_pulses() { return NBG; }

// ---------------------------------------------------------------------------
// Batched persistent launch (host side)
// ---------------------------------------------------------------------------
size_t batch_args_bytes() { return sizeof(MixedArgs); }

void batch_fill_args(const harm_scene *s, void *dst)
{
    MixedArgs A = make_args(s->dev, s->mixed);
    memcpy(dst, &A, sizeof(MixedArgs));
}

int batch_tiles(const harm_scene *s, int ty)
{
    return ((s->desc.nx + TX - 1) / TX) * ((s->desc.ny + ty - 1) / ty);
}

int batch_ctas(int device)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return 2 * sms;
}

cudaError_t batch_launch(const BatchLaunch &L, cudaStream_t st)
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
    PolyArgs P = make_poly(*L.poly);
    const int bytes = layout(L.nc, true).total;
    cudaError_t e;
    if (L.taps == 1) {
        if ((e = prep(batch_mixed_kernel<1>, bytes)) != cudaSuccess) return e;
        batch_mixed_kernel<1><<<L.ctas, NT, bytes, st>>>(B, P, L.counter);
    } else {
        if ((e = prep(batch_mixed_kernel<8>, bytes)) != cudaSuccess) return e;
        batch_mixed_kernel<8><<<L.ctas, NT, bytes, st>>>(B, P, L.counter);
    }
    return cudaGetLastError();
}

}  // namespace harm
