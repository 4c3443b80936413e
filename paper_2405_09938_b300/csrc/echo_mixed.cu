// Mixed-precision echo path: FP64 only for per-pulse platform state, the
// reference bistatic range and each tile's range offset; FP32 for the per-facet
// geometry, antenna patterns, NRCS, phase, interpolation taps and accumulation.
//
// Work decomposition (one CTA = a 32 x 16 facet tile x one batch of pulses):
//  1. FP64 tile references: for every pulse of the batch and every antenna, the
//     range R from the antenna to the tile's reference point on the mean surface,
//     its unit vector and the tile's reduced reference phase and range-bin offset.
//     Per facet, r - R is then a small offset that FP32 carries to ~1e-8 m:
//        r - R = a + (b - a^2) / (2R) + (a^3 - a b) / (2R^2),  a = u.xi, b = |xi|^2
//     for the facet offset xi from the reference point; the linear phase term
//     K0 (u_t + u_r).xi is split into exactly-reduced lattice steps.
//  2. Facet generator: the surface of the tile over the batch is expanded in time
//     about the batch centre, eta(t_c + tau) = sum_m eta_m tau^m, with the
//     Taylor coefficients eta_m = Re sum_w Q_w E_{w,m} accumulated over the wave
//     components (register-blocked FP32 contraction, separable phasors Q).
//  3. For each pulse: Horner gives (eta, eta_x, eta_y); each facet forms its
//     contribution for every channel (Eq. 3, 4, 16), spreads it over 8 bins with
//     the Kaiser-sinc taps (polynomials in the fractional bin) and the warp
//     pre-reduces the 32 lanes' taps through a shared-memory transpose into a
//     16-bin window; the window is added to the CTA's range tile; the tile is
//     flushed to the IQ with one vector atomic per bin and channel.
#include <cuda_runtime.h>

#include <climits>

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
constexpr int NBMAX = 32;     // pulses per batch
constexpr int WCH = 128;      // wave components per shared-memory chunk
constexpr int STG = 20;       // staging row stride (floats) of the warp transpose
constexpr float kPiF = 3.14159265358979f;

struct TxRec {
    float u[3];
    float invR, inv2R, inv2R2;
    float u0, v0;
    float aR[3], eR[3];
    float ampr;
};

struct RxRec {
    float u[3];
    float invR, inv2R, inv2R2;
    float u0, v0;
    float aR[3], eR[3];
    float ampr;
    float psi, ax, ay, gam, pfrac;
    int kbase;
};

struct PulseRec {
    float tau, k0t;
    int epoch;
    int pad;
};

struct MixedArgs {
    DevScene S;
    const float2 *ex, *ey, *wt;
    const float *tau;
    int nb, n_batches;
    float tap[8][kTapDeg + 1];
};

struct Smem {
    float2 w[WCH][3][kOrders];          // Taylor tables chunk
    float2 tile[2][kMaxCh][WT];         // double-buffered range tiles
    TxRec tx[NBMAX];
    RxRec rx[NBMAX][kMaxCh];
    PulseRec pr[NBMAX];
    double txd[NBMAX][4];               // FP64 tx unit vector + tile offset
    float stage[NWARP][32 * STG];       // warp transpose staging
};

__device__ __forceinline__ float sinc2f(float x)
{
    float px = kPiF * x;
    if (fabsf(px) < 1e-4f) return 1.0f - px * px * (1.0f / 3.0f);
    float s = __fdividef(sinpif(x), px);
    return s * s;
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

// FP64 tile reference of one antenna at position p with frame (a, e) for the
// tile reference point X = (xr, yr, 0): D = X - p, R = |D|, u = D / R, and the
// stable offset R - |p| = (|X|^2 - 2 p.X) / (R + |p|).
__device__ void tile_ref(const AntState &A, double xr, double yr, double laz_unused, double &R, double u[3],
                         double &dref, float *uf, float &invR, float &inv2R, float &inv2R2, float &u0, float &v0,
                         float *aR, float *eR, float &ampr)
{
    (void)laz_unused;
    double D[3] = {xr - A.p[0], yr - A.p[1], -A.p[2]};
    R = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    double iR = 1.0 / R;
    for (int i = 0; i < 3; ++i) u[i] = D[i] * iR;
    double xx = xr * xr + yr * yr;
    dref = (xx - 2.0 * (A.p[0] * xr + A.p[1] * yr)) / (R + A.rref);
    for (int i = 0; i < 3; ++i) {
        uf[i] = (float)u[i];
        aR[i] = (float)(A.a[i] * iR);
        eR[i] = (float)(A.e[i] * iR);
    }
    invR = (float)iR;
    inv2R = (float)(0.5 * iR);
    inv2R2 = (float)(0.5 * iR * iR);
    u0 = (float)(u[0] * A.a[0] + u[1] * A.a[1] + u[2] * A.a[2]);
    v0 = (float)(u[0] * A.e[0] + u[1] * A.e[1] + u[2] * A.e[2]);
    ampr = (float)(A.rref * iR);
}

// FP64 references of the batch's pulses [pa, pe) for the tile with reference
// point (xr, yr); thread-parallel over (pulse, antenna). Needs a barrier between
// the transmit and receive stages.
__device__ void build_refs(Smem &sm, const MixedArgs &A, int pa, int pe, double xr, double yr)
{
    const DevScene &S = A.S;
    const int npb = pe - pa;
    for (int t = threadIdx.x; t < npb; t += NT) {
        int n = pa + t;
        const PulseState &P = S.pulses[n];
        TxRec &T = sm.tx[t];
        double R, u[3], dref;
        tile_ref(P.tx, xr, yr, 0.0, R, u, dref, T.u, T.invR, T.inv2R, T.inv2R2, T.u0, T.v0, T.aR, T.eR, T.ampr);
        sm.txd[t][0] = u[0];
        sm.txd[t][1] = u[1];
        sm.txd[t][2] = u[2];
        sm.txd[t][3] = dref;
        PulseRec &pr = sm.pr[t];
        pr.tau = A.tau[n];
        pr.k0t = (float)(S.k0 * P.t);
        pr.epoch = S.epoch_pulses > 0 ? n / S.epoch_pulses : 0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < npb * S.nc; t += NT) {
        int pi = t / S.nc, c = t % S.nc;
        int n = pa + pi;
        const RxState &Rs = S.rx[(size_t)n * S.nc + c];
        RxRec &Q = sm.rx[pi][c];
        double R, u[3], dref;
        tile_ref(Rs.rx, xr, yr, 0.0, R, u, dref, Q.u, Q.invR, Q.inv2R, Q.inv2R2, Q.u0, Q.v0, Q.aR, Q.eR, Q.ampr);
        double off = sm.txd[pi][3] + dref;  // (R_t + R_r) - (Rbar_t + Rbar_r)
        Q.psi = (float)wrap_pi(Rs.psi - S.k0 * off);
        double sx = sm.txd[pi][0] + u[0], sy = sm.txd[pi][1] + u[1], sz = sm.txd[pi][2] + u[2];
        Q.ax = (float)wrap_pi(-S.k0 * sx * S.dx);
        Q.ay = (float)wrap_pi(-S.k0 * sy * S.dx);
        Q.gam = (float)(-S.k0 * sz);
        double p = Rs.p_ref + off * S.inv_dr;
        double kb = floor(p);
        Q.kbase = (int)kb;
        Q.pfrac = (float)(p - kb);
    }
}

// Taylor coefficients of (eta, eta_x, eta_y) in time for two facets (column ix,
// rows iya / iyb), accumulated over the wave components in shared-memory chunks.
__device__ void taylor_coeffs(Smem &sm, const MixedArgs &A, int batch, int ix, int iya, int iyb, bool va, bool vb,
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
        float2 *dst = &sm.w[0][0][0];
        for (int i = threadIdx.x; i < cnt * 3 * kOrders; i += NT) dst[i] = src[i];
        __syncthreads();
        for (int m = 0; m < cnt; ++m) {
            float2 e = __ldg(A.ex + (size_t)(m0 + m) * S.nx + ixc);
            float2 ya = __ldg(A.ey + (size_t)(m0 + m) * S.ny + iyac);
            float2 yb = __ldg(A.ey + (size_t)(m0 + m) * S.ny + iybc);
            float qar = e.x * ya.x - e.y * ya.y, qai = e.x * ya.y + e.y * ya.x;
            float qbr = e.x * yb.x - e.y * yb.y, qbi = e.x * yb.y + e.y * yb.x;
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int o = 0; o < kOrders; ++o) {
                    float2 w = sm.w[m][f][o];
                    ca[f][o] = fmaf(qar, w.x, fmaf(-qai, w.y, ca[f][o]));
                    cb[f][o] = fmaf(qbr, w.x, fmaf(-qbi, w.y, cb[f][o]));
                }
        }
    }
    (void)va;
    (void)vb;
}

__device__ __forceinline__ float horner5(const float c[kOrders], float t)
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
// 16-bin window through a shared-memory transpose, then one shared atomic per
// (bin, component) into the CTA range tile (or a global atomic outside it).
template <typename OutT>
__device__ __forceinline__ void warp_scatter(float *stage, float2 *tile_c, int tile_base, int kb, bool valid,
                                             const float h[8], float sr, float si, int nr, OutT *grow,
                                             unsigned int *flags)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int kmin = __reduce_min_sync(FULL, valid ? kb : INT_MAX);
    if (kmin == INT_MAX) return;
    int kmax = __reduce_max_sync(FULL, valid ? kb : INT_MIN);
    if (kmax - kmin <= 8) {
        int o = valid ? kb - kmin : 0;
        float4 *row = reinterpret_cast<float4 *>(stage + lane * STG);
        float a = valid ? sr : 0.0f, b = valid ? si : 0.0f;
        row[0] = make_float4(h[0] * a, h[0] * b, h[1] * a, h[1] * b);
        row[1] = make_float4(h[2] * a, h[2] * b, h[3] * a, h[3] * b);
        row[2] = make_float4(h[4] * a, h[4] * b, h[5] * a, h[5] * b);
        row[3] = make_float4(h[6] * a, h[6] * b, h[7] * a, h[7] * b);
        __syncwarp();
        const int w = lane >> 1, comp = lane & 1;
        float acc = 0.0f;
#pragma unroll 8
        for (int src = 0; src < 32; ++src) {
            int os = __shfl_sync(FULL, o, src);
            int j = w - os;
            if ((unsigned)j < 8u) acc += stage[src * STG + 2 * j + comp];
        }
        __syncwarp();
        int k = kmin + w;
        if (acc != 0.0f && k >= 0 && k < nr) {
            int tw = k - tile_base;
            if (tw >= 0 && tw < WT) {
                atomicAdd(reinterpret_cast<float *>(tile_c + tw) + comp, acc);
            } else {
                gadd1<OutT>(grow, (size_t)k, comp, acc);
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
    float xi_y;     // y offset from the tile reference point (exact)
    int jrow;       // row offset index
    float base, cu, cv;  // NRCS base and current (cell values or uniform)
    float2 z;       // speckle of the current epoch
    int epoch;      // epoch the speckle belongs to
    uint32_t fid;
    bool valid;
};

template <int TAPS, typename OutT>
__device__ __forceinline__ void facet_pulse(Smem &sm, const MixedArgs &A, const FacetGeo &G, const float c[3][kOrders],
                                            int pi, int n, int n0, int np, int buf, float xi_x, float fi, float *stage,
                                            OutT *iq)
{
    const DevScene &S = A.S;
    const PulseRec &PR = sm.pr[pi];
    const float tau = PR.tau;
    const float eta = horner5(c[0], tau);
    const float sx = horner5(c[1], tau);
    const float sy = horner5(c[2], tau);
    const float xi[3] = {xi_x, G.xi_y, eta};
    const float b2 = fmaf(xi[0], xi[0], fmaf(xi[1], xi[1], eta * eta));
    const float inv_n = rsqrtf(fmaf(sx, sx, fmaf(sy, sy, 1.0f)));
    const float fj = (float)G.jrow;

    // transmit leg (shared by the channels)
    const TxRec &T = sm.tx[pi];
    const float at = fmaf(T.u[0], xi[0], fmaf(T.u[1], xi[1], T.u[2] * xi[2]));
    const float st = fmaf(-at, at, b2);
    const float qt = st * fmaf(-at, T.inv2R2, T.inv2R);
    const float dt = at + qt;
    const float et = dt * T.invR;
    const float rho_t = fmaf(et, et, 1.0f - et);
    const float ut = (T.u0 + fmaf(xi[0], T.aR[0], fmaf(xi[1], T.aR[1], xi[2] * T.aR[2]))) * rho_t;
    const float vt = (T.v0 + fmaf(xi[0], T.eR[0], fmaf(xi[1], T.eR[1], xi[2] * T.eR[2]))) * rho_t;
    const float inv_lam = (float)S.inv_lambda;
    const float gt = sinc2f((float)S.tx_laz * inv_lam * ut) * sinc2f((float)S.tx_lel * inv_lam * vt);
    const float rt[3] = {fmaf(xi[0], T.invR, T.u[0]) * rho_t, fmaf(xi[1], T.invR, T.u[1]) * rho_t,
                         fmaf(xi[2], T.invR, T.u[2]) * rho_t};
    const float ampt = gt * T.ampr * rho_t;
    const float k0f = (float)S.k0;
    const float inv_dr = (float)S.inv_dr;

    for (int ch = 0; ch < S.nc; ++ch) {
        const RxRec &R = sm.rx[pi][ch];
        const float ar = fmaf(R.u[0], xi[0], fmaf(R.u[1], xi[1], R.u[2] * xi[2]));
        const float sr_ = fmaf(-ar, ar, b2);
        const float qr = sr_ * fmaf(-ar, R.inv2R2, R.inv2R);
        const float dr = ar + qr;
        const float er = dr * R.invR;
        const float rho_r = fmaf(er, er, 1.0f - er);
        const float ur = (R.u0 + fmaf(xi[0], R.aR[0], fmaf(xi[1], R.aR[1], xi[2] * R.aR[2]))) * rho_r;
        const float vr = (R.v0 + fmaf(xi[0], R.eR[0], fmaf(xi[1], R.eR[1], xi[2] * R.eR[2]))) * rho_r;
        const float gr = sinc2f((float)S.rx_laz[ch] * inv_lam * ur) * sinc2f((float)S.rx_lel[ch] * inv_lam * vr);
        const float qx = -(rt[0] + fmaf(xi[0], R.invR, R.u[0]) * rho_r);
        const float qy = -(rt[1] + fmaf(xi[1], R.invR, R.u[1]) * rho_r);
        const float qz = -(rt[2] + fmaf(xi[2], R.invR, R.u[2]) * rho_r);
        float sig = G.base;
        if (!S.static_surface) {
            float qh2 = fmaf(qx, qx, qy * qy);
            float cphi = qh2 > 0.0f ? fmaf((float)S.wcos, qx, (float)S.wsin * qy) * rsqrtf(qh2) : 0.0f;
            float nq = fmaf(-sx, qx, fmaf(-sy, qy, qz));
            float tilt = __fdividef(fmaxf(nq, 0.0f) * inv_n, qz);
            sig = G.base * fmaf((float)S.wind_mod, cphi, 1.0f) * tilt;
        }
        const float amp = sqrtf(sig * (float)S.area) * ampt * gr * R.ampr * rho_r;
        const float vc = -fmaf(G.cu, qx, G.cv * qy);
        float phi = R.psi + fmaf(fi, R.ax, fmaf(fj, R.ay, fmaf(R.gam, eta, -k0f * (qt + qr))));
        phi = fmaf(-PR.k0t, vc, phi);
        phi = reduce_phase(phi);
        float sp, cp;
        __sincosf(phi, &sp, &cp);
        const float zr = amp * G.z.x, zi = amp * G.z.y;
        const float vr_ = zr * cp - zi * sp;
        const float vi_ = fmaf(zr, sp, zi * cp);
        const float p = fmaf(dt + dr, inv_dr, R.pfrac);
        const float kf = floorf(p);
        const float fr = p - kf;
        int kb;
        float h[8];
        if (TAPS == 1) {
            kb = R.kbase + (int)kf;
            h[0] = 1.0f;
#pragma unroll
            for (int j = 1; j < 8; ++j) h[j] = 0.0f;
        } else {
            kb = R.kbase + (int)kf - 3;
            const float t = fmaf(2.0f, fr, -1.0f);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float v = A.tap[j][kTapDeg];
#pragma unroll
                for (int d = kTapDeg - 1; d >= 0; --d) v = fmaf(v, t, A.tap[j][d]);
                h[j] = v;
            }
        }
        float2 *tile_c = sm.tile[buf][ch];
        const int tile_base = R.kbase - WT_LO;
        OutT *grow = iq + 2 * ((size_t)ch * np + (n - n0)) * S.nr;
        warp_scatter<OutT>(stage, tile_c, tile_base, kb, G.valid, h, vr_, vi_, S.nr, grow, S.flags);
    }
}

__device__ void facet_setup(const MixedArgs &A, int ix, int iy, int jref, FacetGeo &G)
{
    const DevScene &S = A.S;
    G.valid = ix < S.nx && iy < S.ny;
    G.jrow = iy - jref;
    G.xi_y = (float)(G.jrow * S.dx);
    G.fid = (uint32_t)min(iy, S.ny - 1) * (uint32_t)S.nx + (uint32_t)min(ix, S.nx - 1);
    double base = S.sigma0_base, cu = S.cur_u, cv = S.cur_v;
    if (S.cell_sigma0 || S.cell_uv) {
        double x = (min(ix, S.nx - 1) + 0.5 - 0.5 * S.nx) * S.dx;
        double y = (min(iy, S.ny - 1) + 0.5 - 0.5 * S.ny) * S.dx;
        int cx = (int)floor((x + 0.5 * S.nx * S.dx) / S.cell);
        int cy = (int)floor((y + 0.5 * S.ny * S.dx) / S.cell);
        cx = min(max(cx, 0), S.ncx - 1);
        cy = min(max(cy, 0), S.ncy - 1);
        int ci = cy * S.ncx + cx;
        if (S.cell_sigma0) base = S.cell_sigma0[ci];
        if (S.cell_uv) {
            cu = S.cell_uv[2 * ci];
            cv = S.cell_uv[2 * ci + 1];
        }
    }
    G.base = (float)base;
    G.cu = (float)cu;
    G.cv = (float)cv;
    G.epoch = -1;
}

template <int TAPS, typename OutT>
__global__ void __launch_bounds__(NT, 2) accumulate_mixed_kernel(MixedArgs A, int n0, int np, int b0, OutT *iq)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const DevScene &S = A.S;
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

    for (int i = threadIdx.x; i < 2 * kMaxCh * WT; i += NT) (&sm.tile[0][0][0])[i] = make_float2(0.f, 0.f);
    build_refs(sm, A, pa, pe, xr, yr);

    FacetGeo ga, gb;
    facet_setup(A, ix, ty0 + warp, jref, ga);
    facet_setup(A, ix, ty0 + warp + NWARP, jref, gb);
    float ca[3][kOrders], cb[3][kOrders];
    if (!S.static_surface && S.nw > 0) {
        taylor_coeffs(sm, A, batch, ix, ty0 + warp, ty0 + warp + NWARP, ga.valid, gb.valid, ca, cb);
    } else {
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int o = 0; o < kOrders; ++o) ca[f][o] = cb[f][o] = 0.0f;
    }
    __syncthreads();

    float *stage = sm.stage[warp];
    for (int n = pa; n < pe; ++n) {
        const int pi = n - pa;
        const int buf = pi & 1;
        const int e = sm.pr[pi].epoch;
        if (e != ga.epoch) {
            ga.z = speckle_f(S.speckle_seed, ga.fid, (uint32_t)e);
            ga.epoch = e;
        }
        if (e != gb.epoch) {
            gb.z = speckle_f(S.speckle_seed, gb.fid, (uint32_t)e);
            gb.epoch = e;
        }
        facet_pulse<TAPS, OutT>(sm, A, ga, ca, pi, n, n0, np, buf, xi_x, fi, stage, iq);
        facet_pulse<TAPS, OutT>(sm, A, gb, cb, pi, n, n0, np, buf, xi_x, fi, stage, iq);
        __syncthreads();
        for (int i = threadIdx.x; i < S.nc * WT; i += NT) {
            int ch = i / WT, w = i % WT;
            float2 v = sm.tile[buf][ch][w];
            sm.tile[buf][ch][w] = make_float2(0.f, 0.f);
            int k = sm.rx[pi][ch].kbase - WT_LO + w;
            if ((v.x != 0.0f || v.y != 0.0f) && k >= 0 && k < S.nr)
                gadd<OutT>(iq + 2 * ((size_t)ch * np + (n - n0)) * S.nr, (size_t)k, v.x, v.y);
        }
    }
}

// Facet generator of the mixed path: same Taylor expansion, states written out.
__global__ void __launch_bounds__(NT, 2) generate_mixed_kernel(MixedArgs A, int n0, int np, int b0, float *state)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const DevScene &S = A.S;
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
        taylor_coeffs(sm, A, batch, ix, iya, iyb, va, vb, ca, cb);
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
            o[f] = horner5(ca[0], tau);
            o[nf + f] = horner5(ca[1], tau);
            o[2 * nf + f] = horner5(ca[2], tau);
        }
        if (vb) {
            int64_t f = (int64_t)iyb * S.nx + ix;
            o[f] = horner5(cb[0], tau);
            o[nf + f] = horner5(cb[1], tau);
            o[2 * nf + f] = horner5(cb[2], tau);
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
    for (int j = 0; j < 8; ++j)
        for (int d = 0; d <= kTapDeg; ++d) A.tap[j][d] = M.tap[j][d];
    return A;
}

template <typename K>
cudaError_t set_smem(K kernel)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
}

}  // namespace

cudaError_t launch_generate_mixed(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                                  float *state)
{
    MixedArgs A = make_args(S, M);
    cudaError_t e = set_smem(generate_mixed_kernel);
    if (e != cudaSuccess) return e;
    int tiles = ((S.nx + TX - 1) / TX) * ((S.ny + TY - 1) / TY);
    int b0 = n0 / M.nb, b1 = (n0 + np - 1) / M.nb;
    for (int bb = b0; bb <= b1; bb += 65535) {
        int cnt = min(65535, b1 - bb + 1);
        generate_mixed_kernel<<<dim3(tiles, cnt), NT, sizeof(Smem), st>>>(A, n0, np, bb, state);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_accumulate_mixed(const DevScene &S, const MixedTables &M, cudaStream_t st, int n0, int np,
                                    void *iq, harm_dtype dtype)
{
    MixedArgs A = make_args(S, M);
    int tiles = ((S.nx + TX - 1) / TX) * ((S.ny + TY - 1) / TY);
    int b0 = n0 / M.nb, b1 = (n0 + np - 1) / M.nb;
    cudaError_t e;
    for (int bb = b0; bb <= b1; bb += 65535) {
        int cnt = min(65535, b1 - bb + 1);
        dim3 grid(tiles, cnt);
        if (dtype == HARM_C64) {
            if (S.taps == 1) {
                if ((e = set_smem(accumulate_mixed_kernel<1, float>)) != cudaSuccess) return e;
                accumulate_mixed_kernel<1, float><<<grid, NT, sizeof(Smem), st>>>(A, n0, np, bb, (float *)iq);
            } else {
                if ((e = set_smem(accumulate_mixed_kernel<8, float>)) != cudaSuccess) return e;
                accumulate_mixed_kernel<8, float><<<grid, NT, sizeof(Smem), st>>>(A, n0, np, bb, (float *)iq);
            }
        } else {
            if (S.taps == 1) {
                if ((e = set_smem(accumulate_mixed_kernel<1, double>)) != cudaSuccess) return e;
                accumulate_mixed_kernel<1, double><<<grid, NT, sizeof(Smem), st>>>(A, n0, np, bb, (double *)iq);
            } else {
                if ((e = set_smem(accumulate_mixed_kernel<8, double>)) != cudaSuccess) return e;
                accumulate_mixed_kernel<8, double><<<grid, NT, sizeof(Smem), st>>>(A, n0, np, bb, (double *)iq);
            }
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int mixed_batch_pulses() { return NBMAX; }

}  // namespace harm
