// Plain paths: facet generator and echo accumulator with every per-facet step in
// one real type R -- double (HARM_PREC_FP64, the reference GPU form the mixed
// path is measured against) or float (HARM_PREC_FP32: the same method in single
// precision, which shows what the mixed path's FP64 references are for).
//
// Both evaluate the method as written: each facet's ranges to the transmitter and
// receiver (in the stable offset form (|x|^2 - 2 P.x) / (r + |P|) from the scene-
// centre range), unit vectors, patterns, NRCS, phase and taps. The per-pulse
// state (platform positions, steered frames, the reduced reference phase and the
// range-bin offset of the scene centre) is built in FP64 on the host for every
// path; the FP32 path reads it rounded to float.
//
// Work decomposition: one CTA = a 16 x 16 facet tile x one pulse; one thread per
// facet. Each thread synthesises its facet's state (linear waves or the Choppy
// Wave Model, one wave set or the four corner sets of a heterogeneous sea state,
// separable phasors), then for every channel forms the contribution of Eq. 3 /
// Eq. 16 (analytic or u-v grid gains, AR(1) speckle of Eq. 10 with the Doppler
// rotation of Eq. 7) and spreads it over the range bins (Eq. 17 box or 8-tap
// Kaiser-sinc) into a shared-memory range tile of the CTA. The tile is flushed to
// the IQ with one atomic per bin and channel.
#include <cuda_runtime.h>

#include <algorithm>

#include "harm_internal.cuh"
#include "harm_kernels.cuh"
#include "philox.cuh"

namespace harm {
namespace {

constexpr int kTile = 16;     // facets per tile edge
constexpr int kWin = 64;      // range bins per channel in the CTA tile

// Math of one real type.
template <typename R>
struct M;
template <>
struct M<double> {
    using R2 = double2;
    __device__ static double sqrt_(double x) { return sqrt(x); }
    __device__ static double sinpi_(double x) { return sinpi(x); }
    __device__ static void sincos_(double x, double *s, double *c) { sincos(x, s, c); }
    __device__ static void sincospi_(double x, double *s, double *c) { sincospi(x, s, c); }
    __device__ static double log_(double x) { return log(x); }
    __device__ static double2 pair(double a, double b) { return make_double2(a, b); }
    __device__ static const double2 *ex(const DevScene &S) { return S.ex; }
    __device__ static const double2 *ey(const DevScene &S) { return S.ey; }
    __device__ static const double2 *tt(const DevScene &S) { return S.tt; }
};
template <>
struct M<float> {
    using R2 = float2;
    __device__ static float sqrt_(float x) { return sqrtf(x); }
    __device__ static float sinpi_(float x) { return sinpif(x); }
    __device__ static void sincos_(float x, float *s, float *c) { sincosf(x, s, c); }
    __device__ static void sincospi_(float x, float *s, float *c) { sincospif(x, s, c); }
    __device__ static float log_(float x) { return logf(x); }
    __device__ static float2 pair(float a, float b) { return make_float2(a, b); }
    __device__ static const float2 *ex(const DevScene &S) { return S.ex32; }
    __device__ static const float2 *ey(const DevScene &S) { return S.ey32; }
    __device__ static const float2 *tt(const DevScene &S) { return S.tt32; }
};

template <typename R>
__device__ __forceinline__ R dot3(const R a[3], const R b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

template <typename R>
__device__ __forceinline__ void load3(const double v[3], R o[3])
{
    o[0] = (R)v[0];
    o[1] = (R)v[1];
    o[2] = (R)v[2];
}

// sinc(x) = sin(pi x) / (pi x)
template <typename R>
__device__ __forceinline__ R sinc(R x)
{
    if (x == R(0)) return R(1);
    return M<R>::sinpi_(x) / (R(kPi) * x);
}

// sinc^2 azimuth x sinc^2 elevation field gain for unit direction d (antenna
// axes a, e; aperture lengths over the wavelength).
template <typename R>
__device__ __forceinline__ R gain(const R a[3], const R e[3], R laz_l, R lel_l, const R d[3])
{
    const R sa = sinc<R>(laz_l * dot3(d, a));
    const R se = sinc<R>(lel_l * dot3(d, e));
    return sa * sa * se * se;
}

// Complex gain from a u-v grid (Sec. III-B): bilinear between the four nodes
// around (u, v), zero outside the grid (grid values stored in double).
template <typename R>
__device__ typename M<R>::R2 lut_gain(const PatLut &L, R u, R v)
{
    const R fu = (u - (R)L.u0) * (R)L.inv_du, fv = (v - (R)L.v0) * (R)L.inv_dv;
    if (!(fu >= R(0) && fu <= (R)(L.nu - 1) && fv >= R(0) && fv <= (R)(L.nv - 1))) return M<R>::pair(R(0), R(0));
    const int iu = min((int)floor(fu), L.nu - 2), iv = min((int)floor(fv), L.nv - 2);
    const R a = fu - (R)iu, b = fv - (R)iv;
    const double2 *g = L.g64 + (size_t)iv * L.nu + iu;
    const double2 g00 = g[0], g10 = g[1], g01 = g[L.nu], g11 = g[L.nu + 1];
    const R w00 = (R(1) - a) * (R(1) - b), w10 = a * (R(1) - b), w01 = (R(1) - a) * b, w11 = a * b;
    return M<R>::pair(w00 * (R)g00.x + w10 * (R)g10.x + w01 * (R)g01.x + w11 * (R)g11.x,
                      w00 * (R)g00.y + w10 * (R)g10.y + w01 * (R)g01.y + w11 * (R)g11.y);
}

// Gain of antenna slot (0 = transmitter, 1 + c = receive channel c) for unit
// direction d: the u-v grid when one is set, else the analytic pattern.
template <typename R>
__device__ __forceinline__ typename M<R>::R2 antenna_gain(const DevScene &S, int slot, const R a[3], const R e[3],
                                                          R laz_l, R lel_l, const R d[3])
{
    if (S.lut_mask & (1u << slot)) return lut_gain<R>(S.luts[slot], dot3(d, a), dot3(d, e));
    return M<R>::pair(gain<R>(a, e, laz_l, lel_l, d), R(0));
}

// Fields of one wave set q at rest position (ix, iy), pulse n, added with weight
// w: with Q E = a e^{i(k.x + phi)} e^{-i omega t_s} = (vr, vi),
// eta = vr, slopes -k vi, and for the Choppy Wave Model the horizontal
// displacement -(k / |k|) vi and its gradient -(k_i k_j / |k|) vr.
template <typename R>
__device__ void wave_set(const DevScene &S, int q, int ix, int iy, int n, R w, R st[8])
{
    using R2 = typename M<R>::R2;
    const size_t base = (size_t)q * S.nw;
    const R2 *px = M<R>::ex(S) + base * S.nx + ix;
    const R2 *py = M<R>::ey(S) + base * S.ny + iy;
    const R2 *pt = M<R>::tt(S) + base * S.np_total + n;
    for (int m = 0; m < S.nw; ++m) {
        const R2 a = __ldg(px + (size_t)m * S.nx);
        const R2 b = __ldg(py + (size_t)m * S.ny);
        const R2 t = __ldg(pt + (size_t)m * S.np_total);
        const R qr = a.x * b.x - a.y * b.y;
        const R qi = a.x * b.y + a.y * b.x;
        const R vr = w * (qr * t.x - qi * t.y);
        const R vi = w * (qr * t.y + qi * t.x);
        const R kx = (R)__ldg(S.kx + base + m), ky = (R)__ldg(S.ky + base + m);
        st[0] += vr;
        st[1] -= kx * vi;
        st[2] -= ky * vi;
        if (S.cwm) {
            const R ik = R(1) / (R)__ldg(S.kn + base + m);
            const R ux = kx * ik, uy = ky * ik;
            st[3] -= ux * vi;
            st[4] -= uy * vi;
            st[5] -= ux * kx * vr;
            st[6] -= ux * ky * vr;
            st[7] -= uy * ky * vr;
        }
    }
}

// Facet state (8 fields; the last 5 zero without the Choppy Wave Model) at rest
// position (ix, iy), pulse n. A heterogeneous sea state sums the wave sets of
// the four corners of the facet's TL tile with the weights of Eq. 2 (Eq. 1).
template <typename R>
__device__ void facet_state(const DevScene &S, int ix, int iy, int n, R st[8])
{
    for (int q = 0; q < 8; ++q) st[q] = R(0);
    if (S.static_surface || S.nw == 0) return;
    if (S.het_ncx > 0) {
        const R x = (R)((ix + 0.5 - 0.5 * S.nx) * S.dx), y = (R)((iy + 0.5 - 0.5 * S.ny) * S.dx);
        const R l = (R)S.het_l, x0 = (R)S.het_x0, y0 = (R)S.het_y0;
        const int tx = min(max((int)floor((x - x0) / l), 0), S.het_ncx - 2);
        const int ty = min(max((int)floor((y - y0) / l), 0), S.het_ncy - 2);
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const int cx = tx + dx, cy = ty + dy;
                const R wx = fabs(x0 + (R)cx * l - x) / l;
                const R wy = fabs(y0 + (R)cy * l - y) / l;
                const R v = R(1) - wx - wy + wx * wy;
                if (!(v > R(0))) continue;
                wave_set<R>(S, cy * S.het_ncx + cx, ix, iy, n, M<R>::sqrt_(v), st);
            }
    } else {
        wave_set<R>(S, 0, ix, iy, n, R(1), st);
    }
}

// Intra-facet speckle (Eq. 7 at f_s = 0): Box-Muller on the Philox words w of the
// facet's counter, R, I ~ N(0, 1/2).
template <typename R>
__device__ __forceinline__ void box_muller(const U32x4 &w, R &zr, R &zi)
{
    const R u1 = ((R)w.x + R(1)) * R(0x1p-32);
    const R u2 = (R)w.y * R(0x1p-32);
    const R rad = M<R>::sqrt_(-M<R>::log_(u1));
    R s, c;
    M<R>::sincospi_(R(2) * u2, &s, &c);
    zr = rad * c;
    zi = rad * s;
}

// Speckle under the order-1 autoregressive model of Eq. 10: s_0 = w_0,
// s_e = beta s_(e-1) + sqrt(1 - beta^2) w_e, run from epoch 0.
template <typename R>
__device__ void speckle_ar1(const DevScene &S, uint32_t f, uint32_t epoch, R &zr, R &zi)
{
    if (S.spk_beta == 0.0) {
        box_muller<R>(philox_stream(S.speckle_seed, kStreamSpeckle, f, epoch), zr, zi);
        return;
    }
    box_muller<R>(philox_stream(S.speckle_seed, kStreamSpeckle, f, 0u), zr, zi);
    const R b = (R)S.spk_beta, q = (R)S.spk_q;
    for (uint32_t e = 1; e <= epoch; ++e) {
        R wr, wi;
        box_muller<R>(philox_stream(S.speckle_seed, kStreamSpeckle, f, e), wr, wi);
        zr = b * zr + q * wr;
        zi = b * zi + q * wi;
    }
}

// Kaiser window I0(beta sqrt(1 - (x/4)^2)) / I0(beta) from its power series in
// v = 1 - (x/4)^2 (coefficients prepared on the host), times sinc(x).
template <typename R>
__device__ __forceinline__ R kaiser_sinc(const DevScene &S, R x, R sin_pf, int j)
{
    const R q = R(0.25) * x;
    const R v = R(1) - q * q;
    if (v <= R(0)) return R(0);
    R w = (R)S.i0c[S.n_i0 - 1];
    for (int k = S.n_i0 - 2; k >= 0; --k) w = fma(w, v, (R)S.i0c[k]);
    // sin(pi (j - f)) = -(-1)^j sin(pi f)
    const R sn = (j & 1) ? sin_pf : -sin_pf;
    const R sc = (x == R(0)) ? R(1) : sn / (R(kPi) * x);
    return sc * w;
}

template <typename OutT, typename R>
__device__ __forceinline__ void global_add(OutT *iq, size_t idx, R re, R im)
{
    atomicAdd(iq + 2 * idx, (OutT)re);
    atomicAdd(iq + 2 * idx + 1, (OutT)im);
}

// Deterministic sums: every contribution is rounded to a multiple of 2^-40 and
// added as a 64-bit integer (two's complement), so that the sum is exact and does
// not depend on the order of the atomic additions (reproducible summation by
// fixed-point accumulation). Range: |sum| < 2^23 per component.
constexpr double kFixedScale = 1099511627776.0;  // 2^40
constexpr double kFixedLimit = 8388608.0;        // 2^23

__device__ __forceinline__ unsigned long long to_fixed(double v)
{
    return (unsigned long long)__double2ll_rn(v * kFixedScale);
}

__device__ __forceinline__ void fixed_add(unsigned long long *p, double re, double im)
{
    atomicAdd(p, to_fixed(re));
    atomicAdd(p + 1, to_fixed(im));
}

// In-place conversions of an IQ buffer of n doubles between FP64 and the fixed
// point of the deterministic sums (values outside the range are clamped and
// counted in flags[1]).
__global__ void fixed_from_double_kernel(double *v, size_t n, unsigned int *flags)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double x = v[i];
        if (!(fabs(x) < kFixedLimit)) {
            atomicAdd(flags + 1, 1u);
            x = x > 0.0 ? kFixedLimit : (x < 0.0 ? -kFixedLimit : 0.0);
        }
        reinterpret_cast<unsigned long long *>(v)[i] = to_fixed(x);
    }
}

__global__ void double_from_fixed_kernel(double *v, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        v[i] = (double)reinterpret_cast<const long long *>(v)[i] * (1.0 / kFixedScale);
}

template <typename R>
__global__ void __launch_bounds__(256) generate_plain_kernel(DevScene S, int n0, int nfirst, R *state)
{
    const int64_t nf = (int64_t)S.nx * S.ny;
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = nfirst + blockIdx.y;
    if (f >= nf) return;
    const int ix = (int)(f % S.nx), iy = (int)(f / S.nx);
    R st[8];
    facet_state<R>(S, ix, iy, n, st);
    const int nfl = S.cwm ? 8 : 3;
    R *o = state + (size_t)(n - n0) * nfl * nf;
    for (int q = 0; q < nfl; ++q) o[q * nf + f] = st[q];
}

// Index probe of the plain paths (see harm_probe_indices): per facet and pulse
// the first tap bin in every channel, the speckle draw, its Philox words and the
// cell index, written instead of the contributions.
template <typename R>
struct PlainProbe {
    int *bins;                 // [np][nc][nf]
    typename M<R>::R2 *speckle;  // [np][nf]
    uint4 *words;              // [np][nf]
    int *cells;                // [nf]
};

// DET: deterministic fixed-point sums (see to_fixed; OutT double, the IQ buffer
// holding fixed-point values during the launch).
template <typename R, int TAPS, typename OutT, bool PROBE, bool DET>
__global__ void __launch_bounds__(256)
    accumulate_plain_kernel(DevScene S, int n0, int np, int nfirst, OutT *iq, PlainProbe<R> probe)
{
    using R2 = typename M<R>::R2;
    static_assert(!DET || sizeof(OutT) == 8, "deterministic sums need complex128 output");
    // range tile of the CTA: R2 values, or (re, im) fixed-point pairs
    __shared__ __align__(16) unsigned char tile_raw[kMaxCh * kWin * (DET ? 16 : sizeof(R2))];
    R2(*tile)[kWin] = reinterpret_cast<R2(*)[kWin]>(tile_raw);
    unsigned long long(*tileq)[kWin][2] = reinterpret_cast<unsigned long long(*)[kWin][2]>(tile_raw);
    unsigned long long *iqq = reinterpret_cast<unsigned long long *>(iq);
    __shared__ int kbase[kMaxCh];

    const int tiles_x = (S.nx + kTile - 1) / kTile;
    const int tx0 = (blockIdx.x % tiles_x) * kTile;
    const int ty0 = (blockIdx.x / tiles_x) * kTile;
    const int ix = tx0 + (threadIdx.x % kTile);
    const int iy = ty0 + (threadIdx.x / kTile);
    const bool valid = ix < S.nx && iy < S.ny;
    const int n = nfirst + blockIdx.y;
    const int nr = S.nr;
    const PulseState &P = S.pulses[n];

    for (int i = threadIdx.x; i < S.nc * kWin; i += blockDim.x) {
        if constexpr (DET) {
            tileq[i / kWin][i % kWin][0] = 0ull;
            tileq[i / kWin][i % kWin][1] = 0ull;
        } else {
            tile[i / kWin][i % kWin] = M<R>::pair(R(0), R(0));
        }
    }
    // Window base per channel from the tile centre on the mean surface (FP64: a
    // per-tile value that only places the shared-memory window).
    if (threadIdx.x < S.nc) {
        const int c = threadIdx.x;
        const RxState &Rs = S.rx[(size_t)n * S.nc + c];
        double xc[3] = {(tx0 + 0.5 * kTile - 0.5 * S.nx) * S.dx, (ty0 + 0.5 * kTile - 0.5 * S.ny) * S.dx, 0.0};
        double dt[3] = {xc[0] - P.tx.p[0], xc[1] - P.tx.p[1], xc[2] - P.tx.p[2]};
        double dr[3] = {xc[0] - Rs.rx.p[0], xc[1] - Rs.rx.p[1], xc[2] - Rs.rx.p[2]};
        double rsum = sqrt(dt[0] * dt[0] + dt[1] * dt[1] + dt[2] * dt[2]) +
                      sqrt(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]);
        double pc = Rs.p_ref + (rsum - P.tx.rref - Rs.rx.rref) * S.inv_dr;
        kbase[c] = (int)floor(pc) - kWin / 2;
    }
    __syncthreads();

    if (valid) {
        const uint32_t f = (uint32_t)iy * (uint32_t)S.nx + (uint32_t)ix;
        const size_t nfac = (size_t)S.nx * S.ny;
        R st[8];
        facet_state<R>(S, ix, iy, n, st);
        // rest position, moved by the horizontal displacement (CWM) and lifted to eta
        const R xb = (R)((ix + 0.5 - 0.5 * S.nx) * S.dx), yb = (R)((iy + 0.5 - 0.5 * S.ny) * S.dx);
        const R x[3] = {xb + st[3], yb + st[4], st[0]};
        const R xx = dot3(x, x);
        // normal: cross product of the displaced surface's tangents
        // (1 + dDx/dx, dDx/dy, eta_x) and (dDx/dy, 1 + dDy/dy, eta_y)
        const R nv[3] = {st[6] * st[2] - st[1] * (R(1) + st[7]), st[1] * st[6] - (R(1) + st[5]) * st[2],
                         (R(1) + st[5]) * (R(1) + st[7]) - st[6] * st[6]};
        const R nlen = M<R>::sqrt_(dot3(nv, nv));
        const R area = (R)S.area * fmax(nv[2], R(0));
        const R k0 = (R)S.k0, inv_dr = (R)S.inv_dr, inv_lambda = (R)S.inv_lambda;

        // transmit leg: range offset from the scene-centre range in the stable
        // form (|x|^2 - 2 P.x) / (r + R), unit vector, pattern gain
        R pt[3], at[3], et[3];
        load3(P.tx.p, pt);
        load3(P.tx.a, at);
        load3(P.tx.e, et);
        const R rref_t = (R)P.tx.rref;
        const R dtv[3] = {x[0] - pt[0], x[1] - pt[1], x[2] - pt[2]};
        const R rt = M<R>::sqrt_(dot3(dtv, dtv));
        const R delt = (xx - R(2) * dot3(pt, x)) / (rt + rref_t);
        const R ut[3] = {dtv[0] / rt, dtv[1] / rt, dtv[2] / rt};
        const R2 gt = antenna_gain<R>(S, 0, at, et, (R)(S.tx_laz * S.inv_lambda), (R)(S.tx_lel * S.inv_lambda), ut);

        R base = (R)S.sigma0_base, cu = (R)S.cur_u, cv = (R)S.cur_v;
        int cell = -1;
        if (S.ncx > 0) {
            int cx = (int)floor(((ix + 0.5 - 0.5 * S.nx) * S.dx + 0.5 * S.nx * S.dx) / S.cell);
            int cy = (int)floor(((iy + 0.5 - 0.5 * S.ny) * S.dx + 0.5 * S.ny * S.dx) / S.cell);
            cx = min(max(cx, 0), S.ncx - 1);
            cy = min(max(cy, 0), S.ncy - 1);
            cell = cy * S.ncx + cx;
            if (S.cell_sigma0) base = (R)S.cell_sigma0[cell];
            if (S.cell_uv) {
                cu = (R)S.cell_uv[2 * cell];
                cv = (R)S.cell_uv[2 * cell + 1];
            }
        }
        const uint32_t epoch = S.epoch_pulses > 0 ? (uint32_t)(n / S.epoch_pulses) : 0u;
        R zr, zi;
        speckle_ar1<R>(S, f, epoch, zr, zi);
        const R tn = (R)P.t;
        const R fd_phase = (R)(2.0 * kPi * S.fd_hz * P.t);
        if constexpr (PROBE) {
            const size_t p = (size_t)(n - n0);
            probe.speckle[p * nfac + f] = M<R>::pair(zr, zi);
            const U32x4 w = philox_stream(S.speckle_seed, kStreamSpeckle, f, epoch);
            probe.words[p * nfac + f] = make_uint4(w.x, w.y, w.z, w.w);
            if (n == n0) probe.cells[f] = cell;
        }

        for (int c = 0; c < S.nc; ++c) {
            const RxState &Rs = S.rx[(size_t)n * S.nc + c];
            R pr[3], ar[3], er[3];
            load3(Rs.rx.p, pr);
            load3(Rs.rx.a, ar);
            load3(Rs.rx.e, er);
            const R rref_r = (R)Rs.rx.rref;
            const R drv[3] = {x[0] - pr[0], x[1] - pr[1], x[2] - pr[2]};
            const R rr = M<R>::sqrt_(dot3(drv, drv));
            const R delr = (xx - R(2) * dot3(pr, x)) / (rr + rref_r);
            const R p = (R)Rs.p_ref + (delt + delr) * inv_dr;
            const R fk = floor(p);
            if constexpr (PROBE) {
                probe.bins[((size_t)(n - n0) * S.nc + c) * nfac + f] = (int)fk - (TAPS == 1 ? 0 : 3);
                continue;
            }
            const R ur[3] = {drv[0] / rr, drv[1] / rr, drv[2] / rr};
            const R2 gr = antenna_gain<R>(S, 1 + c, ar, er, (R)(S.rx_laz[c] * S.inv_lambda),
                                          (R)(S.rx_lel[c] * S.inv_lambda), ur);
            R sig = base;
            if (!S.static_surface) {
                const R q[3] = {-(ut[0] + ur[0]), -(ut[1] + ur[1]), -(ut[2] + ur[2])};
                const R qh = M<R>::sqrt_(q[0] * q[0] + q[1] * q[1]);
                const R cphi = qh > R(0) ? ((R)S.wcos * q[0] + (R)S.wsin * q[1]) / qh : R(0);
                const R nq = dot3(nv, q);
                const R tilt = fmax(nq, R(0)) / (nlen * q[2]);
                sig = base * (R(1) + (R)S.wind_mod * cphi) * tilt;
            }
            const R amp = M<R>::sqrt_(sig * area) * (rref_t / rt) * (rref_r / rr);
            const R vc = cu * (ut[0] + ur[0]) + cv * (ut[1] + ur[1]);
            const R phase = (R)Rs.psi - k0 * (delt + delr + vc * tn) + fd_phase;
            R sp, cp;
            M<R>::sincos_(phase, &sp, &cp);
            // field weight G_t G_r (complex for u-v grids) times the speckle
            const R gre = gt.x * gr.x - gt.y * gr.y, gim = gt.x * gr.y + gt.y * gr.x;
            const R are = amp * (zr * gre - zi * gim), aim = amp * (zr * gim + zi * gre);
            const R vr = are * cp - aim * sp;
            const R vi = are * sp + aim * cp;
            if (TAPS == 1) {
                if (fk >= R(0) && fk < (R)nr) {
                    const int k = (int)fk;
                    const int w = k - kbase[c];
                    if (DET && w >= 0 && w < kWin) {
                        fixed_add(tileq[c][w], (double)vr, (double)vi);
                    } else if (DET) {
                        fixed_add(iqq + 2 * (((size_t)c * np + (n - n0)) * nr + k), (double)vr, (double)vi);
                    } else if (w >= 0 && w < kWin) {
                        atomicAdd(&tile[c][w].x, vr);
                        atomicAdd(&tile[c][w].y, vi);
                    } else {
                        global_add<OutT, R>(iq, ((size_t)c * np + (n - n0)) * nr + k, vr, vi);
                    }
                }
            } else {
                if (fk < R(-8) || fk > (R)nr + R(8)) continue;
                const int k0i = (int)fk;
                const R fr = p - fk;
                const R spf = M<R>::sinpi_(fr);
#pragma unroll
                for (int j = -3; j <= 4; ++j) {
                    const int k = k0i + j;
                    if (k < 0 || k >= nr) continue;
                    const R h = kaiser_sinc<R>(S, (R)j - fr, spf, j);
                    const int w = k - kbase[c];
                    if (DET && w >= 0 && w < kWin) {
                        fixed_add(tileq[c][w], (double)(h * vr), (double)(h * vi));
                    } else if (DET) {
                        fixed_add(iqq + 2 * (((size_t)c * np + (n - n0)) * nr + k), (double)(h * vr),
                                  (double)(h * vi));
                    } else if (w >= 0 && w < kWin) {
                        atomicAdd(&tile[c][w].x, h * vr);
                        atomicAdd(&tile[c][w].y, h * vi);
                    } else {
                        global_add<OutT, R>(iq, ((size_t)c * np + (n - n0)) * nr + k, h * vr, h * vi);
                    }
                }
            }
        }
    }
    if constexpr (PROBE) return;
    __syncthreads();
    for (int i = threadIdx.x; i < S.nc * kWin; i += blockDim.x) {
        const int c = i / kWin, w = i % kWin;
        const int k = kbase[c] + w;
        if (k < 0 || k >= nr) continue;
        if constexpr (DET) {
            const unsigned long long re = tileq[c][w][0], im = tileq[c][w][1];
            unsigned long long *o = iqq + 2 * (((size_t)c * np + (n - n0)) * nr + k);
            if (re) atomicAdd(o, re);
            if (im) atomicAdd(o + 1, im);
        } else {
            const R2 v = tile[c][w];
            if (v.x != R(0) || v.y != R(0)) global_add<OutT, R>(iq, ((size_t)c * np + (n - n0)) * nr + k, v.x, v.y);
        }
    }
}

template <typename R>
cudaError_t generate_r(const DevScene &S, cudaStream_t st, int n0, int np, R *state)
{
    const int64_t nf = (int64_t)S.nx * S.ny;
    for (int p0 = 0; p0 < np; p0 += 65535) {
        const int cnt = min(65535, np - p0);
        dim3 grid((unsigned)((nf + 255) / 256), (unsigned)cnt);
        generate_plain_kernel<R><<<grid, 256, 0, st>>>(S, n0, n0 + p0, state);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename R, int TAPS, typename OutT, bool PROBE, bool DET = false>
cudaError_t accumulate_r(const DevScene &S, cudaStream_t st, int n0, int np, OutT *iq, const PlainProbe<R> &probe)
{
    const int tiles = ((S.nx + kTile - 1) / kTile) * ((S.ny + kTile - 1) / kTile);
    for (int p0 = 0; p0 < np; p0 += 65535) {
        const int cnt = min(65535, np - p0);
        dim3 grid((unsigned)tiles, (unsigned)cnt);
        accumulate_plain_kernel<R, TAPS, OutT, PROBE, DET><<<grid, 256, 0, st>>>(S, n0, np, n0 + p0, iq, probe);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Deterministic sums into a complex128 IQ: the buffer is converted to fixed point
// in place (so that it may already hold values to add to), accumulated with
// integer atomics, and converted back.
template <typename R>
cudaError_t accumulate_det(const DevScene &S, cudaStream_t st, int n0, int np, double *iq)
{
    const size_t n = (size_t)2 * S.nc * np * S.nr;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 148 * 8);
    fixed_from_double_kernel<<<blocks, 256, 0, st>>>(iq, n, S.flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const PlainProbe<R> none{};
    e = S.taps == 1 ? accumulate_r<R, 1, double, false, true>(S, st, n0, np, iq, none)
                    : accumulate_r<R, 8, double, false, true>(S, st, n0, np, iq, none);
    if (e != cudaSuccess) return e;
    double_from_fixed_kernel<<<blocks, 256, 0, st>>>(iq, n);
    return cudaGetLastError();
}

template <typename R>
cudaError_t accumulate_dtype(const DevScene &S, cudaStream_t st, int n0, int np, void *iq, harm_dtype dtype)
{
    const PlainProbe<R> none{};
    if (S.det) {
        if (dtype != HARM_C128) return cudaErrorNotSupported;
        return accumulate_det<R>(S, st, n0, np, (double *)iq);
    }
    if (dtype == HARM_C128)
        return S.taps == 1 ? accumulate_r<R, 1, double, false>(S, st, n0, np, (double *)iq, none)
                           : accumulate_r<R, 8, double, false>(S, st, n0, np, (double *)iq, none);
    return S.taps == 1 ? accumulate_r<R, 1, float, false>(S, st, n0, np, (float *)iq, none)
                       : accumulate_r<R, 8, float, false>(S, st, n0, np, (float *)iq, none);
}

template <typename R>
cudaError_t probe_r(const DevScene &S, cudaStream_t st, int n0, int np, int *bins, void *speckle, void *words,
                    int *cells)
{
    PlainProbe<R> pr;
    pr.bins = bins;
    pr.speckle = reinterpret_cast<typename M<R>::R2 *>(speckle);
    pr.words = reinterpret_cast<uint4 *>(words);
    pr.cells = cells;
    return S.taps == 1 ? accumulate_r<R, 1, float, true>(S, st, n0, np, nullptr, pr)
                       : accumulate_r<R, 8, float, true>(S, st, n0, np, nullptr, pr);
}

}  // namespace

cudaError_t launch_generate_plain(const DevScene &S, bool fp64, cudaStream_t st, int n0, int np, void *state)
{
    return fp64 ? generate_r<double>(S, st, n0, np, (double *)state) : generate_r<float>(S, st, n0, np, (float *)state);
}

cudaError_t launch_accumulate_plain(const DevScene &S, bool fp64, cudaStream_t st, int n0, int np, void *iq,
                                    harm_dtype dtype)
{
    return fp64 ? accumulate_dtype<double>(S, st, n0, np, iq, dtype) : accumulate_dtype<float>(S, st, n0, np, iq, dtype);
}

cudaError_t launch_probe_plain(const DevScene &S, bool fp64, cudaStream_t st, int n0, int np, int *bins,
                               void *speckle, void *words, int *cells)
{
    return fp64 ? probe_r<double>(S, st, n0, np, bins, speckle, words, cells)
                : probe_r<float>(S, st, n0, np, bins, speckle, words, cells);
}

}  // namespace harm
