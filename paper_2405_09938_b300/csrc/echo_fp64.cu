// Plain FP64 path: facet generator and echo accumulator with every step in
// double precision (the reference GPU form the mixed path is measured against).
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

#include "harm_internal.cuh"
#include "harm_kernels.cuh"
#include "philox.cuh"

namespace harm {
namespace {

constexpr int kTile = 16;     // facets per tile edge
constexpr int kWin = 64;      // range bins per channel in the CTA tile

__device__ __forceinline__ double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// sinc(x) = sin(pi x) / (pi x)
__device__ __forceinline__ double sinc_d(double x)
{
    if (x == 0.0) return 1.0;
    return sinpi(x) / (kPi * x);
}

// sinc^2 azimuth x sinc^2 elevation field gain for unit direction d.
__device__ __forceinline__ double gain_d(const AntState &s, double laz, double lel, double inv_lambda,
                                         const double d[3])
{
    double sa = sinc_d(laz * inv_lambda * dot3(d, s.a));
    double se = sinc_d(lel * inv_lambda * dot3(d, s.e));
    return sa * sa * se * se;
}

// Complex gain from a u-v grid (Sec. III-B): bilinear between the four nodes
// around (u, v), zero outside the grid.
__device__ double2 lut_gain_d(const PatLut &L, double u, double v)
{
    const double fu = (u - L.u0) * L.inv_du, fv = (v - L.v0) * L.inv_dv;
    if (!(fu >= 0.0 && fu <= (double)(L.nu - 1) && fv >= 0.0 && fv <= (double)(L.nv - 1)))
        return make_double2(0.0, 0.0);
    const int iu = min((int)floor(fu), L.nu - 2), iv = min((int)floor(fv), L.nv - 2);
    const double a = fu - iu, b = fv - iv;
    const double2 *g = L.g64 + (size_t)iv * L.nu + iu;
    const double2 g00 = g[0], g10 = g[1], g01 = g[L.nu], g11 = g[L.nu + 1];
    const double w00 = (1.0 - a) * (1.0 - b), w10 = a * (1.0 - b), w01 = (1.0 - a) * b, w11 = a * b;
    return make_double2(w00 * g00.x + w10 * g10.x + w01 * g01.x + w11 * g11.x,
                        w00 * g00.y + w10 * g10.y + w01 * g01.y + w11 * g11.y);
}

// Gain of antenna slot (0 = transmitter, 1 + c = receive channel c) for unit
// direction d: the u-v grid when one is set, else the analytic pattern.
__device__ __forceinline__ double2 antenna_gain_d(const DevScene &S, int slot, const AntState &a, double laz,
                                                  double lel, const double d[3])
{
    if (S.lut_mask & (1u << slot)) return lut_gain_d(S.luts[slot], dot3(d, a.a), dot3(d, a.e));
    return make_double2(gain_d(a, laz, lel, S.inv_lambda, d), 0.0);
}

// Fields of one wave set q at rest position (ix, iy), pulse n, added with weight
// w: with Q E = a e^{i(k.x + phi)} e^{-i omega t_s} = (vr, vi),
// eta = vr, slopes -k vi, and for the Choppy Wave Model the horizontal
// displacement -(k / |k|) vi and its gradient -(k_i k_j / |k|) vr.
__device__ void wave_set_d(const DevScene &S, int q, int ix, int iy, int n, double w, double st[8])
{
    const size_t base = (size_t)q * S.nw;
    const double2 *px = S.ex + base * S.nx + ix;
    const double2 *py = S.ey + base * S.ny + iy;
    const double2 *pt = S.tt + base * S.np_total + n;
    for (int m = 0; m < S.nw; ++m) {
        double2 a = __ldg(px + (size_t)m * S.nx);
        double2 b = __ldg(py + (size_t)m * S.ny);
        double2 t = __ldg(pt + (size_t)m * S.np_total);
        double qr = a.x * b.x - a.y * b.y;
        double qi = a.x * b.y + a.y * b.x;
        double vr = w * (qr * t.x - qi * t.y);
        double vi = w * (qr * t.y + qi * t.x);
        const double kx = __ldg(S.kx + base + m), ky = __ldg(S.ky + base + m);
        st[0] += vr;
        st[1] -= kx * vi;
        st[2] -= ky * vi;
        if (S.cwm) {
            const double ik = 1.0 / __ldg(S.kn + base + m);
            const double ux = kx * ik, uy = ky * ik;
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
__device__ void facet_state_d(const DevScene &S, int ix, int iy, int n, double st[8])
{
    for (int q = 0; q < 8; ++q) st[q] = 0.0;
    if (S.static_surface || S.nw == 0) return;
    if (S.het_ncx > 0) {
        const double x = (ix + 0.5 - 0.5 * S.nx) * S.dx, y = (iy + 0.5 - 0.5 * S.ny) * S.dx;
        const int tx = min(max((int)floor((x - S.het_x0) / S.het_l), 0), S.het_ncx - 2);
        const int ty = min(max((int)floor((y - S.het_y0) / S.het_l), 0), S.het_ncy - 2);
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const int cx = tx + dx, cy = ty + dy;
                const double wx = fabs(S.het_x0 + cx * S.het_l - x) / S.het_l;
                const double wy = fabs(S.het_y0 + cy * S.het_l - y) / S.het_l;
                const double v = 1.0 - wx - wy + wx * wy;
                if (!(v > 0.0)) continue;
                wave_set_d(S, cy * S.het_ncx + cx, ix, iy, n, sqrt(v), st);
            }
    } else {
        wave_set_d(S, 0, ix, iy, n, 1.0, st);
    }
}

// Intra-facet speckle (Eq. 7 at f_s = 0): Box-Muller on Philox words,
// R, I ~ N(0, 1/2).
__device__ __forceinline__ void speckle_d(uint64_t seed, uint32_t f, uint32_t epoch, double &zr, double &zi)
{
    U32x4 w = philox_stream(seed, kStreamSpeckle, f, epoch);
    double u1 = ((double)w.x + 1.0) * 0x1p-32;
    double u2 = (double)w.y * 0x1p-32;
    double rad = sqrt(-log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    zr = rad * c;
    zi = rad * s;
}

// Speckle under the order-1 autoregressive model of Eq. 10: s_0 = w_0,
// s_e = beta s_(e-1) + sqrt(1 - beta^2) w_e, run from epoch 0.
__device__ void speckle_ar1_d(const DevScene &S, uint32_t f, uint32_t epoch, double &zr, double &zi)
{
    if (S.spk_beta == 0.0) {
        speckle_d(S.speckle_seed, f, epoch, zr, zi);
        return;
    }
    speckle_d(S.speckle_seed, f, 0u, zr, zi);
    for (uint32_t e = 1; e <= epoch; ++e) {
        double wr, wi;
        speckle_d(S.speckle_seed, f, e, wr, wi);
        zr = S.spk_beta * zr + S.spk_q * wr;
        zi = S.spk_beta * zi + S.spk_q * wi;
    }
}

// Kaiser window I0(beta sqrt(1 - (x/4)^2)) / I0(beta) from its power series in
// v = 1 - (x/4)^2 (coefficients prepared on the host), times sinc(x).
__device__ __forceinline__ double kaiser_sinc_d(const DevScene &S, double x, double sin_pf, int j)
{
    double q = 0.25 * x;
    double v = 1.0 - q * q;
    if (v <= 0.0) return 0.0;
    double w = S.i0c[S.n_i0 - 1];
    for (int k = S.n_i0 - 2; k >= 0; --k) w = fma(w, v, S.i0c[k]);
    // sin(pi (j - f)) = -(-1)^j sin(pi f)
    double sn = (j & 1) ? sin_pf : -sin_pf;
    double sc = (x == 0.0) ? 1.0 : sn / (kPi * x);
    return sc * w;
}

template <typename OutT>
__device__ __forceinline__ void global_add(OutT *iq, size_t idx, double re, double im);

template <>
__device__ __forceinline__ void global_add<double>(double *iq, size_t idx, double re, double im)
{
    atomicAdd(iq + 2 * idx, re);
    atomicAdd(iq + 2 * idx + 1, im);
}

template <>
__device__ __forceinline__ void global_add<float>(float *iq, size_t idx, double re, double im)
{
    atomicAdd(iq + 2 * idx, (float)re);
    atomicAdd(iq + 2 * idx + 1, (float)im);
}

__global__ void __launch_bounds__(256) generate_f64_kernel(DevScene S, int n0, int nfirst, double *state)
{
    int64_t nf = (int64_t)S.nx * S.ny;
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int n = nfirst + blockIdx.y;
    if (f >= nf) return;
    int ix = (int)(f % S.nx), iy = (int)(f / S.nx);
    double st[8];
    facet_state_d(S, ix, iy, n, st);
    const int nfl = S.cwm ? 8 : 3;
    double *o = state + (size_t)(n - n0) * nfl * nf;
    for (int q = 0; q < nfl; ++q) o[q * nf + f] = st[q];
}

template <int TAPS, typename OutT>
__global__ void __launch_bounds__(256) accumulate_f64_kernel(DevScene S, int n0, int np, int nfirst, OutT *iq)
{
    __shared__ double2 tile[kMaxCh][kWin];
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

    for (int i = threadIdx.x; i < S.nc * kWin; i += blockDim.x) tile[i / kWin][i % kWin] = make_double2(0.0, 0.0);
    // Window base per channel from the tile centre on the mean surface.
    if (threadIdx.x < S.nc) {
        int c = threadIdx.x;
        const RxState &R = S.rx[(size_t)n * S.nc + c];
        double xc[3] = {(tx0 + 0.5 * kTile - 0.5 * S.nx) * S.dx, (ty0 + 0.5 * kTile - 0.5 * S.ny) * S.dx, 0.0};
        double dt[3] = {xc[0] - P.tx.p[0], xc[1] - P.tx.p[1], xc[2] - P.tx.p[2]};
        double dr[3] = {xc[0] - R.rx.p[0], xc[1] - R.rx.p[1], xc[2] - R.rx.p[2]};
        double rsum = sqrt(dot3(dt, dt)) + sqrt(dot3(dr, dr));
        double pc = R.p_ref + (rsum - P.tx.rref - R.rx.rref) * S.inv_dr;
        kbase[c] = (int)floor(pc) - kWin / 2;
    }
    __syncthreads();

    if (valid) {
        const uint32_t f = (uint32_t)iy * (uint32_t)S.nx + (uint32_t)ix;
        double st[8];
        facet_state_d(S, ix, iy, n, st);
        // rest position, moved by the horizontal displacement (CWM) and lifted to eta
        const double xb = (ix + 0.5 - 0.5 * S.nx) * S.dx, yb = (iy + 0.5 - 0.5 * S.ny) * S.dx;
        const double x[3] = {xb + st[3], yb + st[4], st[0]};
        const double xx = dot3(x, x);
        // normal: cross product of the displaced surface's tangents
        // (1 + dDx/dx, dDx/dy, eta_x) and (dDx/dy, 1 + dDy/dy, eta_y)
        const double nv[3] = {st[6] * st[2] - st[1] * (1.0 + st[7]), st[1] * st[6] - (1.0 + st[5]) * st[2],
                              (1.0 + st[5]) * (1.0 + st[7]) - st[6] * st[6]};
        const double nlen = sqrt(dot3(nv, nv));
        const double area = S.area * fmax(nv[2], 0.0);

        // transmit leg: range offset from the scene-centre range in the stable
        // form (|x|^2 - 2 P.x) / (r + R), unit vector, pattern gain
        double dtv[3] = {x[0] - P.tx.p[0], x[1] - P.tx.p[1], x[2] - P.tx.p[2]};
        double rt = sqrt(dot3(dtv, dtv));
        double delt = (xx - 2.0 * dot3(P.tx.p, x)) / (rt + P.tx.rref);
        double ut[3] = {dtv[0] / rt, dtv[1] / rt, dtv[2] / rt};
        const double2 gt = antenna_gain_d(S, 0, P.tx, S.tx_laz, S.tx_lel, ut);

        double base = S.sigma0_base, cu = S.cur_u, cv = S.cur_v;
        if (S.cell_sigma0 || S.cell_uv) {
            int cx = (int)floor((xb + 0.5 * S.nx * S.dx) / S.cell);
            int cy = (int)floor((yb + 0.5 * S.ny * S.dx) / S.cell);
            cx = min(max(cx, 0), S.ncx - 1);
            cy = min(max(cy, 0), S.ncy - 1);
            int ci = cy * S.ncx + cx;
            if (S.cell_sigma0) base = S.cell_sigma0[ci];
            if (S.cell_uv) {
                cu = S.cell_uv[2 * ci];
                cv = S.cell_uv[2 * ci + 1];
            }
        }
        uint32_t epoch = S.epoch_pulses > 0 ? (uint32_t)(n / S.epoch_pulses) : 0u;
        double zr, zi;
        speckle_ar1_d(S, f, epoch, zr, zi);
        const double fd_phase = 2.0 * kPi * S.fd_hz * P.t;

        for (int c = 0; c < S.nc; ++c) {
            const RxState &R = S.rx[(size_t)n * S.nc + c];
            double drv[3] = {x[0] - R.rx.p[0], x[1] - R.rx.p[1], x[2] - R.rx.p[2]};
            double rr = sqrt(dot3(drv, drv));
            double delr = (xx - 2.0 * dot3(R.rx.p, x)) / (rr + R.rx.rref);
            double ur[3] = {drv[0] / rr, drv[1] / rr, drv[2] / rr};
            const double2 gr = antenna_gain_d(S, 1 + c, R.rx, S.rx_laz[c], S.rx_lel[c], ur);

            double sig = base;
            if (!S.static_surface) {
                double q[3] = {-(ut[0] + ur[0]), -(ut[1] + ur[1]), -(ut[2] + ur[2])};
                double qh = sqrt(q[0] * q[0] + q[1] * q[1]);
                double cphi = qh > 0.0 ? (S.wcos * q[0] + S.wsin * q[1]) / qh : 0.0;
                double nq = dot3(nv, q);
                double tilt = fmax(nq, 0.0) / (nlen * q[2]);
                sig = base * (1.0 + S.wind_mod * cphi) * tilt;
            }
            double amp = sqrt(sig * area) * (P.tx.rref / rt) * (R.rx.rref / rr);
            double vc = cu * (ut[0] + ur[0]) + cv * (ut[1] + ur[1]);
            double phase = R.psi - S.k0 * (delt + delr + vc * P.t) + fd_phase;
            double sp, cp;
            sincos(phase, &sp, &cp);
            // field weight G_t G_r (complex for u-v grids) times the speckle
            const double gre = gt.x * gr.x - gt.y * gr.y, gim = gt.x * gr.y + gt.y * gr.x;
            double ar = amp * (zr * gre - zi * gim), ai = amp * (zr * gim + zi * gre);
            double vr = ar * cp - ai * sp;
            double vi = ar * sp + ai * cp;
            double p = R.p_ref + (delt + delr) * S.inv_dr;
            double fk = floor(p);
            if (TAPS == 1) {
                if (fk >= 0.0 && fk < (double)nr) {
                    int k = (int)fk;
                    int w = k - kbase[c];
                    if (w >= 0 && w < kWin) {
                        atomicAdd(&tile[c][w].x, vr);
                        atomicAdd(&tile[c][w].y, vi);
                    } else {
                        global_add<OutT>(iq, ((size_t)c * np + (n - n0)) * nr + k, vr, vi);
                    }
                }
            } else {
                if (fk < -8.0 || fk > (double)nr + 8.0) continue;
                int k0 = (int)fk;
                double fr = p - fk;
                double spf = sinpi(fr);
#pragma unroll
                for (int j = -3; j <= 4; ++j) {
                    int k = k0 + j;
                    if (k < 0 || k >= nr) continue;
                    double h = kaiser_sinc_d(S, (double)j - fr, spf, j);
                    int w = k - kbase[c];
                    if (w >= 0 && w < kWin) {
                        atomicAdd(&tile[c][w].x, h * vr);
                        atomicAdd(&tile[c][w].y, h * vi);
                    } else {
                        global_add<OutT>(iq, ((size_t)c * np + (n - n0)) * nr + k, h * vr, h * vi);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < S.nc * kWin; i += blockDim.x) {
        int c = i / kWin, w = i % kWin;
        int k = kbase[c] + w;
        double2 v = tile[c][w];
        if (k >= 0 && k < nr && (v.x != 0.0 || v.y != 0.0))
            global_add<OutT>(iq, ((size_t)c * np + (n - n0)) * nr + k, v.x, v.y);
    }
}

}  // namespace

cudaError_t launch_generate_f64(const DevScene &S, cudaStream_t st, int n0, int np, double *state)
{
    int64_t nf = (int64_t)S.nx * S.ny;
    for (int p0 = 0; p0 < np; p0 += 65535) {
        int cnt = min(65535, np - p0);
        dim3 grid((unsigned)((nf + 255) / 256), (unsigned)cnt);
        generate_f64_kernel<<<grid, 256, 0, st>>>(S, n0, n0 + p0, state);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_accumulate_f64(const DevScene &S, cudaStream_t st, int n0, int np, void *iq, harm_dtype dtype)
{
    int tiles = ((S.nx + kTile - 1) / kTile) * ((S.ny + kTile - 1) / kTile);
    for (int p0 = 0; p0 < np; p0 += 65535) {
        int cnt = min(65535, np - p0);
        dim3 grid((unsigned)tiles, (unsigned)cnt);
        int nfirst = n0 + p0;
        if (dtype == HARM_C128) {
            if (S.taps == 1)
                accumulate_f64_kernel<1, double><<<grid, 256, 0, st>>>(S, n0, np, nfirst, (double *)iq);
            else
                accumulate_f64_kernel<8, double><<<grid, 256, 0, st>>>(S, n0, np, nfirst, (double *)iq);
        } else {
            if (S.taps == 1)
                accumulate_f64_kernel<1, float><<<grid, 256, 0, st>>>(S, n0, np, nfirst, (float *)iq);
            else
                accumulate_f64_kernel<8, float><<<grid, 256, 0, st>>>(S, n0, np, nfirst, (float *)iq);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace harm
