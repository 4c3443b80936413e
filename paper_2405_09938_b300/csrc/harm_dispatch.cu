// Launch dispatch by precision, and the host-side tables of the mixed path:
// FP32 separable wave phasors, Taylor-in-time tables per pulse batch, and the
// Kaiser-sinc tap polynomials.
#include <algorithm>
#include <cmath>
#include <vector>

#include "harm_internal.cuh"
#include "harm_kernels.cuh"

namespace harm {

int mixed_batch_pulses();

namespace {

// One wave component as the table kernel reads it.
struct WaveDev {
    double kx, ky, om, amp, ph;
};

template <typename T2>
__device__ __forceinline__ T2 make_pair(double a, double b);
template <>
__device__ __forceinline__ float2 make_pair<float2>(double a, double b)
{
    return make_float2((float)a, (float)b);
}
template <>
__device__ __forceinline__ double2 make_pair<double2>(double a, double b)
{
    return make_double2(a, b);
}

// Separable phasor tables of the linear surface (Sec. III: each component is a
// plane wave, so its phase k.x - omega t + phi splits into an x, a y and a time
// factor), evaluated in FP64 and stored as T2: ex[qm][ix] = e^{i kx x},
// ey[qm][iy] = a e^{i (ky y + phi)} and, when tt is given, tt[qm][n] =
// e^{-i omega t_s(n)}; qm runs over every component of every wave set.
template <typename T2>
__global__ void phasor_tables_kernel(const WaveDev *waves, int nsw, int nx, int ny, int np, double dx,
                                     const PulseState *ps, T2 *ex, T2 *ey, T2 *tt)
{
    const int per = nx + ny + (tt ? np : 0);
    const size_t total = (size_t)nsw * per;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int qm = (int)(i / per), j = (int)(i % per);
        const WaveDev w = waves[qm];
        double sn, cs;
        if (j < nx) {
            sincos(w.kx * ((j + 0.5 - 0.5 * nx) * dx), &sn, &cs);
            ex[(size_t)qm * nx + j] = make_pair<T2>(cs, sn);
        } else if (j < nx + ny) {
            const int iy = j - nx;
            sincos(w.ky * ((iy + 0.5 - 0.5 * ny) * dx) + w.ph, &sn, &cs);
            ey[(size_t)qm * ny + iy] = make_pair<T2>(w.amp * cs, w.amp * sn);
        } else {
            const int n = j - nx - ny;
            sincos(-w.om * ps[n].ts, &sn, &cs);
            tt[(size_t)qm * np + n] = make_pair<T2>(cs, sn);
        }
    }
}

template <typename T>
cudaError_t dev_alloc(harm_scene *s, size_t count, T **out)
{
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    s->allocs.push_back(p);
    *out = (T *)p;
    return cudaSuccess;
}

template <typename T>
cudaError_t upload_raw(harm_scene *s, const std::vector<T> &h, const T **out)
{
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, h.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    s->allocs.push_back(p);
    e = cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s->stream);
    *out = (const T *)p;
    return e;
}

// Kaiser-windowed sinc h(x) for the 8-tap kernel (half-width 4), with the window
// from the scene's power-series coefficients.
double kaiser_sinc_host(const DevScene &S, double x)
{
    double q = 0.25 * x;
    double v = 1.0 - q * q;
    if (v <= 0.0) return 0.0;
    double w = 0.0;
    for (int k = S.n_i0 - 1; k >= 0; --k) w = w * v + S.i0c[k];
    double sc = (x == 0.0) ? 1.0 : std::sin(kPi * x) / (kPi * x);
    return sc * w;
}

// Tap j (bin k0 - 3 + j) as a polynomial of degree kTapDeg in t = 2 f - 1,
// f in [0, 1) the fractional bin: Chebyshev interpolation at the Chebyshev
// nodes, converted to monomial coefficients.
void fit_taps(const DevScene &S, float out[8][kTapDeg + 1])
{
    const int N = kTapDeg + 1;
    for (int j = 0; j < 8; ++j) {
        double fv[N], cheb[N];
        for (int i = 0; i < N; ++i) {
            double t = std::cos(kPi * (i + 0.5) / N);
            double f = 0.5 * (t + 1.0);
            fv[i] = kaiser_sinc_host(S, (double)(j - 3) - f);
        }
        for (int k = 0; k < N; ++k) {
            double acc = 0.0;
            for (int i = 0; i < N; ++i) acc += fv[i] * std::cos(kPi * k * (i + 0.5) / N);
            cheb[k] = acc * (k == 0 ? 1.0 : 2.0) / N;
        }
        // monomial coefficients of sum_k cheb[k] T_k(t)
        double mono[N] = {0};
        double tkm1[N] = {0}, tk[N] = {0}, tkp1[N];
        tkm1[0] = 1.0;  // T_0
        tk[1] = 1.0;    // T_1
        for (int d = 0; d < N; ++d) mono[d] += cheb[0] * tkm1[d];
        if (N > 1)
            for (int d = 0; d < N; ++d) mono[d] += cheb[1] * tk[d];
        for (int k = 2; k < N; ++k) {
            for (int d = 0; d < N; ++d) tkp1[d] = -tkm1[d] + (d > 0 ? 2.0 * tk[d - 1] : 0.0);
            for (int d = 0; d < N; ++d) mono[d] += cheb[k] * tkp1[d];
            for (int d = 0; d < N; ++d) {
                tkm1[d] = tk[d];
                tk[d] = tkp1[d];
            }
        }
        for (int d = 0; d < N; ++d) out[j][d] = (float)mono[d];
    }
}

// sinc^2(x) on |x| <= 1 as a polynomial of degree kSincDeg in t = 2 x^2 - 1
// (Chebyshev interpolation in t, converted to monomials).
void fit_sinc2(float out[kSincDeg + 1])
{
    const int N = kSincDeg + 1;
    double fv[N], cheb[N];
    for (int i = 0; i < N; ++i) {
        double t = std::cos(kPi * (i + 0.5) / N);
        double x = std::sqrt(0.5 * (t + 1.0));
        double s = (x == 0.0) ? 1.0 : std::sin(kPi * x) / (kPi * x);
        fv[i] = s * s;
    }
    for (int k = 0; k < N; ++k) {
        double acc = 0.0;
        for (int i = 0; i < N; ++i) acc += fv[i] * std::cos(kPi * k * (i + 0.5) / N);
        cheb[k] = acc * (k == 0 ? 1.0 : 2.0) / N;
    }
    double mono[N] = {0}, tkm1[N] = {0}, tk[N] = {0}, tkp1[N];
    tkm1[0] = 1.0;
    tk[1] = 1.0;
    for (int d = 0; d < N; ++d) mono[d] += cheb[0] * tkm1[d] + cheb[1] * tk[d];
    for (int k = 2; k < N; ++k) {
        for (int d = 0; d < N; ++d) tkp1[d] = -tkm1[d] + (d > 0 ? 2.0 * tk[d - 1] : 0.0);
        for (int d = 0; d < N; ++d) mono[d] += cheb[k] * tkp1[d];
        for (int d = 0; d < N; ++d) {
            tkm1[d] = tk[d];
            tk[d] = tkp1[d];
        }
    }
    for (int d = 0; d < N; ++d) out[d] = (float)mono[d];
}

}  // namespace

template <typename T2>
cudaError_t phasor_tables(harm_scene *s, const WaveSets &W, const PulseState *ps_dev, const T2 **ex,
                          const T2 **ey, const T2 **tt)
{
    const harm_scene_desc &d = s->desc;
    const int nx = d.nx, ny = d.ny, np = d.n_pulses;
    const int nsw = W.n_sets * std::max(W.nw, 1);
    std::vector<WaveDev> h((size_t)nsw, WaveDev{0.0, 0.0, 0.0, 0.0, 0.0});
    for (int q = 0; q < W.n_sets; ++q)
        for (int m = 0; m < W.nw; ++m) {
            const Wave &w = W.at(q, m);
            h[(size_t)q * W.nw + m] = WaveDev{w.kx, w.ky, w.om, w.amp, w.ph};
        }
    const WaveDev *wd = nullptr;
    T2 *pex = nullptr, *pey = nullptr, *ptt = nullptr;
    cudaError_t e = upload_raw(s, h, &wd);
    if (e == cudaSuccess) e = dev_alloc(s, (size_t)nsw * nx, &pex);
    if (e == cudaSuccess) e = dev_alloc(s, (size_t)nsw * ny, &pey);
    if (e == cudaSuccess && tt) e = dev_alloc(s, (size_t)nsw * np, &ptt);
    if (e != cudaSuccess) return e;
    const size_t total = (size_t)nsw * (nx + ny + (tt ? np : 0));
    const int threads = 256;
    const int blocks = (int)std::min<size_t>((total + threads - 1) / threads, 148 * 16);
    phasor_tables_kernel<T2><<<blocks, threads, 0, s->stream>>>(wd, nsw, nx, ny, np, d.facet_m, ps_dev, pex, pey,
                                                                ptt);
    e = cudaGetLastError();
    *ex = pex;
    *ey = pey;
    if (tt) *tt = ptt;
    return e;
}

template cudaError_t phasor_tables<double2>(harm_scene *, const WaveSets &, const PulseState *, const double2 **,
                                            const double2 **, const double2 **);
template cudaError_t phasor_tables<float2>(harm_scene *, const WaveSets &, const PulseState *, const float2 **,
                                           const float2 **, const float2 **);

harm_status build_mixed_tables(harm_scene *s, const std::vector<PulseState> &ps, const WaveSets &W)
{
    const harm_scene_desc &d = s->desc;
    MixedTables &M = s->mixed;
    const int np = d.n_pulses;
    const int nw = W.nw, nsets = W.n_sets;
    const int nf = d.cwm ? 8 : 3;
    M.nb = mixed_batch_pulses();
    M.n_batches = (np + M.nb - 1) / M.nb;
    M.nf = nf;
    const size_t nsw = (size_t)nsets * std::max(nw, 1);
    // Taylor tables. With the component's space phasor q (e^{i kx x} a e^{i (ky y +
    // phi)}) and Q = q e^{-i omega t_c} at the batch centre t_c, state field f at
    // time offset tau is Re(c_f Q e^{-i omega tau}) summed over components, and
    // e^{-i omega tau} = sum_o (-i)^o r_o tau^o with r_o = omega^o / o!. The field
    // factor c_f is real (eta: 1; with the Choppy Wave Model dD_x/dx: -kx^2/k,
    // dD_x/dy: -kx ky/k, dD_y/dy: -ky^2/k) or imaginary, c_f = i g (eta_x: kx,
    // eta_y: ky; D_x: kx/k, D_y: ky/k). So each Taylor coefficient is a real number
    // times Q_r or Q_i: Re(Q (-i)^o) = Q_r, Q_i, -Q_r, -Q_i, Q_r, Q_i and
    // Re(i Q (-i)^o) = -Q_i, Q_r, Q_i, -Q_r, -Q_i, Q_r for o = 0..5. Tables:
    // tc[b][set][m] = e^{-i omega t_c(b)}; cr[set][m][f][o] = the signed real factor
    // (c or g) r_o (the kernels pair orders 2p, 2p + 1 with (Q_r, Q_i) for real c_f
    // and with (Q_i, Q_r) for imaginary c_f).
    // time tables of the windows: offsets tau from the window centre and the
    // centre phasors, for the default window and for the half-length one
    auto window_tables = [&](int nb, std::vector<float> &tau, std::vector<float2> &tc) {
        const int nbat = (np + nb - 1) / nb;
        tau.assign(np, 0.0f);
        tc.assign((size_t)nbat * nsw, make_float2(0.0f, 0.0f));
        for (int b = 0; b < nbat; ++b) {
            int first = b * nb, last = std::min(np, first + nb) - 1;
            double tcb = 0.5 * (ps[first].ts + ps[last].ts);
            for (int n = first; n <= last; ++n) tau[n] = (float)(ps[n].ts - tcb);
            for (int q = 0; q < nsets; ++q)
                for (int m = 0; m < nw; ++m) {
                    const double a = -W.at(q, m).om * tcb;
                    tc[(size_t)b * nsw + (size_t)q * nw + m] = make_float2((float)std::cos(a), (float)std::sin(a));
                }
        }
    };
    std::vector<float> tau, tau_alt;
    std::vector<float2> tc, tc_alt;
    window_tables(M.nb, tau, tc);
    M.alt_nb = M.nb / 2;
    M.alt_n_batches = (np + M.alt_nb - 1) / M.alt_nb;
    window_tables(M.alt_nb, tau_alt, tc_alt);
    std::vector<float> cr(nsw * nf * kOrders);
    static const double kSignReal[kOrders] = {1.0, 1.0, -1.0, -1.0, 1.0, 1.0};
    static const double kSignImag[kOrders] = {-1.0, 1.0, 1.0, -1.0, -1.0, 1.0};
    for (int q = 0; q < nsets; ++q)
        for (int m = 0; m < nw; ++m) {
            const Wave &w = W.at(q, m);
            const double k = std::sqrt(w.kx * w.kx + w.ky * w.ky);
            // factor c (real c_f) or g (c_f = i g) of each field
            const double g[8] = {1.0, w.kx, w.ky, w.kx / k, w.ky / k, -w.kx * w.kx / k, -w.kx * w.ky / k,
                                 -w.ky * w.ky / k};
            double r = 1.0;  // omega^o / o!
            for (int o = 0; o < kOrders; ++o) {
                if (o > 0) r *= w.om / o;
                for (int f = 0; f < nf; ++f) {
                    const bool real = f == 0 || f >= 5;
                    const double sg = real ? kSignReal[o] : kSignImag[o];
                    cr[(((size_t)q * nw + m) * nf + f) * kOrders + o] = (float)(sg * g[f] * r);
                }
            }
        }
    fit_taps(s->dev, M.tap);
    fit_sinc2(M.sinc2);
    if (phasor_tables<float2>(s, W, nullptr, &M.ex, &M.ey, nullptr) != cudaSuccess ||
        upload_raw(s, tc, &M.tc) != cudaSuccess || upload_raw(s, cr, &M.cr) != cudaSuccess ||
        upload_raw(s, tau, &M.tau) != cudaSuccess || upload_raw(s, tc_alt, &M.alt_tc) != cudaSuccess ||
        upload_raw(s, tau_alt, &M.alt_tau) != cudaSuccess)
        return HARM_E_CUDA;
    return HARM_OK;
}

cudaError_t launch_generate(harm_scene *s, int n0, int np, void *state)
{
    if (s->desc.precision != HARM_PREC_MIXED)
        return launch_generate_plain(s->dev, s->desc.precision == HARM_PREC_FP64, s->stream, n0, np, state);
    return launch_generate_mixed(s->dev, s->mixed, s->stream, n0, np, (float *)state);
}

cudaError_t launch_accumulate(harm_scene *s, int n0, int np, void *iq, harm_dtype dtype)
{
    return launch_accumulate_on(s, s->stream, n0, np, iq, dtype);
}

cudaError_t launch_accumulate_on(harm_scene *s, cudaStream_t st, int n0, int np, void *iq, harm_dtype dtype)
{
    if (s->desc.precision != HARM_PREC_MIXED)
        return launch_accumulate_plain(s->dev, s->desc.precision == HARM_PREC_FP64, st, n0, np, iq, dtype);
    return launch_accumulate_mixed(s->dev, s->mixed, st, n0, np, iq, dtype);
}

cudaError_t launch_adjoint(harm_scene *s, int n0, int np, const void *resid, harm_dtype dtype, double *g_sigma,
                           double *g_uv)
{
    if (s->desc.precision != HARM_PREC_MIXED) return cudaErrorNotSupported;
    return launch_adjoint_mixed(s->dev, s->mixed, s->stream, n0, np, resid, dtype, g_sigma, g_uv);
}

}  // namespace harm
