// Host core of the echo library: descriptor validation, FP64 precompute of the
// wave table and per-pulse platform state, device tables, and the C ABI.
//
// Everything computed here is per scene or per pulse (O(n_pulses x n_channels +
// n_waves x (nx + ny + n_pulses))); all per-facet work runs in the kernels.
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>  // CUtensorMap and its encoder's types (the encoder is fetched through the runtime)

#include "harm.h"
#include "harm_internal.cuh"
#include "harm_kernels.cuh"
#include "philox.cuh"

namespace {

thread_local std::string g_last_error;

harm_status fail(harm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

harm_status cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();  // clear a sticky launch error where possible
    return fail(e == cudaErrorMemoryAllocation ? HARM_E_OOM : HARM_E_CUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

#define HARM_CUDA(call, what)                      \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool finite3(const double v[3]) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

double norm3(const double v[3]) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

void ant_pos(const harm_antenna &a, double t, double p[3])
{
    for (int i = 0; i < 3; ++i) p[i] = a.pos0[i] + a.vel[i] * t;
}

// Frame of an antenna steered to the scene centre: boresight toward the origin,
// azimuth axis = velocity with its boresight part removed, elevation = b x a.
void steer(const harm_antenna &ant, const double p[3], harm::AntState &s)
{
    double r = norm3(p);
    double b[3] = {-p[0] / r, -p[1] / r, -p[2] / r};
    double vb = ant.vel[0] * b[0] + ant.vel[1] * b[1] + ant.vel[2] * b[2];
    double t[3] = {ant.vel[0] - vb * b[0], ant.vel[1] - vb * b[1], ant.vel[2] - vb * b[2]};
    double tn = norm3(t);
    for (int i = 0; i < 3; ++i) {
        s.p[i] = p[i];
        s.a[i] = t[i] / tn;
    }
    s.e[0] = b[1] * s.a[2] - b[2] * s.a[1];
    s.e[1] = b[2] * s.a[0] - b[0] * s.a[2];
    s.e[2] = b[0] * s.a[1] - b[1] * s.a[0];
    s.rref = r;
}

// -K0 R reduced to (-pi, pi]: the phase in cycles is -f0 R / c; its fractional
// part is taken in extended precision.
double reduced_phase(double f0, double r)
{
    long double cyc = -(long double)f0 * (long double)r / (long double)harm::kC;
    long double fr = cyc - std::floor(cyc + 0.5L);
    return (double)(fr * 2.0L * (long double)harm::kPi);
}

struct PulseGeo {
    harm::PulseState ps;
    std::vector<harm::RxState> rx;
};

// Pulse n: transmit at t_n; the surface is sampled at the bounce time
// t_s = t_n + R_t / c; the receive time solves t_r = t_s + R_r(t_r) / c by three
// fixed-point steps started at t_s.
void pulse_geometry(const harm_scene_desc &d, const std::vector<harm_antenna> &rx, int n,
                    harm::PulseState &ps, harm::RxState *rs)
{
    ps.t = (double)n / d.prf_hz;
    double p[3];
    ant_pos(d.tx, ps.t, p);
    steer(d.tx, p, ps.tx);
    ps.ts = ps.t + ps.tx.rref / harm::kC;
    for (int c = 0; c < d.n_channels; ++c) {
        double tr = ps.ts;
        for (int it = 0; it < 3; ++it) {
            ant_pos(rx[c], tr, p);
            tr = ps.ts + norm3(p) / harm::kC;
        }
        ant_pos(rx[c], tr, p);
        steer(rx[c], p, rs[c].rx);
    }
}

// JONSWAP spectrum with fetch-limited peak frequency and Phillips constant.
double jonswap(double w, double u10, double fetch, double gamma)
{
    const double g = 9.80665;
    double xt = g * fetch / (u10 * u10);
    double wp = 22.0 * (g / u10) / std::cbrt(xt);
    double alpha = 0.076 * std::pow(xt, -0.22);
    double sig = w > wp ? 0.09 : 0.07;
    double dw = (w - wp) / (sig * wp);
    double shape = std::exp(-0.5 * dw * dw);
    double q = wp / w;
    return alpha * g * g / (w * w * w * w * w) * std::exp(-1.25 * q * q * q * q) * std::pow(gamma, shape);
}

double peak_omega(double u10, double fetch)
{
    const double g = 9.80665;
    return 22.0 * (g / u10) / std::cbrt(g * fetch / (u10 * u10));
}

// Linear-wave grid: log-spaced frequency bins on [0.7, 2.5] x peak (geometric
// centres), equally spaced directions about the wind, cos^2s spreading,
// amplitude from the spectral energy of each cell, Philox phase (counter word 2
// = word2: 0 for a homogeneous sea state, 1 + corner for a heterogeneous one).
std::vector<harm::Wave> wave_grid(const harm_scene_desc &d, double u10, double wind_dir, uint32_t word2)
{
    std::vector<harm::Wave> w;
    if (d.n_omega <= 0 || d.n_theta <= 0 || d.static_surface) return w;
    const double g = 9.80665;
    double wp = peak_omega(u10, d.fetch_m);
    double lo = 0.7 * wp, ratio = 2.5 / 0.7;
    double dth = 2.0 * harm::kPi / d.n_theta;
    double s = d.spread_s;
    double norm = std::exp2(2.0 * s - 1.0) * std::exp(2.0 * std::lgamma(s + 1.0) - std::lgamma(2.0 * s + 1.0)) / harm::kPi;
    for (int i = 0; i < d.n_omega; ++i) {
        double e0 = lo * std::pow(ratio, (double)i / d.n_omega);
        double e1 = lo * std::pow(ratio, (double)(i + 1) / d.n_omega);
        double om = std::sqrt(e0 * e1);
        double sw = jonswap(om, u10, d.fetch_m, d.gamma);
        double k = om * om / g;
        for (int j = 0; j < d.n_theta; ++j) {
            int m = i * d.n_theta + j;
            double rel = -harm::kPi + (j + 0.5) * dth;
            double th = wind_dir + rel;
            double spread = norm * std::pow(std::cos(0.5 * rel), 2.0 * s);
            harm::U32x4 r = harm::philox_stream(d.wave_seed, harm::kStreamWave, (uint32_t)m, word2);
            harm::Wave v;
            v.kx = k * std::cos(th);
            v.ky = k * std::sin(th);
            v.om = om;
            v.amp = std::sqrt(2.0 * sw * (e1 - e0) * spread * dth);
            v.ph = 2.0 * harm::kPi * ((double)r.x * 0x1p-32);
            w.push_back(v);
        }
    }
    return w;
}

// Every wave set of the scene: the scene's spectrum, or one per corner of a
// heterogeneous sea state with the corner's wind speed and direction (Eq. 1).
harm::WaveSets wave_sets(const harm_scene *s)
{
    const harm_scene_desc &d = s->desc;
    harm::WaveSets W;
    if (d.hetero_ncx > 0) {
        W.n_sets = d.hetero_ncx * d.hetero_ncy;
        for (int i = 0; i < W.n_sets; ++i) {
            std::vector<harm::Wave> w = wave_grid(d, s->het_u10[i], s->het_dir[i], 1u + (uint32_t)i);
            W.nw = (int)w.size();
            W.w.insert(W.w.end(), w.begin(), w.end());
        }
    } else {
        W.w = wave_grid(d, d.u10, d.wind_dir_rad, 0u);
        W.nw = (int)W.w.size();
    }
    return W;
}

// Size of a version-1 descriptor: everything before the version-2 fields.
constexpr size_t kDescV1Size = offsetof(harm_scene_desc, speckle_tau_s);

// Copy a descriptor of either version into *out (version-2 fields zero for a
// version-1 descriptor).
harm_status normalize(const harm_scene_desc *d, harm_scene_desc *out)
{
    if (!d) return fail(HARM_E_INVALID, "desc is NULL");
    std::memset(out, 0, sizeof(*out));
    if (d->abi_version == 1u) {
        if (d->struct_size != kDescV1Size)
            return fail(HARM_E_INVALID, "struct_size %u, a version-1 descriptor has %zu", d->struct_size, kDescV1Size);
        std::memcpy(out, d, kDescV1Size);
    } else if (d->abi_version == HARM_ABI_VERSION) {
        if (d->struct_size != sizeof(harm_scene_desc))
            return fail(HARM_E_INVALID, "struct_size %u, library expects %zu", d->struct_size, sizeof(harm_scene_desc));
        std::memcpy(out, d, sizeof(*out));
    } else {
        return fail(HARM_E_INVALID, "abi_version %u, library is %u (accepts 1 and %u)", d->abi_version,
                    HARM_ABI_VERSION, HARM_ABI_VERSION);
    }
    out->abi_version = HARM_ABI_VERSION;
    out->struct_size = sizeof(harm_scene_desc);
    return HARM_OK;
}

// Validate a normalized descriptor.
harm_status validate(const harm_scene_desc *d)
{
    if (!(d->f0_hz > 0 && std::isfinite(d->f0_hz)) || !(d->fs_hz > 0 && std::isfinite(d->fs_hz)) ||
        !(d->prf_hz > 0 && std::isfinite(d->prf_hz)))
        return fail(HARM_E_INVALID, "f0, fs and prf must be positive and finite");
    if (d->n_pulses < 1 || d->n_pulses > (1 << 24)) return fail(HARM_E_INVALID, "n_pulses out of range");
    if (d->n_range < 1 || d->n_range > (1 << 24)) return fail(HARM_E_INVALID, "n_range out of range");
    if (d->n_channels < 1 || d->n_channels > HARM_MAX_CHANNELS)
        return fail(HARM_E_INVALID, "n_channels must be 1..%d", HARM_MAX_CHANNELS);
    if (!d->rx) return fail(HARM_E_INVALID, "rx is NULL");
    if (d->nx < 1 || d->ny < 1) return fail(HARM_E_INVALID, "facet grid must be at least 1 x 1");
    if ((int64_t)d->nx * (int64_t)d->ny > 0xFFFFFFFFll)
        return fail(HARM_E_INVALID, "more than 2^32 - 1 facets");
    if (!(d->facet_m > 0 && std::isfinite(d->facet_m))) return fail(HARM_E_INVALID, "facet_m must be positive");
    if (d->n_omega < 0 || d->n_theta < 0 || (d->n_omega == 0) != (d->n_theta == 0))
        return fail(HARM_E_INVALID, "n_omega and n_theta must both be 0 or both positive");
    if ((int64_t)d->n_omega * d->n_theta > 4096) return fail(HARM_E_INVALID, "more than 4096 wave components");
    if (d->n_omega > 0 && !d->static_surface) {
        if (!(d->u10 > 0) || !(d->fetch_m > 0) || !(d->gamma >= 1.0) || !(d->spread_s > 0) ||
            !std::isfinite(d->wind_dir_rad))
            return fail(HARM_E_INVALID, "sea-state parameters out of range");
    }
    if (!std::isfinite(d->wind_dir_rad) || !std::isfinite(d->current_u) || !std::isfinite(d->current_v))
        return fail(HARM_E_INVALID, "wind direction and current must be finite");
    if (!(d->sigma0_base >= 0 && std::isfinite(d->sigma0_base)) || !std::isfinite(d->wind_mod))
        return fail(HARM_E_INVALID, "sigma0_base / wind_mod out of range");
    if (d->epoch_pulses < 0) return fail(HARM_E_INVALID, "epoch_pulses must be >= 0");
    if (d->taps != 1 && d->taps != 8) return fail(HARM_E_UNSUPPORTED, "taps must be 1 or 8");
    if (!(d->kaiser_beta >= 0 && d->kaiser_beta <= 20)) return fail(HARM_E_INVALID, "kaiser_beta must be in [0, 20]");
    if (d->precision != HARM_PREC_FP64 && d->precision != HARM_PREC_MIXED && d->precision != HARM_PREC_FP32)
        return fail(HARM_E_INVALID, "unknown precision %d", d->precision);
    const harm_antenna *ants[1 + HARM_MAX_CHANNELS];
    ants[0] = &d->tx;
    for (int c = 0; c < d->n_channels; ++c) ants[1 + c] = &d->rx[c];
    for (int i = 0; i <= d->n_channels; ++i) {
        const harm_antenna &a = *ants[i];
        if (!finite3(a.pos0) || !finite3(a.vel)) return fail(HARM_E_INVALID, "antenna %d: non-finite state", i);
        if (!(a.len_az > 0) || !(a.len_el > 0)) return fail(HARM_E_INVALID, "antenna %d: lengths must be positive", i);
        if (!(a.pos0[2] > 0)) return fail(HARM_E_INVALID, "antenna %d must be above the surface", i);
        double v = norm3(a.vel);
        double p = norm3(a.pos0);
        double cross[3] = {a.pos0[1] * a.vel[2] - a.pos0[2] * a.vel[1], a.pos0[2] * a.vel[0] - a.pos0[0] * a.vel[2],
                           a.pos0[0] * a.vel[1] - a.pos0[1] * a.vel[0]};
        if (!(v > 0) || norm3(cross) < 1e-9 * v * p)
            return fail(HARM_E_INVALID, "antenna %d: velocity must be nonzero and not along the line of sight", i);
    }
    // version-2 variants
    if (!(d->speckle_tau_s >= 0 && std::isfinite(d->speckle_tau_s)))
        return fail(HARM_E_INVALID, "speckle_tau_s must be finite and >= 0");
    if (!std::isfinite(d->speckle_doppler_hz)) return fail(HARM_E_INVALID, "speckle_doppler_hz must be finite");
    if (d->cwm != 0 && d->cwm != 1) return fail(HARM_E_INVALID, "cwm must be 0 or 1");
    if (d->hetero_ncx != 0 || d->hetero_ncy != 0) {
        if (d->hetero_ncx < 2 || d->hetero_ncy < 2 || (int64_t)d->hetero_ncx * d->hetero_ncy > 1024)
            return fail(HARM_E_INVALID, "hetero corner grid %d x %d: need 2..1024 corners, at least 2 per axis",
                        d->hetero_ncx, d->hetero_ncy);
        if (!(d->hetero_tile_m > 0 && std::isfinite(d->hetero_tile_m)))
            return fail(HARM_E_INVALID, "hetero_tile_m must be positive");
        if (!d->hetero_u10 || !d->hetero_wind_dir_rad)
            return fail(HARM_E_INVALID, "hetero_u10 and hetero_wind_dir_rad must not be NULL");
        const double lx = d->nx * d->facet_m, ly = d->ny * d->facet_m;
        if ((d->hetero_ncx - 1) * d->hetero_tile_m < lx * (1.0 - 1e-12) ||
            (d->hetero_ncy - 1) * d->hetero_tile_m < ly * (1.0 - 1e-12))
            return fail(HARM_E_INVALID, "hetero corner grid (%d x %d corners of %g m) does not cover the patch",
                        d->hetero_ncx, d->hetero_ncy, d->hetero_tile_m);
        for (int i = 0; i < d->hetero_ncx * d->hetero_ncy; ++i)
            if (!(d->hetero_u10[i] > 0 && std::isfinite(d->hetero_u10[i])) || !std::isfinite(d->hetero_wind_dir_rad[i]))
                return fail(HARM_E_INVALID, "hetero corner %d: wind speed must be positive, direction finite", i);
    }
    return HARM_OK;
}

}  // namespace

namespace {

template <typename T>
harm_status upload(harm_scene *s, const std::vector<T> &h, const T **out)
{
    *out = nullptr;
    if (h.empty()) return HARM_OK;
    void *p = nullptr;
    HARM_CUDA(cudaMalloc(&p, h.size() * sizeof(T)), "cudaMalloc scene table");
    s->allocs.push_back(p);
    HARM_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s->stream),
              "upload scene table");
    *out = (const T *)p;
    return HARM_OK;
}

void free_scene(harm_scene *s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    harm::release_host_ring(s);
    for (void *p : s->allocs) cudaFree(p);
    for (void *p : s->lut_mem)
        if (p) cudaFree(p);
    delete s;
}

harm_status check_window(const harm_scene *s, int32_t n0, int32_t np)
{
    if (!s) return fail(HARM_E_INVALID, "scene is NULL");
    if (np < 0 || n0 < 0 || (int64_t)n0 + np > s->desc.n_pulses)
        return fail(HARM_E_INVALID, "pulse window [%d, %d) outside [0, %d)", n0, n0 + np, s->desc.n_pulses);
    return HARM_OK;
}

harm_status check_device(const harm_scene *s)
{
    int dev = -1;
    HARM_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != s->device) return fail(HARM_E_INVALID, "scene lives on device %d, current device is %d", s->device, dev);
    return HARM_OK;
}

harm_status check_ptr(const void *p, size_t bytes, const char *what)
{
    return harm::check_device_span(p, bytes, what);
}

// Driver query of the allocation that holds a device address (base, size),
// fetched through the runtime so that the library does not link the driver
// library itself; null when the driver does not offer it.
typedef int (*AddressRangeFn)(unsigned long long *base, size_t *size, unsigned long long ptr);

AddressRangeFn address_range_fn()
{
    static AddressRangeFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<AddressRangeFn>(f);
    }();
    return fn;
}

typedef int (*TensorMapEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tiled tensor-map encoder, fetched through the runtime; null when
// the driver does not offer it.
TensorMapEncodeFn tensor_map_encode_fn()
{
    static TensorMapEncodeFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<TensorMapEncodeFn>(f);
    }();
    return fn;
}

}  // namespace

namespace harm {

cudaError_t encode_state_map(void *map, float *state, int nx, int ny, int nf, int np, int box_x, int box_y)
{
    TensorMapEncodeFn fn = tensor_map_encode_fn();
    if (!fn || nx <= 0 || ny <= 0 || np <= 0 || nx % 4 != 0 || reinterpret_cast<uintptr_t>(state) % 16 != 0)
        return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nf, (cuuint64_t)np};
    const cuuint64_t strides[3] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4, (cuuint64_t)nx * ny * nf * 4};
    const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)nf, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const int r = fn(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, state, dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == 0 ? cudaSuccess : cudaErrorInvalidValue;
}

harm_status check_device_span(const void *p, size_t bytes, const char *what)
{
    if (!p) return fail(HARM_E_INVALID, "%s is NULL", what);
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes");
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(HARM_E_INVALID, "%s is not device memory", what);
    int dev = -1;
    HARM_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
        return fail(HARM_E_INVALID, "%s is memory of device %d, the current device is %d", what, a.device, dev);
    if (a.type == cudaMemoryTypeDevice && bytes > 0) {
        if (AddressRangeFn fn = address_range_fn()) {
            unsigned long long base = 0;
            size_t size = 0;
            const unsigned long long ptr = (unsigned long long)(uintptr_t)p;
            if (fn(&base, &size, ptr) == 0 && ptr >= base) {
                const size_t avail = (size_t)(base + size - ptr);
                if (bytes > avail)
                    return fail(HARM_E_INVALID,
                                "%s: the call touches %zu bytes, its allocation holds %zu from the pointer", what,
                                bytes, avail);
            }
        }
    }
    return HARM_OK;
}

}  // namespace harm

namespace harm {
harm_status set_error(harm_status s, const char *msg)
{
    g_last_error = msg;
    return s;
}
}  // namespace harm

extern "C" {

const char *harm_last_error(void) { return g_last_error.c_str(); }

harm_status harm_scene_create(const harm_scene_desc *desc, void *cuda_stream, harm_scene **out)
{
    if (!out) return fail(HARM_E_INVALID, "out is NULL");
    *out = nullptr;
    harm_scene_desc dn;
    harm_status st = normalize(desc, &dn);
    if (st != HARM_OK) return st;
    if ((st = validate(&dn)) != HARM_OK) return st;
    harm_scene *s = new (std::nothrow) harm_scene;
    if (!s) return fail(HARM_E_OOM, "host allocation failed");
    s->desc = dn;
    s->rx.assign(dn.rx, dn.rx + dn.n_channels);
    s->desc.rx = nullptr;
    if (dn.hetero_ncx > 0) {
        const int nco = dn.hetero_ncx * dn.hetero_ncy;
        s->het_u10.assign(dn.hetero_u10, dn.hetero_u10 + nco);
        s->het_dir.assign(dn.hetero_wind_dir_rad, dn.hetero_wind_dir_rad + nco);
    }
    s->desc.hetero_u10 = nullptr;
    s->desc.hetero_wind_dir_rad = nullptr;
    s->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "cudaGetDevice");
    }
    st = harm::build_scene_tables(s);
    if (st != HARM_OK) {
        std::string msg = g_last_error;
        free_scene(s);
        g_last_error = msg;
        return st;
    }
    *out = s;
    return HARM_OK;
}

harm_status harm_scene_destroy(harm_scene *scene)
{
    free_scene(scene);
    return HARM_OK;
}

harm_status harm_scene_query(const harm_scene *s, harm_scene_info *info)
{
    if (!s || !info) return fail(HARM_E_INVALID, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->n_facets = s->nf;
    info->n_pulses = s->desc.n_pulses;
    info->n_range = s->desc.n_range;
    info->n_channels = s->desc.n_channels;
    info->n_waves = s->nw;
    info->precision = s->desc.precision;
    info->pulse_batch = s->mixed.nb;
    info->range_bin_m = harm::kC / s->desc.fs_hz;
    for (int c = 0; c < s->desc.n_channels; ++c) info->range_start_m[c] = s->r0[c];
    return HARM_OK;
}

harm_status harm_scene_set_cells(harm_scene *s, int32_t ncx, int32_t ncy, double cell_m, const double *sigma0_dev,
                                 const double *uv_dev)
{
    if (!s) return fail(HARM_E_INVALID, "scene is NULL");
    if (ncx == 0) {
        s->dev.ncx = s->dev.ncy = 0;
        s->dev.cell_sigma0 = s->dev.cell_uv = nullptr;
        return HARM_OK;
    }
    if (ncx < 1 || ncy < 1 || !(cell_m > 0) || (int64_t)ncx * ncy > (1 << 27))
        return fail(HARM_E_INVALID, "bad cell grid %d x %d of %g m", ncx, ncy, cell_m);
    if (sigma0_dev) {
        harm_status st = check_ptr(sigma0_dev, (size_t)ncx * ncy * sizeof(double), "sigma0_dev");
        if (st != HARM_OK) return st;
    }
    if (uv_dev) {
        harm_status st = check_ptr(uv_dev, (size_t)ncx * ncy * 2 * sizeof(double), "uv_dev");
        if (st != HARM_OK) return st;
    }
    s->dev.ncx = ncx;
    s->dev.ncy = ncy;
    s->dev.cell = cell_m;
    s->dev.cell_sigma0 = sigma0_dev;
    s->dev.cell_uv = uv_dev;
    return HARM_OK;
}

harm_status harm_scene_set_pattern(harm_scene *s, int32_t antenna, int32_t nu, int32_t nv, double u0, double du,
                                   double v0, double dv, const double *gain_host)
{
    if (!s) return fail(HARM_E_INVALID, "scene is NULL");
    if (antenna < -1 || antenna >= s->desc.n_channels)
        return fail(HARM_E_INVALID, "antenna %d: -1 (transmitter) or 0..%d", antenna, s->desc.n_channels - 1);
    harm_status st = check_device(s);
    if (st != HARM_OK) return st;
    const int slot = antenna + 1;
    if (gain_host) {
        if (nu < 2 || nv < 2 || nu > 65536 || nv > 65536)
            return fail(HARM_E_INVALID, "u-v grid %d x %d: need 2..65536 nodes per axis", nu, nv);
        if (!(du > 0) || !(dv > 0) || !std::isfinite(du) || !std::isfinite(dv) || !std::isfinite(u0) ||
            !std::isfinite(v0))
            return fail(HARM_E_INVALID, "u-v grid origin must be finite and steps positive");
        const size_t nn = (size_t)nu * nv;
        for (size_t i = 0; i < 2 * nn; ++i)
            if (!std::isfinite(gain_host[i])) return fail(HARM_E_INVALID, "u-v grid holds a non-finite gain");
    }
    HARM_CUDA(cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");  // kernels may still read the old grid
    if (s->lut_mem[slot]) {
        cudaFree(s->lut_mem[slot]);
        s->lut_mem[slot] = nullptr;
    }
    s->dev.lut_mask &= ~(1u << slot);
    harm::PatLut L{};
    if (gain_host) {
        const size_t nn = (size_t)nu * nv;
        L.nu = nu;
        L.nv = nv;
        L.u0 = u0;
        L.inv_du = 1.0 / du;
        L.v0 = v0;
        L.inv_dv = 1.0 / dv;
        void *p = nullptr;
        if (s->desc.precision != HARM_PREC_MIXED) {  // the plain paths read the grid in double
            HARM_CUDA(cudaMalloc(&p, nn * sizeof(double2)), "cudaMalloc u-v grid");
            cudaError_t e = cudaMemcpy(p, gain_host, nn * sizeof(double2), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                cudaFree(p);
                return cuda_fail(e, "upload u-v grid");
            }
            L.g64 = (const double2 *)p;
        } else {
            // each entry holds a node and its right neighbour: a bilinear lookup reads two
            // 16-byte entries (rows j and j + 1)
            const size_t np = (size_t)(nu - 1) * nv;
            std::vector<float4> g32(np);
            for (int j = 0; j < nv; ++j)
                for (int i = 0; i + 1 < nu; ++i) {
                    const double *a = gain_host + 2 * ((size_t)j * nu + i);
                    g32[(size_t)j * (nu - 1) + i] = make_float4((float)a[0], (float)a[1], (float)a[2], (float)a[3]);
                }
            HARM_CUDA(cudaMalloc(&p, np * sizeof(float4)), "cudaMalloc u-v grid");
            cudaError_t e = cudaMemcpy(p, g32.data(), np * sizeof(float4), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                cudaFree(p);
                return cuda_fail(e, "upload u-v grid");
            }
            L.g32 = (const float4 *)p;
        }
        s->lut_mem[slot] = p;
        s->dev.lut_mask |= 1u << slot;
    }
    s->luts[slot] = L;
    HARM_CUDA(cudaMemcpy(s->luts_dev + slot, &L, sizeof(L), cudaMemcpyHostToDevice), "upload u-v grid descriptor");
    return HARM_OK;
}

harm_status harm_facets_generate(harm_scene *s, int32_t n0, int32_t np, void *state_dev)
{
    harm_status st = check_window(s, n0, np);
    if (st != HARM_OK) return st;
    if ((st = check_device(s)) != HARM_OK) return st;
    if (np == 0) return HARM_OK;
    const size_t state_bytes = (size_t)np * (s->desc.cwm ? 8 : 3) * (size_t)s->nf *
                               (s->desc.precision == HARM_PREC_FP64 ? sizeof(double) : sizeof(float));
    if ((st = check_ptr(state_dev, state_bytes, "state_dev")) != HARM_OK) return st;
    cudaError_t e = harm::launch_generate(s, n0, np, state_dev);
    if (e != cudaSuccess) return cuda_fail(e, "facet generator launch");
    return HARM_OK;
}

harm_status harm_scene_set_deterministic(harm_scene *s, int32_t on)
{
    if (!s) return fail(HARM_E_INVALID, "scene is NULL");
    if (on && s->desc.precision == HARM_PREC_MIXED)
        return fail(HARM_E_UNSUPPORTED, "deterministic sums are offered by the plain paths (FP64, FP32)");
    s->dev.det = on ? 1 : 0;
    return HARM_OK;
}

harm_status harm_echo_accumulate(harm_scene *s, int32_t n0, int32_t np, void *iq_dev, harm_dtype dtype,
                                 int32_t zero_first)
{
    harm_status st = check_window(s, n0, np);
    if (st != HARM_OK) return st;
    if ((st = check_device(s)) != HARM_OK) return st;
    if (dtype != HARM_C64 && dtype != HARM_C128) return fail(HARM_E_INVALID, "unknown dtype %d", (int)dtype);
    if (s->dev.det && dtype != HARM_C128)
        return fail(HARM_E_UNSUPPORTED, "deterministic sums need complex128 output");
    if (np == 0) return HARM_OK;
    size_t bytes = (size_t)s->desc.n_channels * np * s->desc.n_range * (dtype == HARM_C64 ? 8 : 16);
    if ((st = check_ptr(iq_dev, bytes, "iq_dev")) != HARM_OK) return st;
    if (zero_first) HARM_CUDA(cudaMemsetAsync(iq_dev, 0, bytes, s->stream), "cudaMemsetAsync iq");
    cudaError_t e = harm::launch_accumulate(s, n0, np, iq_dev, dtype);
    if (e != cudaSuccess) return cuda_fail(e, "echo accumulator launch");
    return HARM_OK;
}

harm_status harm_echo_adjoint(harm_scene *s, int32_t n0, int32_t np, const void *resid_dev, harm_dtype dtype,
                              double *grad_sigma0_dev, double *grad_uv_dev)
{
    harm_status st = check_window(s, n0, np);
    if (st != HARM_OK) return st;
    if ((st = check_device(s)) != HARM_OK) return st;
    if (dtype != HARM_C64 && dtype != HARM_C128) return fail(HARM_E_INVALID, "unknown dtype %d", (int)dtype);
    if (s->dev.ncx == 0) return fail(HARM_E_INVALID, "adjoint needs per-cell fields (harm_scene_set_cells)");
    if (np == 0) return HARM_OK;
    const size_t rbytes = (size_t)s->desc.n_channels * np * s->desc.n_range * (dtype == HARM_C64 ? 8 : 16);
    const size_t cells = (size_t)s->dev.ncx * s->dev.ncy;
    if ((st = check_ptr(resid_dev, rbytes, "resid_dev")) != HARM_OK) return st;
    if (grad_sigma0_dev && (st = check_ptr(grad_sigma0_dev, cells * sizeof(double), "grad_sigma0_dev")) != HARM_OK)
        return st;
    if (grad_uv_dev && (st = check_ptr(grad_uv_dev, cells * 2 * sizeof(double), "grad_uv_dev")) != HARM_OK)
        return st;
    cudaError_t e = harm::launch_adjoint(s, n0, np, resid_dev, dtype, grad_sigma0_dev, grad_uv_dev);
    if (e == cudaErrorNotSupported) return fail(HARM_E_UNSUPPORTED, "adjoint not available for this scene");
    if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
    return HARM_OK;
}

harm_status harm_probe_indices(harm_scene *s, int32_t n0, int32_t np, int32_t *bins_dev, void *speckle_dev,
                               uint32_t *words_dev, int32_t *cells_dev)
{
    harm_status st = check_window(s, n0, np);
    if (st != HARM_OK) return st;
    if ((st = check_device(s)) != HARM_OK) return st;
    if (np == 0) return HARM_OK;
    const bool fp64 = s->desc.precision == HARM_PREC_FP64;
    const size_t nf = (size_t)s->nf, npl = (size_t)np;
    if ((st = check_ptr(bins_dev, npl * s->desc.n_channels * nf * 4, "bins_dev")) != HARM_OK) return st;
    if ((st = check_ptr(speckle_dev, npl * nf * (fp64 ? 16 : 8), "speckle_dev")) != HARM_OK) return st;
    if ((st = check_ptr(words_dev, npl * nf * 16, "words_dev")) != HARM_OK) return st;
    if ((st = check_ptr(cells_dev, nf * 4, "cells_dev")) != HARM_OK) return st;
    cudaError_t e =
        s->desc.precision == HARM_PREC_MIXED
            ? harm::launch_probe_mixed(s->dev, s->mixed, s->stream, n0, np, bins_dev, speckle_dev, words_dev, cells_dev)
            : harm::launch_probe_plain(s->dev, fp64, s->stream, n0, np, bins_dev, speckle_dev, words_dev, cells_dev);
    if (e != cudaSuccess) return cuda_fail(e, "index probe launch");
    return HARM_OK;
}

harm_status harm_scene_sync(harm_scene *s)
{
    if (!s) return fail(HARM_E_INVALID, "scene is NULL");
    HARM_CUDA(cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    unsigned int flags[4] = {0, 0, 0, 0};
    HARM_CUDA(cudaMemcpy(flags, s->dev.flags, sizeof(flags), cudaMemcpyDeviceToHost), "read device flags");
    HARM_CUDA(cudaMemset(s->dev.flags, 0, sizeof(flags)), "clear device flags");
    if (flags[0]) return fail(HARM_E_TIMEOUT, "a bounded device wait gave up (%u times)", flags[0]);
    if (flags[1]) return fail(HARM_E_CUDA, "device bounds check failed (%u times)", flags[1]);
    return HARM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Scene tables
// ---------------------------------------------------------------------------
namespace harm {

harm_status build_scene_tables(harm_scene *s)
{
    const harm_scene_desc &d = s->desc;
    const int np = d.n_pulses, nc = d.n_channels, nx = d.nx, ny = d.ny;
    s->nf = (int64_t)nx * ny;
    DevScene &v = s->dev;
    v.nx = nx;
    v.ny = ny;
    v.nc = nc;
    v.nr = d.n_range;
    v.np_total = np;
    v.taps = d.taps;
    v.static_surface = d.static_surface ? 1 : 0;
    v.epoch_pulses = d.epoch_pulses;
    v.dx = d.facet_m;
    double lambda = kC / d.f0_hz;
    v.k0 = 2.0 * kPi / lambda;
    v.inv_lambda = 1.0 / lambda;
    v.inv_dr = d.fs_hz / kC;
    v.area = d.facet_m * d.facet_m;
    v.tx_laz = d.tx.len_az;
    v.tx_lel = d.tx.len_el;
    for (int c = 0; c < nc; ++c) {
        v.rx_laz[c] = s->rx[c].len_az;
        v.rx_lel[c] = s->rx[c].len_el;
    }
    v.sigma0_base = d.sigma0_base;
    v.wind_mod = d.wind_mod;
    v.wcos = std::cos(d.wind_dir_rad);
    v.wsin = std::sin(d.wind_dir_rad);
    v.cur_u = d.current_u;
    v.cur_v = d.current_v;
    v.speckle_seed = d.speckle_seed;
    // AR(1) speckle (Eq. 10) between epochs of epoch_pulses / prf; when a pulse
    // window starts mid-burst the recurrence is restarted from the last terms
    // whose weight beta^m is above 2^-40
    v.spk_beta = 0.0;
    v.spk_q = 1.0;
    v.spk_terms = 1;
    if (d.speckle_tau_s > 0.0 && d.epoch_pulses > 0) {
        double b = std::exp(-((double)d.epoch_pulses / d.prf_hz) / d.speckle_tau_s);
        if (b > 0.0) {
            v.spk_beta = b;
            v.spk_q = std::sqrt(1.0 - b * b);
            double m = std::ceil(40.0 * std::log(2.0) / -std::log(b)) + 1.0;
            v.spk_terms = m > 1e9 ? 1000000000 : (int)m;
        }
    }
    v.fd_hz = d.speckle_doppler_hz;
    // phase centres of one receive antenna: same aperture, same velocity, within
    // 50 m of the previous channel. Their direction cosines to any facet differ by
    // ~(patch size / R) x (separation / R) ~ 1e-8, so the mixed path evaluates the
    // analytic pattern once per antenna.
    v.rx_share = 0u;
    for (int c = 1; c < nc; ++c) {
        const harm_antenna &a = s->rx[c], &b = s->rx[c - 1];
        double sep[3] = {a.pos0[0] - b.pos0[0], a.pos0[1] - b.pos0[1], a.pos0[2] - b.pos0[2]};
        if (a.len_az == b.len_az && a.len_el == b.len_el && a.vel[0] == b.vel[0] && a.vel[1] == b.vel[1] &&
            a.vel[2] == b.vel[2] && norm3(sep) <= 50.0)
            v.rx_share |= 1u << c;
    }
    v.cwm = d.cwm;
    v.het_ncx = d.hetero_ncx;
    v.het_ncy = d.hetero_ncy;
    v.het_l = d.hetero_tile_m;
    v.het_x0 = -0.5 * nx * d.facet_m;
    v.het_y0 = -0.5 * ny * d.facet_m;
    v.lut_mask = 0u;
    // Kaiser window I0(beta sqrt(v)) / I0(beta) as a power series in v = 1 - (x/4)^2:
    // coefficient k is (beta^2/4)^k / (k!)^2, divided by I0(beta) = sum of them.
    {
        double q = 0.25 * d.kaiser_beta * d.kaiser_beta;
        double c[kMaxI0Terms];
        double term = 1.0, sum = 0.0;
        int n = 0;
        for (; n < kMaxI0Terms; ++n) {
            if (n > 0) term *= q / ((double)n * n);
            c[n] = term;
            sum += term;
            if (n > 2 && term < 1e-18 * sum) {
                ++n;
                break;
            }
        }
        v.n_i0 = n;
        for (int k = 0; k < n; ++k) v.i0c[k] = c[k] / sum;
    }

    // per-pulse platform state
    std::vector<PulseState> ps(np);
    std::vector<RxState> rs((size_t)np * nc);
    for (int n = 0; n < np; ++n) pulse_geometry(d, s->rx, n, ps[n], &rs[(size_t)n * nc]);
    double dr = kC / d.fs_hz;
    s->r0.resize(nc);
    for (int c = 0; c < nc; ++c) {
        const PulseState &pm = ps[np / 2];
        const RxState &rm = rs[(size_t)(np / 2) * nc + c];
        s->r0[c] = pm.tx.rref + rm.rx.rref - 0.5 * d.n_range * dr;
    }
    for (int n = 0; n < np; ++n)
        for (int c = 0; c < nc; ++c) {
            RxState &r = rs[(size_t)n * nc + c];
            double rsum = ps[n].tx.rref + r.rx.rref;
            r.psi = reduced_phase(d.f0_hz, rsum);
            r.p_ref = (rsum - s->r0[c]) / dr;
        }

    // waves: wave numbers and frequencies of every wave set here; their separable
    // phasor tables e^{i kx x}, a e^{i phi} e^{i ky y} (and e^{-i omega t_s} for the
    // FP64 path) are evaluated on the device by phasor_tables
    const WaveSets W = wave_sets(s);
    const int nw = W.nw, nsets = W.n_sets;
    s->nw = nw;
    v.nw = nw;
    v.n_sets = nsets;
    std::vector<double> kx((size_t)nsets * nw), ky((size_t)nsets * nw), om((size_t)nsets * nw),
        kn((size_t)nsets * nw);
    for (int q = 0; q < nsets; ++q)
        for (int m = 0; m < nw; ++m) {
            const Wave &w = W.at(q, m);
            const size_t qm = (size_t)q * nw + m;
            kx[qm] = w.kx;
            ky[qm] = w.ky;
            om[qm] = w.om;
            kn[qm] = std::sqrt(w.kx * w.kx + w.ky * w.ky);
        }

    harm_status st;
    if ((st = upload(s, ps, &v.pulses)) != HARM_OK) return st;
    if ((st = upload(s, rs, &v.rx)) != HARM_OK) return st;
    if ((st = upload(s, kx, &v.kx)) != HARM_OK) return st;
    if ((st = upload(s, ky, &v.ky)) != HARM_OK) return st;
    if ((st = upload(s, om, &v.om)) != HARM_OK) return st;
    if ((st = upload(s, kn, &v.kn)) != HARM_OK) return st;
    // u-v gain grids: none until harm_scene_set_pattern
    s->luts.assign(1 + nc, PatLut{});
    s->lut_mem.assign(1 + nc, nullptr);
    {
        const PatLut *lp = nullptr;
        if ((st = upload(s, s->luts, &lp)) != HARM_OK) return st;
        s->luts_dev = const_cast<PatLut *>(lp);
        v.luts = lp;
    }
    if (d.precision == HARM_PREC_FP64)
        HARM_CUDA(phasor_tables<double2>(s, W, v.pulses, &v.ex, &v.ey, &v.tt), "wave phasor tables");
    if (d.precision == HARM_PREC_FP32)
        HARM_CUDA(phasor_tables<float2>(s, W, v.pulses, &v.ex32, &v.ey32, &v.tt32), "wave phasor tables");
    std::vector<unsigned int> flags(4, 0u);
    const unsigned int *fl = nullptr;
    if ((st = upload(s, flags, &fl)) != HARM_OK) return st;
    v.flags = const_cast<unsigned int *>(fl);
    if (d.precision == HARM_PREC_MIXED) {
        st = build_mixed_tables(s, ps, W);
        if (st != HARM_OK) return fail(st, "mixed-precision table upload failed");
    }
    HARM_CUDA(cudaStreamSynchronize(s->stream), "scene upload");
    return HARM_OK;
}

}  // namespace harm
