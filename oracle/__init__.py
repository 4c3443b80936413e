"""Plain FP64 CPU oracle of the facet-to-IQ echo -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg may
import this package. The product path never does, and this package imports
nothing from the CUDA path. The arithmetic lives in ``harm_oracle.c`` (plain C,
double precision, direct evaluation of every definition); this module compiles it
with gcc and marshals scene descriptors from :mod:`harm_scenes` into its own
struct.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "harm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXC = 16


class _Antenna(C.Structure):
    _fields_ = [("pos0", C.c_double * 3), ("vel", C.c_double * 3),
                ("len_az", C.c_double), ("len_el", C.c_double)]


class _Lut(C.Structure):
    _fields_ = [("nu", C.c_int), ("nv", C.c_int), ("u0", C.c_double), ("du", C.c_double),
                ("v0", C.c_double), ("dv", C.c_double), ("g", C.POINTER(C.c_double))]


class OrScene(C.Structure):
    _fields_ = [
        ("f0", C.c_double), ("fs", C.c_double), ("prf", C.c_double),
        ("n_pulses", C.c_int), ("n_range", C.c_int),
        ("tx", _Antenna),
        ("n_channels", C.c_int),
        ("rx", _Antenna * MAXC),
        ("nx", C.c_int), ("ny", C.c_int),
        ("facet", C.c_double),
        ("n_omega", C.c_int), ("n_theta", C.c_int),
        ("u10", C.c_double), ("fetch", C.c_double), ("wind_dir", C.c_double),
        ("spread_s", C.c_double), ("gamma", C.c_double),
        ("wave_seed", C.c_uint64),
        ("cur_u", C.c_double), ("cur_v", C.c_double),
        ("sigma0_base", C.c_double), ("wind_mod", C.c_double),
        ("epoch_pulses", C.c_int),
        ("speckle_seed", C.c_uint64),
        ("static_surface", C.c_int),
        ("taps", C.c_int),
        ("beta", C.c_double),
        ("ncx", C.c_int), ("ncy", C.c_int), ("cell", C.c_double),
        ("cell_sigma0", C.POINTER(C.c_double)),
        ("cell_uv", C.POINTER(C.c_double)),
        ("tau_s", C.c_double), ("doppler_hz", C.c_double),
        ("cwm", C.c_int),
        ("het_l", C.c_double), ("het_ncx", C.c_int), ("het_ncy", C.c_int),
        ("het_u10", C.POINTER(C.c_double)), ("het_dir", C.POINTER(C.c_double)),
        ("lut", _Lut * (1 + MAXC)),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, OpenMP,
    no floating-point contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                       C.POINTER(C.c_uint32)]
        L.or_speckle.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, dp, dp]
        L.or_jonswap_params.argtypes = [C.c_double, C.c_double, dp, dp]
        L.or_jonswap.argtypes = [C.c_double] * 4
        L.or_jonswap.restype = C.c_double
        L.or_spreading.argtypes = [C.c_double, C.c_double]
        L.or_spreading.restype = C.c_double
        L.or_wave_table.argtypes = [C.POINTER(OrScene), dp, dp, dp, dp, dp]
        L.or_wave_table.restype = C.c_int
        L.or_surface.argtypes = [C.c_int, dp, dp, dp, dp, dp, C.c_double, C.c_double,
                                 C.c_double, dp]
        L.or_pulse_state_flat.argtypes = [C.POINTER(OrScene), C.c_int, C.c_int, dp]
        L.or_pattern.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp, dp]
        L.or_pattern.restype = C.c_double
        L.or_bessel_i0.argtypes = [C.c_double]
        L.or_bessel_i0.restype = C.c_double
        L.or_kaiser_sinc.argtypes = [C.c_double, C.c_int, C.c_double]
        L.or_kaiser_sinc.restype = C.c_double
        L.or_sigma0.argtypes = [C.POINTER(OrScene), C.c_double, dp, dp, C.c_double, C.c_double]
        L.or_sigma0.restype = C.c_double
        L.or_range_start.argtypes = [C.POINTER(OrScene), C.c_int]
        L.or_range_start.restype = C.c_double
        L.or_epoch.argtypes = [C.POINTER(OrScene), C.c_int]
        L.or_epoch.restype = C.c_uint32
        L.or_facet_states.argtypes = [C.POINTER(OrScene), C.c_int, dp]
        L.or_speckle_beta.argtypes = [C.POINTER(OrScene)]
        L.or_speckle_beta.restype = C.c_double
        L.or_speckle_ar1.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_double, dp, dp]
        L.or_wave_table_corner.argtypes = [C.POINTER(OrScene), C.c_int, dp, dp, dp, dp, dp]
        L.or_wave_table_corner.restype = C.c_int
        L.or_surface_cwm.argtypes = [C.c_int, dp, dp, dp, dp, dp, C.c_double, C.c_double,
                                     C.c_double, dp]
        L.or_hetero_weight.argtypes = [C.POINTER(OrScene), C.c_int, C.c_int, C.c_double, C.c_double]
        L.or_hetero_weight.restype = C.c_double
        L.or_lut_gain.argtypes = [C.POINTER(_Lut), C.c_double, C.c_double, dp]
        L.or_sigma0_normal.argtypes = [C.POINTER(OrScene), C.c_double, dp, dp, dp]
        L.or_sigma0_normal.restype = C.c_double
        L.or_echo.argtypes = [C.POINTER(OrScene), C.c_int, C.POINTER(C.c_int), C.c_int64,
                              C.POINTER(C.c_int64), dp]
        L.or_echo.restype = C.c_int
        L.or_contribution.argtypes = [C.POINTER(OrScene), C.c_int, C.c_int, C.c_int64, dp, dp]
        L.or_num_threads.restype = C.c_int
        L.or_set_num_threads.argtypes = [C.c_int]
        L.or_set_num_threads.restype = None
        L.or_bin_positions.argtypes = [C.POINTER(OrScene), C.c_int, C.POINTER(C.c_int), dp,
                                       C.POINTER(C.c_int)]
        L.or_bin_positions.restype = C.c_int
        u32p = C.POINTER(C.c_uint32)
        L.or_speckle_words.argtypes = [C.c_uint64, C.c_int64, u32p, u32p, u32p]
        L.or_speckle_words.restype = None
        L.or_adjoint.argtypes = [C.POINTER(OrScene), C.c_int, C.POINTER(C.c_int), dp, dp, dp]
        L.or_adjoint.restype = C.c_int
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Scene:
    """A descriptor (dict from :mod:`harm_scenes`) marshalled into the oracle's
    struct. Keeps the per-cell arrays alive."""

    def __init__(self, desc: dict):
        self.desc = desc
        s = OrScene()
        s.f0, s.fs, s.prf = desc["f0_hz"], desc["fs_hz"], desc["prf_hz"]
        s.n_pulses, s.n_range = desc["n_pulses"], desc["n_range"]
        _fill_antenna(s.tx, desc["tx"])
        rx = desc["rx"]
        if len(rx) > MAXC:
            raise ValueError("too many channels for the oracle")
        s.n_channels = len(rx)
        for i, a in enumerate(rx):
            _fill_antenna(s.rx[i], a)
        s.nx, s.ny, s.facet = desc["nx"], desc["ny"], desc["facet_m"]
        s.n_omega, s.n_theta = desc["n_omega"], desc["n_theta"]
        s.u10, s.fetch, s.wind_dir = desc["u10"], desc["fetch_m"], desc["wind_dir_rad"]
        s.spread_s, s.gamma, s.wave_seed = desc["spread_s"], desc["gamma"], desc["wave_seed"]
        s.cur_u, s.cur_v = desc["current_u"], desc["current_v"]
        s.sigma0_base, s.wind_mod = desc["sigma0_base"], desc["wind_mod"]
        s.epoch_pulses, s.speckle_seed = desc["epoch_pulses"], desc["speckle_seed"]
        s.static_surface = desc["static_surface"]
        s.taps, s.beta = desc["taps"], desc["kaiser_beta"]
        self._keep = []
        cells = desc.get("cells")
        if cells is not None:
            s.ncx, s.ncy, s.cell = cells["ncx"], cells["ncy"], cells["cell_m"]
            if cells.get("sigma0") is not None:
                a = np.ascontiguousarray(cells["sigma0"], dtype=np.float64)
                self._keep.append(a)
                s.cell_sigma0 = _dptr(a)
            if cells.get("uv") is not None:
                a = np.ascontiguousarray(cells["uv"], dtype=np.float64)
                self._keep.append(a)
                s.cell_uv = _dptr(a)
        s.tau_s = desc.get("speckle_tau_s", 0.0)
        s.doppler_hz = desc.get("speckle_doppler_hz", 0.0)
        s.cwm = int(desc.get("cwm", 0))
        het = desc.get("hetero")
        if het is not None:
            u = np.ascontiguousarray(het["u10"], dtype=np.float64)
            w = np.ascontiguousarray(het["wind_dir"], dtype=np.float64)
            s.het_ncy, s.het_ncx = u.shape
            s.het_l = het["tile_m"]
            self._keep += [u, w]
            s.het_u10, s.het_dir = _dptr(u), _dptr(w)
        for ant, pat in (desc.get("patterns") or {}).items():
            _fill_lut(s.lut[0 if ant == "tx" else 1 + int(ant)], pat, self._keep)
        self.s = s

    @property
    def ref(self):
        return C.byref(self.s)


def _fill_lut(dst, pat, keep):
    g = np.asarray(pat["gain"], dtype=np.complex128)
    a = np.ascontiguousarray(np.stack([g.real, g.imag], axis=-1))
    keep.append(a)
    dst.nv, dst.nu = g.shape
    dst.u0, dst.du, dst.v0, dst.dv = pat["u0"], pat["du"], pat["v0"], pat["dv"]
    dst.g = _dptr(a)


def _fill_antenna(dst, a):
    for i in range(3):
        dst.pos0[i] = a["pos0"][i]
        dst.vel[i] = a["vel"][i]
    dst.len_az, dst.len_el = a["len_az"], a["len_el"]


# --------------------------------------------------------------------------
# thin wrappers
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def speckle(seed, f, epoch):
    re, im = C.c_double(), C.c_double()
    lib().or_speckle(seed, f, epoch, C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def jonswap_params(u10, fetch):
    wp, al = C.c_double(), C.c_double()
    lib().or_jonswap_params(u10, fetch, C.byref(wp), C.byref(al))
    return wp.value, al.value


def jonswap(omega, u10, fetch, gamma):
    return lib().or_jonswap(omega, u10, fetch, gamma)


def spreading(dtheta, s):
    return lib().or_spreading(dtheta, s)


def wave_table(desc):
    sc = Scene(desc)
    n = desc["n_omega"] * desc["n_theta"]
    arrs = [np.zeros(n) for _ in range(5)]
    lib().or_wave_table(sc.ref, *[_dptr(a) for a in arrs])
    return dict(zip(["kx", "ky", "omega", "amp", "phase"], arrs))


def surface(table, x, y, t):
    n = len(table["kx"])
    out = np.zeros(3)
    ts = [np.ascontiguousarray(table[k]) for k in ("kx", "ky", "omega", "amp", "phase")]
    lib().or_surface(n, *[_dptr(a) for a in ts], float(x), float(y), float(t), _dptr(out))
    return out


def pulse_state(desc, n, c):
    sc = Scene(desc)
    o = np.zeros(23)
    lib().or_pulse_state_flat(sc.ref, n, c, _dptr(o))
    return {"t": o[0], "ts": o[1], "trx": o[2], "ptx": o[3:6].copy(), "prx": o[6:9].copy(),
            "rt_ref": o[9], "rr_ref": o[10], "atx": o[11:14].copy(), "etx": o[14:17].copy(),
            "arx": o[17:20].copy(), "erx": o[20:23].copy()}


def pattern(len_az, len_el, lam, d, a, e):
    arr = [np.ascontiguousarray(v, dtype=np.float64) for v in (d, a, e)]
    return lib().or_pattern(len_az, len_el, lam, *[_dptr(v) for v in arr])


def bessel_i0(x):
    return lib().or_bessel_i0(float(x))


def kaiser_sinc(x, m, beta):
    return lib().or_kaiser_sinc(float(x), int(m), float(beta))


def sigma0(desc, base, rt_hat, rr_hat, sx, sy):
    sc = Scene(desc)
    a = np.ascontiguousarray(rt_hat, dtype=np.float64)
    b = np.ascontiguousarray(rr_hat, dtype=np.float64)
    return lib().or_sigma0(sc.ref, base, _dptr(a), _dptr(b), sx, sy)


def range_start(desc, c):
    return lib().or_range_start(Scene(desc).ref, c)


def epoch(desc, n):
    return lib().or_epoch(Scene(desc).ref, n)


def facet_states(desc, n, fields=3):
    """Facet states of every facet at pulse n: array [fields, ny, nx] of
    (eta, eta_x, eta_y, D_x, D_y, dD_x/dx, dD_x/dy, dD_y/dy)[:fields]."""
    sc = Scene(desc)
    out = np.zeros((8, desc["ny"], desc["nx"]))
    lib().or_facet_states(sc.ref, n, _dptr(out))
    return out[:fields].copy()


def speckle_beta(desc):
    return lib().or_speckle_beta(Scene(desc).ref)


def speckle_ar1(seed, f, epoch, beta):
    re, im = C.c_double(), C.c_double()
    lib().or_speckle_ar1(seed, f, epoch, beta, C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def wave_table_corner(desc, corner):
    sc = Scene(desc)
    n = desc["n_omega"] * desc["n_theta"]
    arrs = [np.zeros(n) for _ in range(5)]
    lib().or_wave_table_corner(sc.ref, corner, *[_dptr(a) for a in arrs])
    return dict(zip(["kx", "ky", "omega", "amp", "phase"], arrs))


def surface_cwm(table, x, y, t):
    n = len(table["kx"])
    out = np.zeros(8)
    ts = [np.ascontiguousarray(table[k]) for k in ("kx", "ky", "omega", "amp", "phase")]
    lib().or_surface_cwm(n, *[_dptr(a) for a in ts], float(x), float(y), float(t), _dptr(out))
    return out


def hetero_weight(desc, cx, cy, x, y):
    return lib().or_hetero_weight(Scene(desc).ref, cx, cy, float(x), float(y))


def lut_gain(pat, u, v):
    keep = []
    L = _Lut()
    _fill_lut(L, pat, keep)
    out = np.zeros(2)
    lib().or_lut_gain(C.byref(L), float(u), float(v), _dptr(out))
    return complex(out[0], out[1])


def sigma0_normal(desc, base, rt_hat, rr_hat, nvec):
    sc = Scene(desc)
    a, b, nv = [np.ascontiguousarray(v, dtype=np.float64) for v in (rt_hat, rr_hat, nvec)]
    return lib().or_sigma0_normal(sc.ref, base, _dptr(a), _dptr(b), _dptr(nv))


def contribution(desc, n, c, f, state):
    """One facet's contribution and bin position; state holds (eta, eta_x,
    eta_y) or all 8 fields of the facet state (missing fields are zero)."""
    sc = Scene(desc)
    st = np.zeros(8)
    st[:len(state)] = state
    out = np.zeros(3)
    lib().or_contribution(sc.ref, n, c, f, _dptr(st), _dptr(out))
    return complex(out[0], out[1]), out[2]


def echo(desc, pulses, facets=None):
    """IQ of the listed pulses for every channel: complex128 [n_ch, len(pulses), n_range]."""
    sc = Scene(desc)
    pl = np.ascontiguousarray(pulses, dtype=np.int32)
    nc, nr = len(desc["rx"]), desc["n_range"]
    out = np.zeros((nc, len(pl), nr, 2))
    if facets is None:
        fp, nfac = None, 0
    else:
        fa = np.ascontiguousarray(facets, dtype=np.int64)
        fp, nfac = fa.ctypes.data_as(C.POINTER(C.c_int64)), len(fa)
    lib().or_echo(sc.ref, len(pl), pl.ctypes.data_as(C.POINTER(C.c_int)), nfac, fp, _dptr(out))
    return out[..., 0] + 1j * out[..., 1]


def bin_positions(desc, pulses):
    """Fractional range-bin position p of every facet's contribution at the listed
    pulses, p[i, c, iy, ix], and the facets' cell indices cells[iy, ix] (-1
    without per-cell fields)."""
    sc = Scene(desc)
    pl = np.ascontiguousarray(pulses, dtype=np.int32)
    nc, nx, ny = len(desc["rx"]), desc["nx"], desc["ny"]
    p = np.zeros((len(pl), nc, ny, nx))
    cells = np.zeros((ny, nx), dtype=np.int32)
    lib().or_bin_positions(sc.ref, len(pl), pl.ctypes.data_as(C.POINTER(C.c_int)), _dptr(p),
                           cells.ctypes.data_as(C.POINTER(C.c_int)))
    return p, cells


def speckle_words(seed, facets, epochs):
    """Philox4x32-10 words of the speckle draws of (facet, epoch) pairs:
    uint32 [n, 4]."""
    f = np.ascontiguousarray(facets, dtype=np.uint32)
    e = np.ascontiguousarray(np.broadcast_to(epochs, f.shape), dtype=np.uint32)
    out = np.zeros((f.size, 4), dtype=np.uint32)
    u32p = C.POINTER(C.c_uint32)
    lib().or_speckle_words(int(seed), f.size, f.ctypes.data_as(u32p), e.ctypes.data_as(u32p),
                           out.ctypes.data_as(u32p))
    return out


def num_threads():
    return lib().or_num_threads()


def set_num_threads(n):
    """Threads of later oracle calls (timing only); returns the previous count."""
    prev = num_threads()
    lib().or_set_num_threads(int(n))
    return prev


def adjoint(desc, pulses, resid):
    """Gradients of L = sum |IQ - target|^2 for the residual resid = IQ - target
    (complex [n_ch, len(pulses), n_range]) with respect to the per-cell NRCS base
    and (u, v) current: returns (g_sigma [ncy, ncx], g_uv [ncy, ncx, 2])."""
    sc = Scene(desc)
    cells = desc["cells"]
    ncx, ncy = cells["ncx"], cells["ncy"]
    pl = np.ascontiguousarray(pulses, dtype=np.int32)
    r = np.ascontiguousarray(np.stack([resid.real, resid.imag], axis=-1), dtype=np.float64)
    gs = np.zeros(ncx * ncy)
    gu = np.zeros(ncx * ncy * 2)
    rc = lib().or_adjoint(sc.ref, len(pl), pl.ctypes.data_as(C.POINTER(C.c_int)), _dptr(r), _dptr(gs),
                          _dptr(gu))
    if rc != 0:
        raise ValueError("adjoint needs per-cell fields")
    return gs.reshape(ncy, ncx), gu.reshape(ncy, ncx, 2)


def misfit(desc, pulses, target):
    iq = echo(desc, pulses)
    return float(np.sum(np.abs(iq - target) ** 2)), iq
