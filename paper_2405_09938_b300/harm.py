"""Thin ctypes binding of ``libharm.so`` (the C ABI declared in ``include/harm.h``).

Argument marshalling only: every step of the echo path runs in the library's
CUDA kernels. Torch tensors are used as device buffers and torch streams as CUDA
streams. There is no CPU fallback: loading fails loudly when the library is
missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libharm.so")

HARM_ABI_VERSION = 2
HARM_MAX_CHANNELS = 16
HARM_OK, HARM_E_INVALID, HARM_E_CUDA, HARM_E_OOM, HARM_E_TIMEOUT, HARM_E_UNSUPPORTED = range(6)
HARM_C64, HARM_C128 = 0, 1
HARM_PREC_FP64, HARM_PREC_MIXED, HARM_PREC_FP32 = 0, 1, 2
STATUS_NAMES = {0: "HARM_OK", 1: "HARM_E_INVALID", 2: "HARM_E_CUDA", 3: "HARM_E_OOM",
                4: "HARM_E_TIMEOUT", 5: "HARM_E_UNSUPPORTED"}


class HarmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class harm_antenna(C.Structure):
    _fields_ = [("pos0", C.c_double * 3), ("vel", C.c_double * 3),
                ("len_az", C.c_double), ("len_el", C.c_double)]


class harm_scene_desc(C.Structure):
    _fields_ = [
        ("abi_version", C.c_uint32), ("struct_size", C.c_uint32),
        ("f0_hz", C.c_double), ("fs_hz", C.c_double), ("prf_hz", C.c_double),
        ("n_pulses", C.c_int32), ("n_range", C.c_int32),
        ("tx", harm_antenna),
        ("n_channels", C.c_int32),
        ("rx", C.POINTER(harm_antenna)),
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("facet_m", C.c_double),
        ("n_omega", C.c_int32), ("n_theta", C.c_int32),
        ("u10", C.c_double), ("fetch_m", C.c_double), ("wind_dir_rad", C.c_double),
        ("spread_s", C.c_double), ("gamma", C.c_double),
        ("wave_seed", C.c_uint64),
        ("current_u", C.c_double), ("current_v", C.c_double),
        ("sigma0_base", C.c_double), ("wind_mod", C.c_double),
        ("epoch_pulses", C.c_int32),
        ("speckle_seed", C.c_uint64),
        ("static_surface", C.c_int32),
        ("taps", C.c_int32),
        ("kaiser_beta", C.c_double),
        ("precision", C.c_int32),
        # abi_version >= 2
        ("speckle_tau_s", C.c_double), ("speckle_doppler_hz", C.c_double),
        ("cwm", C.c_int32),
        ("hetero_ncx", C.c_int32), ("hetero_ncy", C.c_int32),
        ("hetero_tile_m", C.c_double),
        ("hetero_u10", C.POINTER(C.c_double)), ("hetero_wind_dir_rad", C.POINTER(C.c_double)),
    ]


class harm_scene_info(C.Structure):
    _fields_ = [("n_facets", C.c_int64), ("n_pulses", C.c_int32), ("n_range", C.c_int32),
                ("n_channels", C.c_int32), ("n_waves", C.c_int32), ("precision", C.c_int32),
                ("pulse_batch", C.c_int32), ("range_bin_m", C.c_double),
                ("range_start_m", C.c_double * HARM_MAX_CHANNELS)]


# Every function the header declares, with its ctypes signature.
_VP = C.c_void_p
SIGNATURES = {
    "harm_scene_create": (C.c_int, [C.POINTER(harm_scene_desc), _VP, C.POINTER(_VP)]),
    "harm_scene_destroy": (C.c_int, [_VP]),
    "harm_scene_query": (C.c_int, [_VP, C.POINTER(harm_scene_info)]),
    "harm_scene_set_cells": (C.c_int, [_VP, C.c_int32, C.c_int32, C.c_double, _VP, _VP]),
    "harm_scene_set_pattern": (C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                         C.c_double, C.c_double, C.POINTER(C.c_double)]),
    "harm_facets_generate": (C.c_int, [_VP, C.c_int32, C.c_int32, _VP]),
    "harm_echo_accumulate": (C.c_int, [_VP, C.c_int32, C.c_int32, _VP, C.c_int, C.c_int32]),
    "harm_echo_accumulate_host": (C.c_int, [_VP, C.c_int32, C.c_int32, _VP, C.c_int, C.c_int32]),
    "harm_echo_adjoint": (C.c_int, [_VP, C.c_int32, C.c_int32, _VP, C.c_int, _VP, _VP]),
    "harm_scene_sync": (C.c_int, [_VP]),
    "harm_batch_create": (C.c_int, [C.POINTER(_VP), C.c_int32, C.POINTER(_VP)]),
    "harm_batch_tune": (C.c_int, [_VP, C.POINTER(_VP)]),
    "harm_batch_tile_rows": (C.c_int, [_VP, C.POINTER(C.c_int32)]),
    "harm_batch_set_tile_rows": (C.c_int, [_VP, C.POINTER(C.c_int32)]),
    "harm_batch_config": (C.c_int, [_VP, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "harm_batch_set_config": (C.c_int, [_VP, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int32]),
    "harm_batch_run": (C.c_int, [_VP, C.POINTER(_VP), C.c_int32]),
    "harm_batch_destroy": (C.c_int, [_VP]),
    "harm_batch_run_noalloc": (C.c_int, [C.POINTER(_VP), C.c_int32, C.POINTER(_VP), C.c_int32]),
    "harm_probe_indices": (C.c_int, [_VP, C.c_int32, C.c_int32, _VP, _VP, _VP, _VP]),
    "harm_scene_set_deterministic": (C.c_int, [_VP, C.c_int32]),
    "harm_last_error": (C.c_char_p, []),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load ``libharm.so``; raise if it is missing (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("libharm.so not built at %s (run python -m paper_2405_09938_b300.build)"
                              % path)
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def harm_last_error() -> str:
    """Message of the last non-OK status on this thread ("" if none)."""
    return load_library().harm_last_error().decode()


def _check(status):
    if status != HARM_OK:
        raise HarmError(status, harm_last_error())


def _antenna(a):
    s = harm_antenna()
    for i in range(3):
        s.pos0[i] = a["pos0"][i]
        s.vel[i] = a["vel"][i]
    s.len_az, s.len_el = a["len_az"], a["len_el"]
    return s


def make_desc(d: dict, precision: int):
    """Marshal a scene dictionary (see :mod:`harm_scenes`) into harm_scene_desc.
    Returns (desc, keepalive) -- the arrays it points to must outlive the create
    call."""
    rx = (harm_antenna * len(d["rx"]))(*[_antenna(a) for a in d["rx"]])
    keep = [rx]
    s = harm_scene_desc()
    s.abi_version = HARM_ABI_VERSION
    s.struct_size = C.sizeof(harm_scene_desc)
    s.f0_hz, s.fs_hz, s.prf_hz = d["f0_hz"], d["fs_hz"], d["prf_hz"]
    s.n_pulses, s.n_range = d["n_pulses"], d["n_range"]
    s.tx = _antenna(d["tx"])
    s.n_channels = len(d["rx"])
    s.rx = C.cast(rx, C.POINTER(harm_antenna))
    s.nx, s.ny, s.facet_m = d["nx"], d["ny"], d["facet_m"]
    s.n_omega, s.n_theta = d["n_omega"], d["n_theta"]
    s.u10, s.fetch_m, s.wind_dir_rad = d["u10"], d["fetch_m"], d["wind_dir_rad"]
    s.spread_s, s.gamma, s.wave_seed = d["spread_s"], d["gamma"], d["wave_seed"]
    s.current_u, s.current_v = d["current_u"], d["current_v"]
    s.sigma0_base, s.wind_mod = d["sigma0_base"], d["wind_mod"]
    s.epoch_pulses, s.speckle_seed = d["epoch_pulses"], d["speckle_seed"]
    s.static_surface = d["static_surface"]
    s.taps, s.kaiser_beta = d["taps"], d["kaiser_beta"]
    s.precision = precision
    s.speckle_tau_s = d.get("speckle_tau_s", 0.0)
    s.speckle_doppler_hz = d.get("speckle_doppler_hz", 0.0)
    s.cwm = int(d.get("cwm", 0))
    het = d.get("hetero")
    if het is not None:
        u = np.ascontiguousarray(het["u10"], dtype=np.float64)
        w = np.ascontiguousarray(het["wind_dir"], dtype=np.float64)
        s.hetero_ncy, s.hetero_ncx = u.shape
        s.hetero_tile_m = het["tile_m"]
        s.hetero_u10 = u.ctypes.data_as(C.POINTER(C.c_double))
        s.hetero_wind_dir_rad = w.ctypes.data_as(C.POINTER(C.c_double))
        keep += [u, w]
    return s, keep


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Scene:
    """Owning handle of a ``harm_scene``."""

    def __init__(self, ptr, desc: dict, precision: int, stream, device: int = -1):
        self._ptr = ptr
        self.desc = desc
        self.precision = precision
        self.stream = stream
        self.device = device
        self._cells = None
        self._ncells = 0

    @property
    def handle(self):
        if self._ptr is None:
            raise HarmError(HARM_E_INVALID, "scene destroyed")
        return self._ptr

    def close(self):
        if self._ptr is not None and _lib is not None:
            _lib.harm_scene_destroy(self._ptr)
        self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def harm_scene_create(desc: dict, precision: int = HARM_PREC_FP64, stream=None) -> Scene:
    """Create a scene on the current device from a scene dictionary (see
    :mod:`harm_scenes`); `stream` is a torch stream or None (default stream).
    Raises HarmError for an invalid descriptor."""
    lib = load_library()
    s, keep = make_desc(desc, precision)
    out = C.c_void_p()
    _check(lib.harm_scene_create(C.byref(s), C.c_void_p(_stream_handle(stream)), C.byref(out)))
    del keep
    import torch
    scene = Scene(out, desc, precision, stream, torch.cuda.current_device())
    # u-v gain grids listed in the descriptor dictionary ("tx" or channel index)
    for ant, pat in (desc.get("patterns") or {}).items():
        harm_scene_set_pattern(scene, -1 if ant == "tx" else int(ant), pat)
    return scene


def harm_scene_set_pattern(scene: Scene, antenna: int, pattern):
    """Set (pattern = dict with u0, du, v0, dv and a complex [nv, nu] "gain"
    array) or remove (pattern = None) the u-v gain grid of an antenna (-1 =
    transmitter, c = receive channel c)."""
    lib = load_library()
    if pattern is None:
        _check(lib.harm_scene_set_pattern(scene.handle, antenna, 0, 0, 0.0, 0.0, 0.0, 0.0, None))
        return
    g = np.asarray(pattern["gain"], dtype=np.complex128)
    if g.ndim != 2:
        raise HarmError(HARM_E_INVALID, "gain must be a 2-D [nv, nu] array")
    buf = np.ascontiguousarray(np.stack([g.real, g.imag], axis=-1))
    nv, nu = g.shape
    _check(lib.harm_scene_set_pattern(scene.handle, antenna, nu, nv, pattern["u0"], pattern["du"],
                                      pattern["v0"], pattern["dv"],
                                      buf.ctypes.data_as(C.POINTER(C.c_double))))


def harm_scene_destroy(scene: Scene):
    """Release the scene after its stream has drained."""
    scene.close()


def harm_scene_query(scene: Scene) -> dict:
    """Sizes of the scene: facets, pulses, range samples, channels, waves,
    precision, pulses per work item, range bin and per-channel range starts."""
    info = harm_scene_info()
    _check(load_library().harm_scene_query(scene.handle, C.byref(info)))
    return {"n_facets": info.n_facets, "n_pulses": info.n_pulses, "n_range": info.n_range,
            "n_channels": info.n_channels, "n_waves": info.n_waves, "precision": info.precision,
            "pulse_batch": info.pulse_batch, "range_bin_m": info.range_bin_m,
            "range_start_m": np.array(info.range_start_m[:info.n_channels])}


def _dev_ptr(t, what, size=None, dtype=None):
    """Device address of a contiguous CUDA tensor. With `size` = (scene, numel),
    also checks that the tensor holds exactly numel elements (of `dtype`, when
    given) on the scene's device: the library reads or writes that many elements
    from the address."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise HarmError(HARM_E_INVALID, "%s must be a CUDA tensor" % what)
    if not t.is_contiguous():
        raise HarmError(HARM_E_INVALID, "%s must be contiguous" % what)
    if dtype is not None and t.dtype != dtype:
        raise HarmError(HARM_E_INVALID, "%s must be %s, not %s" % (what, dtype, t.dtype))
    if size is not None:
        scene, numel = size
        if numel > 0 and t.numel() != numel:
            raise HarmError(HARM_E_INVALID, "%s holds %d elements, the call needs %d" % (what, t.numel(), numel))
        if scene.device >= 0 and t.device.index != scene.device:
            raise HarmError(HARM_E_INVALID, "%s is on cuda:%s, the scene on cuda:%d"
                            % (what, t.device.index, scene.device))
    return C.c_void_p(t.data_ptr())


def _iq_numel(scene, np_):
    return len(scene.desc["rx"]) * np_ * scene.desc["n_range"]


def _n_facets(scene):
    return scene.desc["nx"] * scene.desc["ny"]


def harm_scene_set_cells(scene: Scene, ncx, ncy, cell_m, sigma0=None, uv=None):
    """Per-cell NRCS base (float64 CUDA tensor [ncy, ncx]) and current
    ([ncy, ncx, 2]) on cells of cell_m metres; either may be None. The tensors are
    kept alive with the scene."""
    import torch
    nce = int(ncx) * int(ncy)
    sp = _dev_ptr(sigma0, "sigma0", (scene, nce), torch.float64) if sigma0 is not None else None
    up = _dev_ptr(uv, "uv", (scene, 2 * nce), torch.float64) if uv is not None else None
    _check(load_library().harm_scene_set_cells(scene.handle, ncx, ncy, cell_m, sp, up))
    scene._cells = (sigma0, uv)
    scene._ncells = nce


def harm_facets_generate(scene: Scene, n0: int, np_: int, state):
    """Facet states of pulses [n0, n0 + np_) into `state`, a CUDA tensor
    [np_][F][n_facets] (float64 for FP64 scenes, float32 for mixed; F = 3, or 8
    with the Choppy Wave Model)."""
    import torch
    nfield = 8 if scene.desc.get("cwm") else 3
    dt = torch.float64 if scene.precision == HARM_PREC_FP64 else torch.float32
    _dev_ptr(state, "state")
    ptr = _dev_ptr(state, "state", (scene, np_ * nfield * _n_facets(scene)), dt)
    _check(load_library().harm_facets_generate(scene.handle, n0, np_, ptr))


def _dtype_code(t):
    import torch
    if t.dtype == torch.complex64:
        return HARM_C64
    if t.dtype == torch.complex128:
        return HARM_C128
    raise HarmError(HARM_E_INVALID, "IQ tensors must be complex64 or complex128")


def harm_echo_accumulate(scene: Scene, n0: int, np_: int, iq, zero_first: bool = True):
    """Add the echo of pulses [n0, n0 + np_) into `iq`, a contiguous CUDA tensor
    [n_channels][np_][n_range] (complex64 or complex128), cleared first unless
    zero_first is False. Asynchronous on the scene's stream."""
    _dev_ptr(iq, "iq")
    ptr = _dev_ptr(iq, "iq", (scene, _iq_numel(scene, np_)))
    _check(load_library().harm_echo_accumulate(scene.handle, n0, np_, ptr, _dtype_code(iq),
                                               1 if zero_first else 0))


def harm_scene_set_deterministic(scene: Scene, on: bool = True):
    """Deterministic (bit-reproducible) fixed-point sums for a plain-path scene
    (FP64 or FP32); needs complex128 IQ outputs."""
    _check(load_library().harm_scene_set_deterministic(scene.handle, 1 if on else 0))


def harm_echo_accumulate_host(scene: Scene, n0: int, np_: int, iq_host, block_pulses: int = 0):
    """Echo of pulses [n0, n0 + np_) written to ``iq_host``, a contiguous pinned CPU
    tensor [n_channels][np_][n_range] (complex64 or complex128); complete after
    :func:`harm_scene_sync`."""
    import torch
    if not isinstance(iq_host, torch.Tensor) or iq_host.is_cuda:
        raise HarmError(HARM_E_INVALID, "iq_host must be a CPU tensor")
    if not iq_host.is_contiguous():
        raise HarmError(HARM_E_INVALID, "iq_host must be contiguous")
    if np_ > 0 and iq_host.numel() != _iq_numel(scene, np_):
        raise HarmError(HARM_E_INVALID, "iq_host holds %d elements, the call needs %d"
                        % (iq_host.numel(), _iq_numel(scene, np_)))
    _check(load_library().harm_echo_accumulate_host(scene.handle, n0, np_, C.c_void_p(iq_host.data_ptr()),
                                                    _dtype_code(iq_host), block_pulses))


def harm_echo_adjoint(scene: Scene, n0: int, np_: int, resid, grad_sigma0=None, grad_uv=None):
    """Add the gradients of sum |IQ - target|^2 for the residual `resid` (IQ -
    target, same layout and dtype as the IQ) to grad_sigma0 [ncy, ncx] and grad_uv
    [ncy, ncx, 2] (float64 CUDA tensors, either may be None). Needs cells."""
    import torch
    _dev_ptr(resid, "resid")
    rp = _dev_ptr(resid, "resid", (scene, _iq_numel(scene, np_)))
    nce = scene._ncells
    if nce == 0 and (grad_sigma0 is not None or grad_uv is not None):
        raise HarmError(HARM_E_INVALID, "the adjoint needs per-cell fields (harm_scene_set_cells)")
    gs = _dev_ptr(grad_sigma0, "grad_sigma0", (scene, nce), torch.float64) if grad_sigma0 is not None else None
    gu = _dev_ptr(grad_uv, "grad_uv", (scene, 2 * nce), torch.float64) if grad_uv is not None else None
    _check(load_library().harm_echo_adjoint(scene.handle, n0, np_, rp, _dtype_code(resid), gs, gu))


def harm_probe_indices(scene: Scene, n0: int, np_: int):
    """Integer work of the accumulator for pulses [n0, n0 + np_) (see
    include/harm.h): returns CUDA tensors bins [np_, n_channels, ny, nx] int32,
    speckle [np_, ny, nx] (complex128 for FP64 scenes, complex64 otherwise),
    words [np_, ny, nx, 4] int32 (the uint32 Philox words, reinterpreted) and
    cells [ny, nx] int32."""
    import torch
    d = scene.desc
    nc, nx, ny = len(d["rx"]), d["nx"], d["ny"]
    dev = torch.device("cuda", scene.device)
    bins = torch.empty((np_, nc, ny, nx), dtype=torch.int32, device=dev)
    sdt = torch.complex128 if scene.precision == HARM_PREC_FP64 else torch.complex64
    spk = torch.empty((np_, ny, nx), dtype=sdt, device=dev)
    words = torch.empty((np_, ny, nx, 4), dtype=torch.int32, device=dev)
    cells = torch.empty((ny, nx), dtype=torch.int32, device=dev)
    _check(load_library().harm_probe_indices(scene.handle, n0, np_, C.c_void_p(bins.data_ptr()),
                                             C.c_void_p(spk.data_ptr()), C.c_void_p(words.data_ptr()),
                                             C.c_void_p(cells.data_ptr())))
    return bins, spk, words, cells


def harm_scene_sync(scene: Scene):
    """Wait for the scene's stream; raises HarmError for device-side errors."""
    _check(load_library().harm_scene_sync(scene.handle))


class Batch:
    """Owning handle of a ``harm_batch`` (keeps its scenes alive)."""

    def __init__(self, ptr, scenes):
        self._ptr = ptr
        self.scenes = list(scenes)

    @property
    def handle(self):
        if self._ptr is None:
            raise HarmError(HARM_E_INVALID, "batch destroyed")
        return self._ptr

    def close(self):
        if self._ptr is not None and _lib is not None:
            _lib.harm_batch_destroy(self._ptr)
        self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr_array(tensors, what, scenes):
    """Pointer array of one complex64 IQ tensor per scene, each checked to hold the
    scene's whole burst [n_channels][n_pulses][n_range] on the scene's device."""
    import torch
    if len(tensors) != len(scenes):
        raise HarmError(HARM_E_INVALID, "%d %s tensors for %d scenes" % (len(tensors), what, len(scenes)))
    arr = (C.c_void_p * len(tensors))()
    for i, (t, sc) in enumerate(zip(tensors, scenes)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.complex64:
            raise HarmError(HARM_E_INVALID, "%s[%d] must be a complex64 CUDA tensor" % (what, i))
        arr[i] = _dev_ptr(t, "%s[%d]" % (what, i), (sc, _iq_numel(sc, sc.desc["n_pulses"]))).value
    return arr


def harm_batch_create(scenes) -> Batch:
    """Group mixed-precision scenes (same device, channels and taps) into one
    persistent batched launch."""
    arr = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    out = C.c_void_p()
    _check(load_library().harm_batch_create(arr, len(scenes), C.byref(out)))
    return Batch(out, scenes)


def harm_batch_tune(batch: Batch, iqs):
    """Pick the launch shape (tile rows and time-Taylor window per scene-size
    class, CTAs per SM) by timing, or from the choices already made in this
    process for batches of the same kind; overwrites the complex64 CUDA tensors
    `iqs` (one per scene). Synchronous."""
    _check(load_library().harm_batch_tune(batch.handle, _ptr_array(iqs, "iq", batch.scenes)))


def harm_batch_tile_rows(batch: Batch):
    """Tile height (8 or 16 facet rows) of each scene."""
    rows = (C.c_int32 * len(batch.scenes))()
    _check(load_library().harm_batch_tile_rows(batch.handle, rows))
    return [int(v) for v in rows]


def harm_batch_set_tile_rows(batch: Batch, rows):
    """Pin the tile height (8 or 16) of each scene instead of tuning."""
    arr = (C.c_int32 * len(batch.scenes))(*[int(r) for r in rows])
    _check(load_library().harm_batch_set_tile_rows(batch.handle, arr))


def harm_batch_config(batch: Batch):
    """Launch shape in use: {"rows": [...], "windows": [...], "ctas_per_sm": c}."""
    n = len(batch.scenes)
    rows, wins, cps = (C.c_int32 * n)(), (C.c_int32 * n)(), C.c_int32()
    _check(load_library().harm_batch_config(batch.handle, rows, wins, C.byref(cps)))
    return {"rows": [int(v) for v in rows], "windows": [int(v) for v in wins], "ctas_per_sm": int(cps.value)}


def harm_batch_set_config(batch: Batch, rows, windows, ctas_per_sm: int):
    """Pin the launch shape: rows 8 or 16 and windows (a scene's pulse_batch or
    half of it) per scene, ctas_per_sm 1 or 2."""
    n = len(batch.scenes)
    r = (C.c_int32 * n)(*[int(v) for v in rows])
    w = (C.c_int32 * n)(*[int(v) for v in windows])
    _check(load_library().harm_batch_set_config(batch.handle, r, w, int(ctas_per_sm)))


def harm_batch_run(batch: Batch, iqs, zero_first: bool = True):
    """Echo of every scene over its burst into `iqs` (complex64 CUDA tensors, one
    per scene), replayed from a CUDA graph."""
    outs = _ptr_array(iqs, "iq", batch.scenes)
    _check(load_library().harm_batch_run(batch.handle, outs, 1 if zero_first else 0))


def harm_batch_destroy(batch: Batch):
    """Release the batch (its scenes stay valid)."""
    batch.close()


def harm_batch_run_noalloc(scenes, iqs, zero_first: bool = True):
    """Allocation-free batched run (see include/harm.h): scratch in a fixed device
    array, at most 64 scenes per call, calls must not overlap on the GPU."""
    outs = _ptr_array(iqs, "iq", scenes)
    arr = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    _check(load_library().harm_batch_run_noalloc(arr, len(scenes), outs,
                                                 1 if zero_first else 0))
