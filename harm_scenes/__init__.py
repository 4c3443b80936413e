"""Seeded synthetic scene descriptors shared by the CUDA path, the oracle and the bench.

This module only *describes* inputs: instrument geometry, acquisition parameters and
sea-state parameters as plain numbers. It holds none of the echo model's arithmetic
(no ranges, patterns, spectra, phases or range spreading); each side turns a
descriptor into its own data structures.

Frame (flat-earth, local): x along-track (platform velocity +x), y ground range away
from the radars, z up, origin at the scene centre on the mean surface. Antenna phase
centres move linearly, P(t) = pos0 + vel * t, with t = 0 at the first pulse.

Workloads follow the instrument of the paper's Sec. II-B / Fig. 1 (Sentinel-1
transmitter, two Harmony receivers about 250 km ahead and behind, three along-track
phase centres each) and the raw-data generator of Sec. IV, on 2 m facets: a 200 m
static patch (100 x 100 facets, 64 pulses, 1 channel, 512 range samples; the small
case), a 4 km x 2 km wave-covered ATI scene (2000 x 1000 facets, 2048 pulses,
6 channels, 4096 range samples; the headline case), a 20 km x 5 km mixed-precision
scene (10000 x 2500 facets, 4096 pulses, 3 channels), a 2 km x 1 km differentiable
scene (1000 x 500 facets, 1024 pulses, 6 channels, 100 m cells), and a batch of 48
uneven scenes (0.5 x 0.5 km to 8 x 4 km, 256 to 2048 pulses, 1024 to 8192 range
samples).
"""
from __future__ import annotations

import copy
import math

import numpy as np

C_LIGHT = 299792458.0

# Instrument constants (Sentinel-1 C-band, Harmony companions).
F0_HZ = 5.405e9
FS_HZ = 64e6
PRF_HZ = 1700.0
ALTITUDE_M = 693e3
INCIDENCE_DEG = 35.0
V_PLATFORM = 7500.0
HARMONY_OFFSET_M = 250e3
PHASE_CENTRE_SPACING_M = 5.0
TX_LEN = (12.3, 0.82)
RX_LEN = (4.0, 0.82)


def _antenna(x0, y0, z0, length):
    return {"pos0": [float(x0), float(y0), float(z0)],
            "vel": [V_PLATFORM, 0.0, 0.0],
            "len_az": float(length[0]), "len_el": float(length[1])}


def geometry(n_pulses: int, sats=("A",), phase_centres=(0.0,), prf=PRF_HZ):
    """Transmitter + receivers for a burst of ``n_pulses`` pulses.

    The transmitter is at broadside of the scene centre at mid-burst; receivers
    ride the same (y, z) track, Harmony A ahead (+x) and Harmony B behind (-x),
    each with along-track phase centres at the given offsets.
    """
    t_mid = (n_pulses - 1) / (2.0 * prf)
    y_t = -ALTITUDE_M * math.tan(math.radians(INCIDENCE_DEG))
    x_mid = -V_PLATFORM * t_mid
    tx = _antenna(x_mid, y_t, ALTITUDE_M, TX_LEN)
    rx = []
    for sat in sats:
        off = HARMONY_OFFSET_M if sat == "A" else -HARMONY_OFFSET_M
        for pc in phase_centres:
            rx.append(_antenna(x_mid + off + pc, y_t, ALTITUDE_M, RX_LEN))
    return tx, rx


def _base(n_pulses, n_range, sats, pcs, nx, ny):
    tx, rx = geometry(n_pulses, sats, pcs)
    return {
        "f0_hz": F0_HZ, "fs_hz": FS_HZ, "prf_hz": PRF_HZ,
        "n_pulses": int(n_pulses), "n_range": int(n_range),
        "tx": tx, "rx": rx,
        "nx": int(nx), "ny": int(ny), "facet_m": 2.0,
        "n_omega": 0, "n_theta": 0,
        "u10": 8.0, "fetch_m": 100e3, "wind_dir_rad": math.radians(45.0),
        "spread_s": 4.0, "gamma": 3.3, "wave_seed": 7,
        "current_u": 0.0, "current_v": 0.0,
        "sigma0_base": 0.05, "wind_mod": 0.0,
        "epoch_pulses": 0, "speckle_seed": 1,
        "static_surface": 1,
        "taps": 8, "kaiser_beta": 6.0,
        "cells": None,
    }


def small_static(n_pulses=64):
    """200 m x 200 m static patch, 1 receive channel (Harmony A, centre phase
    centre), 64 pulses, 512 range samples, 8-tap Kaiser(6) sinc."""
    return _base(n_pulses, 512, ("A",), (0.0,), 100, 100)


def ati_scene(n_pulses=2048, nx=2000, ny=1000, n_range=4096):
    """4 km x 2 km wave-covered ATI scene: Tx + Harmony A/B x 3 phase centres
    (6 channels), 256 linear wave components (16 x 16 JONSWAP grid, U10 8 m/s,
    fetch 100 km, cos^2s spreading s = 4, wind toward 45 deg), uniform current
    (0.5, 0.2) m/s, NRCS 0.02 (1 + 0.5 cos phi_wind) x tilt, speckle redrawn every
    20 ms epoch (34 pulses at 1700 Hz), 2048 pulses x 4096 range samples."""
    pcs = (-PHASE_CENTRE_SPACING_M, 0.0, PHASE_CENTRE_SPACING_M)
    d = _base(n_pulses, n_range, ("A", "B"), pcs, nx, ny)
    d.update({
        "n_omega": 16, "n_theta": 16,
        "current_u": 0.5, "current_v": 0.2,
        "sigma0_base": 0.02, "wind_mod": 0.5,
        "epoch_pulses": 34, "static_surface": 0,
    })
    return d


def mixed_scene(n_pulses=4096, nx=10000, ny=2500):
    """20 km x 5 km scene, Tx + Harmony A x 3 phase centres, 4096 pulses."""
    pcs = (-PHASE_CENTRE_SPACING_M, 0.0, PHASE_CENTRE_SPACING_M)
    d = ati_scene(n_pulses=n_pulses, nx=nx, ny=ny, n_range=4096)
    tx, rx = geometry(n_pulses, ("A",), pcs)
    d["tx"], d["rx"] = tx, rx
    return d


def adjoint_scene(n_pulses=1024, nx=1000, ny=500):
    """2 km x 1 km scene, 6 channels, 1024 pulses, with per-cell NRCS and
    current on 100 m cells (20 x 10 cells)."""
    d = ati_scene(n_pulses=n_pulses, nx=nx, ny=ny, n_range=4096)
    ncx = int(round(nx * d["facet_m"] / 100.0))
    ncy = int(round(ny * d["facet_m"] / 100.0))
    d["cells"] = {
        "ncx": ncx, "ncy": ncy, "cell_m": 100.0,
        "sigma0": np.full((ncy, ncx), 0.02, dtype=np.float64),
        "uv": np.tile(np.array([0.5, 0.2], dtype=np.float64), (ncy, ncx, 1)),
    }
    return d


def current_perturbation(ncx=20, ncy=10, cell_m=100.0, std=0.1, length_m=500.0,
                         seed=23):
    """Gaussian-correlated (u, v) perturbation per cell: covariance
    std^2 exp(-d^2 / (2 l^2)) between cell centres, drawn by Cholesky factor of the
    covariance (+1e-10 jitter) applied to standard normals from numpy's Philox
    generator with the given seed. Returns an array [ncy, ncx, 2]."""
    yy, xx = np.meshgrid((np.arange(ncy) + 0.5) * cell_m, (np.arange(ncx) + 0.5) * cell_m,
                         indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel()], axis=1)
    d2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    cov = std * std * np.exp(-d2 / (2.0 * length_m * length_m))
    cov += 1e-10 * np.eye(len(pts))
    L = np.linalg.cholesky(cov)
    rng = np.random.Generator(np.random.Philox(seed))
    w = rng.standard_normal((2, len(pts)))
    du = L @ w[0]
    dv = L @ w[1]
    return np.stack([du.reshape(ncy, ncx), dv.reshape(ncy, ncx)], axis=-1)


def batch_scenes(n_scenes=48, seed=11):
    """Uneven batch: per scene, uniforms from numpy's Philox generator (seed 11)
    set the patch (0.5 km .. 8 km along-track, half that across, at least 0.5 km),
    the burst (256 .. 2048 pulses), the range window (1024 .. 8192 samples), U10
    (3 .. 15 m/s) and wind direction (0 .. 360 deg). 6 channels, complex64."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for s in range(n_scenes):
        u = rng.random(5)
        lx = 500.0 * 16.0 ** u[0]
        ly = max(500.0, lx / 2.0)
        nx = int(round(lx / 2.0))
        ny = int(round(ly / 2.0))
        n_p = 256 * 2 ** int(math.floor(4 * u[1]))
        n_r = 1024 * 2 ** int(math.floor(4 * u[2]))
        d = ati_scene(n_pulses=n_p, nx=nx, ny=ny, n_range=n_r)
        d["u10"] = 3.0 + 12.0 * u[3]
        d["wind_dir_rad"] = 2.0 * math.pi * u[4]
        d["speckle_seed"] = 1000 + s
        out.append(d)
    return out


# ---------------------------------------------------------------------------
# Variants of the surface and scattering model (Sec. III): each takes a
# descriptor and returns a copy with the variant switched on.
# ---------------------------------------------------------------------------
def ar1_speckle(desc, tau_s=0.05, doppler_hz=12.0, epoch_pulses=8):
    """Order-1 autoregressive speckle (Eq. 10) with correlation time tau_s,
    updated every epoch of ``epoch_pulses`` pulses, and a uniform intra-facet
    Doppler shift f_s (Eq. 7)."""
    d = copy.deepcopy(desc)
    d.update({"speckle_tau_s": float(tau_s), "speckle_doppler_hz": float(doppler_hz),
              "epoch_pulses": int(epoch_pulses)})
    return d


def choppy(desc):
    """Choppy Wave Model on: facets follow the waves' orbital motion horizontally."""
    d = copy.deepcopy(desc)
    d["cwm"] = 1
    return d


def hetero_sea(desc, tile_m=512.0, u10=(6.0, 12.0), wind_dir_deg=(20.0, 80.0)):
    """Heterogeneous sea state (Eq. 1, 2): TL tiles of ``tile_m`` from the patch
    corner, with a corner grid just covering the patch. The corner spectra vary
    smoothly: wind speed ramps linearly along x over ``u10``, wind direction
    along y over ``wind_dir_deg``."""
    d = copy.deepcopy(desc)
    lx, ly = d["nx"] * d["facet_m"], d["ny"] * d["facet_m"]
    ncx = int(math.ceil(lx / tile_m - 1e-9)) + 1
    ncy = int(math.ceil(ly / tile_m - 1e-9)) + 1
    ax = np.linspace(0.0, 1.0, ncx)
    ay = np.linspace(0.0, 1.0, ncy)
    u = u10[0] + (u10[1] - u10[0]) * np.tile(ax, (ncy, 1))
    w = np.radians(wind_dir_deg[0] + (wind_dir_deg[1] - wind_dir_deg[0]) * np.tile(ay[:, None], (1, ncx)))
    d["hetero"] = {"tile_m": float(tile_m), "u10": u, "wind_dir": w}
    return d


def phased_array_gain(len_az, len_el, seed, nu=161, nv=81, u_span=0.02, v_span=0.02,
                      tiles=(14, 4), amp_err_db=0.5, phase_err_deg=5.0):
    """Complex u-v gain grid of a planar phased array (the form in which the
    antenna patterns reach the simulator, Sec. III-B): the aperture
    len_az x len_el split into tiles[0] x tiles[1] sub-arrays, each with a
    uniform field sinc(L_t u / lambda) sinc(H_t v / lambda) and a random complex
    excitation error (amplitude ``amp_err_db`` rms in dB, phase
    ``phase_err_deg`` rms) from numpy's Philox generator; normalised to unit
    gain at boresight of the error-free array. Grid: nu x nv nodes over
    [-u_span/2, u_span/2] x [-v_span/2, v_span/2] (direction cosines along the
    azimuth and elevation axes). Returns the pattern dict of a descriptor."""
    lam = C_LIGHT / F0_HZ
    rng = np.random.Generator(np.random.Philox(seed))
    mt, nt = tiles
    lt, ht = len_az / mt, len_el / nt
    xt = (np.arange(mt) + 0.5 - 0.5 * mt) * lt
    zt = (np.arange(nt) + 0.5 - 0.5 * nt) * ht
    err = (10.0 ** (amp_err_db / 20.0 * rng.standard_normal((nt, mt)))
           * np.exp(1j * np.radians(phase_err_deg) * rng.standard_normal((nt, mt))))
    u = np.linspace(-0.5 * u_span, 0.5 * u_span, nu)
    v = np.linspace(-0.5 * v_span, 0.5 * v_span, nv)
    k = 2.0 * math.pi / lam
    ex = np.exp(1j * k * np.outer(u, xt))  # [nu, mt]
    ez = np.exp(1j * k * np.outer(v, zt))  # [nv, nt]
    af = np.einsum("vn,nm,um->vu", ez, err, ex)  # [nv, nu]
    elem = np.outer(np.sinc(ht * v / lam), np.sinc(lt * u / lam))
    g = af * elem / (mt * nt)
    return {"u0": float(u[0]), "du": float(u[1] - u[0]), "v0": float(v[0]), "dv": float(v[1] - v[0]),
            "gain": g}


def uv_patterns(desc, seed=31):
    """u-v gain grids for the transmitter and every receive channel (phase
    centres of one satellite share their array but not its errors)."""
    d = copy.deepcopy(desc)
    pats = {"tx": phased_array_gain(d["tx"]["len_az"], d["tx"]["len_el"], seed)}
    for c, a in enumerate(d["rx"]):
        pats[c] = phased_array_gain(a["len_az"], a["len_el"], seed + 1 + c)
    d["patterns"] = pats
    return d


def with_overrides(desc, **kw):
    d = copy.deepcopy(desc)
    d.update(kw)
    return d


def n_facets(desc):
    return int(desc["nx"]) * int(desc["ny"])


def n_contributions(desc, n_pulses=None):
    npul = desc["n_pulses"] if n_pulses is None else n_pulses
    return n_facets(desc) * int(npul) * len(desc["rx"])
