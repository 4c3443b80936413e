"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here compares the oracle with something other than itself: a library
routine (cuRAND's host Philox generator, scipy / numpy special functions and
quadrature), a closed form (point-target delay and phase, bistatic Doppler, the
Pierson-Moskowitz integral, sinc nulls, specular tilt), an invariant (linearity,
light-time residuals, orthonormal frames) or a brute-force sum on a small scene.
"""
import ctypes
import math
import os

import mpmath as mp
import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as ss
import scipy.stats as st

import harm_scenes as hs
import oracle
from tests import _kinematics as kin

C_LIGHT = 299792458.0
G = 9.80665


# ---------------------------------------------------------------------------
# Philox4x32-10 against cuRAND's host generator (a library routine).
# cuRAND's host PHILOX4_32_10 stream puts output block b at counter
# (b // 65536, 0, b % 65536, 0) with key (seed_lo, seed_hi).
# ---------------------------------------------------------------------------
def _curand():
    for p in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    pytest.skip("libcurand not available")


def _curand_blocks(seed, block0, nblocks):
    cr = _curand()
    g = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(g), 161) == 0  # PHILOX4_32_10
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert cr.curandSetGeneratorOffset(g, ctypes.c_ulonglong(4 * block0)) == 0
        out = np.zeros(4 * nblocks, dtype=np.uint32)
        assert cr.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.c_size_t(out.size)) == 0
    finally:
        cr.curandDestroyGenerator(g)
    return out.reshape(nblocks, 4)


@pytest.mark.parametrize("seed", [0, 1, 7, 23, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand(seed):
    # word 2 (the speckle epoch) spans a run of consecutive blocks
    blocks = _curand_blocks(seed, 0, 300)
    for b in list(range(0, 300, 7)) + [299]:
        ref = oracle.philox4x32_10([0, 0, b, 0], [seed & 0xFFFFFFFF, seed >> 32])
        assert ref == [int(v) for v in blocks[b]]
    # word 0 (the facet id) via the generator offset
    for w0, w2 in [(1, 0), (5, 3), (123457, 61), (2**32 - 1, 120), (25_000_000, 7)]:
        blk = _curand_blocks(seed, w0 * 65536 + w2, 1)[0]
        ref = oracle.philox4x32_10([w0, 0, w2, 0], [seed & 0xFFFFFFFF, seed >> 32])
        assert ref == [int(v) for v in blk]


def test_wave_phases_are_the_wave_stream():
    d = hs.ati_scene()
    tab = oracle.wave_table(d)
    seed = d["wave_seed"] ^ (0x57415645 << 32)
    blocks = _curand_blocks(seed, 0, 1)  # counter (0,0,0,0)
    assert math.isclose(tab["phase"][0], 2 * math.pi * blocks[0][0] / 2**32, rel_tol=0,
                        abs_tol=1e-15)
    for m in (1, 17, 255):
        blk = _curand_blocks(seed, m * 65536, 1)[0]  # counter (m, 0, 0, 0)
        assert math.isclose(tab["phase"][m], 2 * math.pi * blk[0] / 2**32, abs_tol=1e-14)


# ---------------------------------------------------------------------------
# Speckle: R, I ~ N(0, 1/2), <s s*> = 1 (Sec. III-A, after Eq. 8)
# ---------------------------------------------------------------------------
def test_speckle_statistics():
    n = 40000
    z = np.array([oracle.speckle(1, f, 3) for f in range(n)])
    se = 1.0 / math.sqrt(n)
    assert abs(z.real.mean()) < 5 * se * math.sqrt(0.5)
    assert abs(z.imag.mean()) < 5 * se * math.sqrt(0.5)
    p2 = np.abs(z) ** 2
    assert abs(p2.mean() - 1.0) < 5 * se  # |z|^2 ~ Exp(1): sd 1
    assert abs((z.real ** 2).mean() - 0.5) < 5 * se * math.sqrt(0.5)
    assert abs((z.imag ** 2).mean() - 0.5) < 5 * se * math.sqrt(0.5)
    assert abs(np.mean(z.real * z.imag)) < 5 * se * 0.5
    assert st.kstest(z.real, st.norm(0, math.sqrt(0.5)).cdf).pvalue > 1e-3
    assert st.kstest(z.imag, st.norm(0, math.sqrt(0.5)).cdf).pvalue > 1e-3
    assert st.kstest(p2, st.expon().cdf).pvalue > 1e-3


def test_speckle_epochs_independent():
    n = 20000
    a = np.array([oracle.speckle(1, f, 0) for f in range(n)])
    b = np.array([oracle.speckle(1, f, 1) for f in range(n)])
    corr = np.abs(np.vdot(a, b)) / n
    assert corr < 5 / math.sqrt(n)
    # same (f, e) -> same draw
    assert oracle.speckle(1, 77, 5) == oracle.speckle(1, 77, 5)


# ---------------------------------------------------------------------------
# Kaiser-windowed sinc interpolation (replaces the Eq. 17 box)
# ---------------------------------------------------------------------------
def test_bessel_i0_matches_scipy():
    for x in [0.0, 1e-3, 0.5, 1.0, 2.5, 4.0, 6.0, 7.3]:
        assert math.isclose(oracle.bessel_i0(x), float(ss.i0(x)), rel_tol=2e-15)
    assert abs(oracle.bessel_i0(6.0) - 67.234407) < 1e-6


def test_kaiser_sinc_matches_numpy():
    beta, m = 6.0, 4
    M = 17
    win = np.kaiser(M, beta)
    for nidx in range(M):
        x = m * (2.0 * nidx / (M - 1) - 1.0)
        if abs(x) >= m:
            assert oracle.kaiser_sinc(x, m, beta) == 0.0
            continue
        ref = np.sinc(x) * win[nidx]
        assert math.isclose(oracle.kaiser_sinc(x, m, beta), ref, rel_tol=1e-13, abs_tol=1e-16)
    rng = np.random.default_rng(3)
    for x in rng.uniform(-4, 4, 50):
        ref = np.sinc(x) * ss.i0(beta * math.sqrt(1 - (x / m) ** 2)) / ss.i0(beta)
        assert math.isclose(oracle.kaiser_sinc(x, m, beta), ref, rel_tol=1e-13, abs_tol=1e-16)


def test_kaiser_sinc_special_values():
    assert oracle.kaiser_sinc(0.0, 4, 6.0) == 1.0
    for k in (1, 2, 3):
        assert abs(oracle.kaiser_sinc(float(k), 4, 6.0)) < 1e-16
        assert abs(oracle.kaiser_sinc(-float(k), 4, 6.0)) < 1e-16
    assert oracle.kaiser_sinc(4.0, 4, 6.0) == 0.0
    assert oracle.kaiser_sinc(-4.5, 4, 6.0) == 0.0


# ---------------------------------------------------------------------------
# Sea state
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("s", [1.0, 2.5, 4.0, 8.0])
def test_spreading_normalised(s):
    val, _ = si.quad(lambda th: oracle.spreading(th, s), -math.pi, math.pi, epsabs=1e-13)
    assert abs(val - 1.0) < 1e-10


def test_spreading_grid_sum_exact():
    # cos^8(theta/2) is a trig polynomial of degree 4; the 16-point midpoint rule
    # integrates it exactly.
    d = hs.ati_scene()
    nt = d["n_theta"]
    dth = 2 * math.pi / nt
    tot = sum(oracle.spreading(-math.pi + (j + 0.5) * dth, d["spread_s"]) * dth for j in range(nt))
    assert abs(tot - 1.0) < 1e-13


def test_pierson_moskowitz_integral():
    # gamma = 1: integral of alpha g^2 w^-5 exp(-5/4 (wp/w)^4) over (0, inf) is
    # alpha g^2 / (5 wp^4).
    u10, fetch = 8.0, 100e3
    wp, alpha = oracle.jonswap_params(u10, fetch)
    val, _ = si.quad(lambda w: oracle.jonswap(w, u10, fetch, 1.0), 0.05, 50.0, limit=400,
                     epsrel=1e-12)
    tail, _ = si.quad(lambda w: oracle.jonswap(w, u10, fetch, 1.0), 50.0, np.inf)
    assert math.isclose(val + tail, alpha * G * G / (5 * wp ** 4), rel_tol=1e-8)


def test_jonswap_peak_and_enhancement():
    u10, fetch, gamma = 8.0, 100e3, 3.3
    wp, alpha = oracle.jonswap_params(u10, fetch)
    # fetch laws at U10 = 8 m/s, F = 100 km
    assert abs(wp - 1.0858) < 5e-4
    assert abs(alpha - 0.00912) < 5e-5
    ratio = oracle.jonswap(wp, u10, fetch, gamma) / oracle.jonswap(wp, u10, fetch, 1.0)
    assert math.isclose(ratio, gamma, rel_tol=1e-13)
    w = np.linspace(0.8 * wp, 1.2 * wp, 4001)
    s = np.array([oracle.jonswap(x, u10, fetch, gamma) for x in w])
    assert abs(w[np.argmax(s)] - wp) < 2e-4 * wp


def test_wave_table_energy_and_dispersion():
    d = hs.ati_scene()
    tab = oracle.wave_table(d)
    wp, _ = oracle.jonswap_params(d["u10"], d["fetch_m"])
    m0, _ = si.quad(lambda w: oracle.jonswap(w, d["u10"], d["fetch_m"], d["gamma"]),
                    0.7 * wp, 2.5 * wp, limit=200)
    assert abs((tab["amp"] ** 2 / 2).sum() / m0 - 1.0) < 0.02
    k = np.hypot(tab["kx"], tab["ky"])
    assert np.allclose(tab["omega"] ** 2, G * k, rtol=1e-13)
    th = np.arctan2(tab["ky"], tab["kx"])
    nt = d["n_theta"]
    for m in range(len(th)):
        j = m % nt
        want = d["wind_dir_rad"] - math.pi + (j + 0.5) * 2 * math.pi / nt
        assert abs(kin.wrap(th[m] - want)) < 1e-12
    assert np.all((tab["phase"] >= 0) & (tab["phase"] < 2 * math.pi))
    # significant wave height from the grid
    assert abs(4 * math.sqrt((tab["amp"] ** 2 / 2).sum()) - 1.75) < 0.05


def test_surface_slopes_are_gradients():
    tab = oracle.wave_table(hs.ati_scene())
    h = 1e-3
    rng = np.random.default_rng(0)
    for x, y, t in zip(rng.uniform(-2000, 2000, 5), rng.uniform(-1000, 1000, 5),
                       rng.uniform(0, 1.2, 5)):
        s = oracle.surface(tab, x, y, t)
        ex = (oracle.surface(tab, x + h, y, t)[0] - oracle.surface(tab, x - h, y, t)[0]) / (2 * h)
        ey = (oracle.surface(tab, x, y + h, t)[0] - oracle.surface(tab, x, y - h, t)[0]) / (2 * h)
        assert abs(ex - s[1]) < 1e-8
        assert abs(ey - s[2]) < 1e-8


def test_surface_variance_matches_spectrum():
    tab = oracle.wave_table(hs.ati_scene())
    rng = np.random.default_rng(1)
    pts = rng.uniform(-20000, 20000, (3000, 2))
    eta = np.array([oracle.surface(tab, x, y, 0.3)[0] for x, y in pts])
    m0 = (tab["amp"] ** 2 / 2).sum()
    assert abs(eta.var() / m0 - 1) < 0.1
    assert abs(eta.mean()) < 0.05


def test_surface_precision_vs_mpmath():
    tab = oracle.wave_table(hs.ati_scene())
    x, y, t = 1733.0, -911.0, 1.07
    s = oracle.surface(tab, x, y, t)
    eta = mp.mpf(0)
    for m in range(len(tab["kx"])):
        arg = (mp.mpf(tab["kx"][m]) * x + mp.mpf(tab["ky"][m]) * y - mp.mpf(tab["omega"][m]) * t
               + mp.mpf(tab["phase"][m]))
        eta += mp.mpf(tab["amp"][m]) * mp.cos(arg)
    assert abs(s[0] - float(eta)) < 1e-12


# ---------------------------------------------------------------------------
# Geometry: light time, antenna frames, patterns, NRCS
# ---------------------------------------------------------------------------
def test_light_time_residuals():
    d = hs.ati_scene(n_pulses=2048, nx=10, ny=10)
    for n in (0, 1023, 2047):
        for c in range(len(d["rx"])):
            g = oracle.pulse_state(d, n, c)
            assert abs((g["ts"] - g["t"]) * C_LIGHT - g["rt_ref"]) < 1e-6
            assert abs((g["trx"] - g["ts"]) * C_LIGHT - g["rr_ref"]) < 1e-6
            ref = kin.pulse(d, n, c)
            assert abs(float(ref["rr"]) - g["rr_ref"]) < 1e-8
            assert abs(float(ref["rt"]) - g["rt_ref"]) < 1e-8


def test_antenna_frames_orthonormal():
    d = hs.ati_scene(nx=10, ny=10)
    for c in range(len(d["rx"])):
        g = oracle.pulse_state(d, 100, c)
        for p, a, e, vel in ((g["ptx"], g["atx"], g["etx"], d["tx"]["vel"]),
                             (g["prx"], g["arx"], g["erx"], d["rx"][c]["vel"])):
            b = -p / np.linalg.norm(p)
            assert abs(np.dot(a, b)) < 1e-14 and abs(np.dot(e, b)) < 1e-14
            assert abs(np.dot(a, e)) < 1e-14
            assert abs(np.linalg.norm(a) - 1) < 1e-14 and abs(np.linalg.norm(e) - 1) < 1e-14
            assert np.allclose(np.cross(b, a), e, atol=1e-14)
            assert np.dot(a, vel) > 0


def test_pattern_boresight_nulls_and_sinc():
    lam = C_LIGHT / hs.F0_HZ
    d = hs.ati_scene(nx=10, ny=10)
    g = oracle.pulse_state(d, 0, 0)
    p, a, e = g["ptx"], g["atx"], g["etx"]
    b = -p / np.linalg.norm(p)
    laz, lel = hs.TX_LEN
    assert math.isclose(oracle.pattern(laz, lel, lam, b, a, e), 1.0, rel_tol=1e-15)
    for u, v in ((lam / laz, 0.0), (0.0, lam / lel), (2 * lam / laz, 0.01)):
        dd = u * a + v * e + math.sqrt(1 - u * u - v * v) * b
        assert abs(oracle.pattern(laz, lel, lam, dd, a, e)) < 1e-25
    rng = np.random.default_rng(5)
    for u, v in rng.uniform(-0.05, 0.05, (20, 2)):
        dd = u * a + v * e + math.sqrt(1 - u * u - v * v) * b
        ref = np.sinc(laz * u / lam) ** 2 * np.sinc(lel * v / lam) ** 2
        assert math.isclose(oracle.pattern(laz, lel, lam, dd, a, e), ref, rel_tol=1e-11,
                            abs_tol=1e-20)


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def test_sigma0_flat_wind_and_specular():
    d = hs.ati_scene(nx=10, ny=10)
    base, mod = d["sigma0_base"], d["wind_mod"]
    ut = _unit([0.1, 0.57, -0.81])
    ur = _unit([-0.28, 0.60, -0.75])
    q = -(ut + ur)
    qh = q[:2] / np.linalg.norm(q[:2])
    # wind along Q_H: upwind maximum
    dw = dict(d, wind_dir_rad=math.atan2(qh[1], qh[0]))
    assert math.isclose(oracle.sigma0(dw, base, ut, ur, 0.0, 0.0), base * (1 + mod), rel_tol=1e-14)
    # wind normal to Q_H: no modulation
    dp = dict(d, wind_dir_rad=math.atan2(qh[1], qh[0]) + math.pi / 2)
    assert math.isclose(oracle.sigma0(dp, base, ut, ur, 0.0, 0.0), base, rel_tol=1e-13)
    # specular tilt: n parallel to Q gives T = |Q| / Q_z
    sx, sy = -q[0] / q[2], -q[1] / q[2]
    want = base * np.linalg.norm(q) / q[2]
    assert math.isclose(oracle.sigma0(dp, base, ut, ur, sx, sy), want, rel_tol=1e-13)
    # facet turned away from Q: no backscatter
    assert oracle.sigma0(dp, base, ut, ur, 40 * q[0] / q[2], 40 * q[1] / q[2]) == 0.0
    # static surfaces keep the constant base value
    ds = dict(d, static_surface=1)
    assert oracle.sigma0(ds, 0.05, ut, ur, 0.3, 0.2) == 0.05


# ---------------------------------------------------------------------------
# Echo: point target, Doppler, linearity, current, brute force (Eq. 3, 4, 16, 17)
# ---------------------------------------------------------------------------
def _centre_scene(taps=1, n_pulses=64, **kw):
    d = hs.small_static(n_pulses=n_pulses)
    d.update(nx=101, ny=101, taps=taps)
    d.update(kw)
    return d


def _centre_facet(d):
    return (d["ny"] // 2) * d["nx"] + d["nx"] // 2


@pytest.mark.parametrize("n", [0, 31, 63])
def test_point_target_box_delay_and_phase(n):
    d = _centre_scene(taps=1)
    f = _centre_facet(d)
    iq = oracle.echo(d, [n], facets=[f])[0, 0]
    g = kin.pulse(d, n, 0)
    r0 = kin.range_start(d, 0)
    dr = mp.mpf(C_LIGHT) / mp.mpf(d["fs_hz"])
    k = int(mp.floor((g["rt"] + g["rr"] - r0) / dr))
    nz = np.nonzero(iq)[0]
    assert list(nz) == [k]
    k0 = 2 * mp.pi * mp.mpf(d["f0_hz"]) / kin.C
    z = oracle.speckle(d["speckle_seed"], f, 0)
    amp = math.sqrt(d["sigma0_base"] * d["facet_m"] ** 2)
    ph = -k0 * (g["rt"] + g["rr"])
    want = amp * z * complex(float(mp.cos(ph)), float(mp.sin(ph)))
    assert abs(iq[k] - want) < 1e-7 * abs(want)


def test_point_target_kaiser_taps():
    d = _centre_scene(taps=8)
    f = _centre_facet(d)
    n = 17
    iq = oracle.echo(d, [n], facets=[f])[0, 0]
    g = kin.pulse(d, n, 0)
    dr = mp.mpf(C_LIGHT) / mp.mpf(d["fs_hz"])
    p = float((g["rt"] + g["rr"] - kin.range_start(d, 0)) / dr)
    k0 = int(math.floor(p))
    nz = np.nonzero(iq)[0]
    assert nz.min() >= k0 - 3 and nz.max() <= k0 + 4
    K0 = 2 * mp.pi * mp.mpf(d["f0_hz"]) / kin.C
    ph = -K0 * (g["rt"] + g["rr"])
    s = (math.sqrt(d["sigma0_base"] * d["facet_m"] ** 2) * oracle.speckle(d["speckle_seed"], f, 0)
         * complex(float(mp.cos(ph)), float(mp.sin(ph))))
    for k in range(k0 - 3, k0 + 5):
        x = k - p
        h = np.sinc(x) * ss.i0(6.0 * math.sqrt(max(0.0, 1 - (x / 4) ** 2))) / ss.i0(6.0)
        # FP64 carries the 2e8-rad phase to ~2e-8 rad
        assert abs(iq[k] - s * h) < 1e-7 * abs(s)


def _mp_steered_axes(p, vel):
    """Azimuth / elevation axes of an antenna at p steered to the scene centre
    (mpmath, from the reading of the paper: boresight toward the origin, azimuth
    = velocity with its boresight part removed, elevation = boresight x azimuth)."""
    r = kin.norm(p)
    b = [-x / r for x in p]
    v = kin.vec(vel)
    vb = kin.dot(v, b)
    t = [v[i] - vb * b[i] for i in range(3)]
    tn = kin.norm(t)
    a = [x / tn for x in t]
    e = [b[1] * a[2] - b[2] * a[1], b[2] * a[0] - b[0] * a[2], b[0] * a[1] - b[1] * a[0]]
    return a, e


def _mp_sinc2_gain(len_az, len_el, lam, d, a, e):
    def sinc(x):
        return mp.mpf(1) if x == 0 else mp.sin(mp.pi * x) / (mp.pi * x)
    return (sinc(mp.mpf(len_az) * kin.dot(d, a) / lam) ** 2
            * sinc(mp.mpf(len_el) * kin.dot(d, e) / lam) ** 2)


@pytest.mark.parametrize("n", [0, 700, 2047])
def test_off_centre_amplitude(n):
    """|contribution| of a static facet far from the scene centre (Eq. 3, Eq. 16):
    sqrt(sigma0 A) |z| G_t G_r Rbar_t Rbar_r / (r_t r_r), every factor evaluated
    here at 50 digits from the descriptor alone: ranges to the facet and to the
    scene centre from the light-time solution, sinc^2 field gains of both antennas
    steered to the scene centre, and |z| = sqrt(-ln u1) from the Philox word (the
    Box-Muller radius). At the patch corners the range ratio departs from 1 by
    ~1e-3 and the transmit gain from 1 by ~0.3, so an inverted or missing range
    factor, a gain applied as power instead of field weight, or the wrong antenna's
    pattern fails by orders of magnitude more than the tolerance."""
    d = hs.ati_scene(n_pulses=2048, nx=2000, ny=1000)
    d.update(static_surface=1, n_omega=0, n_theta=0)
    lam = kin.C / mp.mpf(d["f0_hz"])
    nx, ny = d["nx"], d["ny"]
    facets = [0, nx - 1, (ny - 1) * nx, ny * nx - 1, (ny // 2) * nx + 37]
    epoch = n // d["epoch_pulses"]
    seed = d["speckle_seed"]
    for c in (0, 2, 3, 5):
        g = kin.pulse(d, n, c)
        at, et = _mp_steered_axes(g["ptx"], d["tx"]["vel"])
        ar, er = _mp_steered_axes(g["prx"], d["rx"][c]["vel"])
        for f in facets:
            x, y = kin.facet_xy(d, f)
            xf = [x, y, mp.mpf(0)]
            vt, vr = kin.sub(xf, g["ptx"]), kin.sub(xf, g["prx"])
            rt, rr = kin.norm(vt), kin.norm(vr)
            gt = _mp_sinc2_gain(d["tx"]["len_az"], d["tx"]["len_el"], lam, [v / rt for v in vt], at, et)
            gr = _mp_sinc2_gain(d["rx"][c]["len_az"], d["rx"][c]["len_el"], lam, [v / rr for v in vr], ar, er)
            w0 = oracle.philox4x32_10([f, 0, epoch, 0], [seed & 0xFFFFFFFF, seed >> 32])[0]
            zabs = mp.sqrt(-mp.log((mp.mpf(w0) + 1) / mp.mpf(2) ** 32))
            want = (mp.sqrt(mp.mpf(d["sigma0_base"]) * mp.mpf(d["facet_m"]) ** 2) * zabs * gt * gr
                    * g["rt"] * g["rr"] / (rt * rr))
            val, p = oracle.contribution(d, n, c, f, [0.0, 0.0, 0.0])
            assert abs(abs(val) / float(want) - 1.0) < 1e-11, (n, c, f, abs(val), float(want))
            # the bin position of the same contribution
            dr = kin.C / mp.mpf(d["fs_hz"])
            assert abs(p - float((rt + rr - kin.range_start(d, c)) / dr)) < 1e-8
            # the geometry really is off centre: the factors being pinned are not 1
            if f != (ny // 2) * nx + 37:
                assert abs(float(g["rt"] * g["rr"] / (rt * rr)) - 1.0) > 5e-4
    assert float(gt) < 0.99 or float(gr) < 0.99


def test_bistatic_doppler_phase_history():
    """Corner facet over the burst: the pulse-to-pulse phase equals -K0 times the
    exact bistatic range history, and its central difference matches the closed
    form Doppler -(1/lambda) d(r_t + r_r)/dt (aliased by the PRF)."""
    d = _centre_scene(taps=1)
    f = 0  # corner facet (-100, -100)
    pulses = list(range(0, 64))
    iq = oracle.echo(d, pulses, facets=[f])[0]
    z = oracle.speckle(d["speckle_seed"], f, 0)
    x, y = kin.facet_xy(d, f)
    xf = [x, y, mp.mpf(0)]
    K0 = 2 * mp.pi * mp.mpf(d["f0_hz"]) / kin.C
    phases = []
    for i, n in enumerate(pulses):
        row = iq[i]
        k = int(np.argmax(np.abs(row)))
        assert np.count_nonzero(row) == 1
        g = kin.pulse(d, n, 0)
        rsum = kin.norm(kin.sub(xf, g["ptx"])) + kin.norm(kin.sub(xf, g["prx"]))
        got = np.angle(row[k] / z)
        assert abs(kin.wrap(got + K0 * rsum)) < 2e-7
        phases.append(got)
    # closed-form Doppler at pulse 32 (central difference over 2 PRIs)
    n = 32
    g = kin.pulse(d, n, 0)
    vt, vr = kin.vec(d["tx"]["vel"]), kin.vec(d["rx"][0]["vel"])
    rt_vec, rr_vec = kin.sub(g["ptx"], xf), kin.sub(g["prx"], xf)
    rt_dot = kin.dot(rt_vec, vt) / kin.norm(rt_vec)
    rr_dot = kin.dot(rr_vec, vr) / kin.norm(rr_vec)
    # receive time drifts with the scene-centre ranges
    Rt_dot = kin.dot(g["ptx"], vt) / g["rt"]
    Rr_dot = kin.dot(g["prx"], vr) / g["rr"]
    dtrx = (1 + Rt_dot / kin.C) / (1 - Rr_dot / kin.C)
    rdot = rt_dot + rr_dot * dtrx
    dt = 1 / mp.mpf(d["prf_hz"])
    want = -K0 * rdot * 2 * dt
    got = phases[n + 1] - phases[n - 1]
    assert abs(kin.wrap(got - want)) < 1e-5
    f_d = float(-rdot * mp.mpf(d["f0_hz"]) / kin.C)
    assert -39000 < f_d < -37500  # the bistatic Harmony A Doppler, ~ -38.3 kHz


def test_linearity_in_facets_and_amplitude():
    d = hs.small_static()
    nf = d["nx"] * d["ny"]
    rng = np.random.default_rng(9)
    perm = rng.permutation(nf)
    a, b = np.sort(perm[: nf // 3]), np.sort(perm[nf // 3:])
    pulses = [0, 40]
    full = oracle.echo(d, pulses)
    part = oracle.echo(d, pulses, facets=a) + oracle.echo(d, pulses, facets=b)
    scale = np.abs(full).max()
    assert np.abs(full - part).max() < 1e-12 * scale
    d4 = dict(d, sigma0_base=4 * d["sigma0_base"])
    assert np.abs(oracle.echo(d4, pulses) - 2 * full).max() < 1e-12 * scale


def test_current_phase_single_facet():
    """A uniform current multiplies a facet's contribution by exp(-i K0 v_c t_n)
    with v_c = V . (r_t_hat + r_r_hat) (Eq. 3, Eq. 4) and moves no range bin."""
    d0 = _centre_scene(taps=8)
    dv = dict(d0, current_u=0.5, current_v=0.2)
    f = 123
    x, y = kin.facet_xy(d0, f)
    xf = [x, y, mp.mpf(0)]
    K0 = 2 * mp.pi * mp.mpf(d0["f0_hz"]) / kin.C
    pulses = [0, 20, 63]
    a = oracle.echo(d0, pulses, facets=[f])[0]
    b = oracle.echo(dv, pulses, facets=[f])[0]
    for i, n in enumerate(pulses):
        g = kin.pulse(d0, n, 0)
        dt_, dr_ = kin.sub(xf, g["ptx"]), kin.sub(xf, g["prx"])
        ut = [v / kin.norm(dt_) for v in dt_]
        ur = [v / kin.norm(dr_) for v in dr_]
        vc = mp.mpf(0.5) * (ut[0] + ur[0]) + mp.mpf(0.2) * (ut[1] + ur[1])
        ph = -K0 * vc * g["t"]
        want = complex(float(mp.cos(ph)), float(mp.sin(ph)))
        assert np.array_equal(np.nonzero(a[i])[0], np.nonzero(b[i])[0])
        k = int(np.argmax(np.abs(a[i])))
        assert abs(b[i][k] / a[i][k] - want) < 1e-7  # FP64 phase of a 2e8-rad argument


def test_box_binning_equals_range_slice_brute_force():
    """taps = 1 is the range-slice sum of Eq. 17: each bin is the plain sum of the
    contributions with R_i <= r_t + r_r < R_i+1."""
    d = hs.small_static(n_pulses=8)
    d["taps"] = 1
    nf = d["nx"] * d["ny"]
    n = 5
    iq = oracle.echo(d, [n])[0, 0]
    sums = {}
    zero = np.zeros(3)
    for f in range(nf):
        s, p = oracle.contribution(d, n, 0, f, zero)
        sums.setdefault(int(math.floor(p)), []).append(s)
    want = np.zeros(d["n_range"], dtype=complex)
    for k, v in sums.items():
        if 0 <= k < d["n_range"]:
            want[k] = complex(math.fsum(c.real for c in v), math.fsum(c.imag for c in v))
    assert np.abs(iq - want).max() < 1e-13 * np.abs(want).max()


def test_kaiser_spread_equals_brute_force():
    d = hs.ati_scene(n_pulses=64, nx=24, ny=20, n_range=512)
    n, c = 37, 4
    iq = oracle.echo(d, [n])[c, 0]
    states = oracle.facet_states(d, n)
    acc = [[] for _ in range(d["n_range"])]
    for f in range(d["nx"] * d["ny"]):
        st_ = states[:, f // d["nx"], f % d["nx"]]
        s, p = oracle.contribution(d, n, c, f, st_)
        k0 = int(math.floor(p))
        for k in range(k0 - 3, k0 + 5):
            if 0 <= k < d["n_range"]:
                x = k - p
                h = np.sinc(x) * ss.i0(6.0 * math.sqrt(max(0.0, 1 - (x / 4) ** 2))) / ss.i0(6.0)
                acc[k].append(s * h)
    want = np.array([complex(math.fsum(v.real for v in a), math.fsum(v.imag for v in a))
                     for a in acc])
    assert np.abs(iq - want).max() < 1e-12 * np.abs(want).max()


def test_wave_scene_bins_and_energy():
    """On the wave scene every channel's energy lands inside the range window and
    the facet states follow the surface at the bounce time."""
    d = hs.ati_scene(n_pulses=2048, nx=40, ny=30)
    n = 1000
    iq = oracle.echo(d, [n])
    assert iq.shape == (6, 1, 4096)
    for c in range(6):
        nz = np.nonzero(iq[c, 0])[0]
        assert len(nz) > 0 and nz.min() > 100 and nz.max() < 4000
    states = oracle.facet_states(d, n)
    g = oracle.pulse_state(d, n, 0)
    tab = oracle.wave_table(d)
    f = 17 * d["nx"] + 5
    x, y = kin.facet_xy(d, f)
    s = oracle.surface(tab, float(x), float(y), g["ts"])
    assert np.allclose(states[:, 17, 5], s, atol=1e-14)


# ---------------------------------------------------------------------------
# Bulk exports used by the GPU index parity: the same quantities as the pinned
# single-facet and single-draw functions
# ---------------------------------------------------------------------------
def test_bin_positions_are_the_contributions_positions():
    d = hs.ati_scene(n_pulses=64, nx=24, ny=13, n_range=1024)
    d["cells"] = {"ncx": 5, "ncy": 3, "cell_m": 10.0, "sigma0": np.full((3, 5), 0.02),
                  "uv": np.zeros((3, 5, 2))}
    p, cells = oracle.bin_positions(d, [3, 40])
    nx = d["nx"]
    for i, n in enumerate((3, 40)):
        st = oracle.facet_states(d, n)
        for c in (0, 4):
            for f in (0, 7, nx + 3, 13 * nx - 1):
                _, pf = oracle.contribution(d, n, c, f, st[:, f // nx, f % nx] if st.ndim == 3 else st[:, f])
                assert p[i, c, f // nx, f % nx] == pf
    # cells of 10 m on 2 m facets: 5 facets per cell, clamped at the far edges
    assert cells[0, 0] == 0 and cells[0, 4] == 0 and cells[0, 5] == 1
    assert cells[0, nx - 1] == 4 and cells[12, 0] == 2 * 5


def test_speckle_words_match_curand():
    seed = 1
    facets = [0, 3, 77, 123457, 2**32 - 1]
    epochs = [0, 5, 60, 61, 7]
    got = oracle.speckle_words(seed, facets, epochs)
    for q, (f, e) in enumerate(zip(facets, epochs)):
        blk = _curand_blocks(seed, f * 65536 + e, 1)[0]
        assert [int(v) for v in got[q]] == [int(v) for v in blk]
