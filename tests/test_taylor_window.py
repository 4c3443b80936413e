"""Bound on the time-Taylor truncation of the mixed path's facet generator.

The mixed path expands each wave component's time factor e^{-i omega tau} about
the centre of a 256-pulse window to order 5 (Sec. III surface, evaluated per
pulse). On the headline spectrum (256 JONSWAP / cos^2s components, U10 8 m/s,
1700 Hz PRF) the remainder, summed over all components as if they were in phase,
must stay well below the FP32 phase error of the path (~3e-5 rad RMS): this pins
the window length to the wave spectrum and the pulse rate. The spectrum comes
from the oracle's wave table; the remainder is the exact difference between
e^{-i omega tau} and its truncated series at the window edge.
"""
import math

import numpy as np

import harm_scenes as hs
import oracle

WINDOW_PULSES = 256  # pulses per time-Taylor window of the mixed path
ORDERS = 6           # Taylor orders 0..5


def _bounds(desc, window):
    t = oracle.wave_table(desc)
    om, a = t["omega"], t["amp"]
    k = np.hypot(t["kx"], t["ky"])
    tau = 0.5 * window / desc["prf_hz"]
    z = -1j * om * tau
    series = sum(z ** m / math.factorial(m) for m in range(ORDERS))
    rem = np.abs(np.exp(z) - series)
    k0 = 2.0 * math.pi * desc["f0_hz"] / 299792458.0
    height = float(np.sum(a * rem))          # m
    slope = float(np.sum(a * k * rem))       # rad of slope
    return height, slope, 2.0 * k0 * height  # two-way phase, rad


def test_remainder_matches_the_lagrange_bound():
    # |e^{z} - sum_{m<6} z^m/m!| <= |z|^6 / 6! for imaginary z
    d = hs.ati_scene(n_pulses=8, nx=4, ny=4)
    t = oracle.wave_table(d)
    tau = 0.5 * WINDOW_PULSES / d["prf_hz"]
    z = -1j * t["omega"] * tau
    rem = np.abs(np.exp(z) - sum(z ** m / math.factorial(m) for m in range(ORDERS)))
    assert np.all(rem <= np.abs(z) ** ORDERS / math.factorial(ORDERS) * (1 + 1e-9))
    assert np.max(np.abs(z)) < 0.2


def test_headline_window_truncation_below_fp32_phase_error():
    d = hs.ati_scene(n_pulses=8, nx=4, ny=4)
    height, slope, phase = _bounds(d, WINDOW_PULSES)
    assert height < 1e-7
    assert slope < 1e-7
    assert phase < 2e-5
    # each doubling of the window multiplies the remainder by ~2^6: a 512-pulse
    # window would reach the path's 1e-4 tolerance
    assert _bounds(d, 2 * WINDOW_PULSES)[2] > 1e-4
