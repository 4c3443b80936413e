"""Independent high-precision kinematics for the oracle's pin tests.

Solves the transmit / bounce / receive light-time relations of Eq. 3 with mpmath
at 50 digits, from the scene descriptor alone, so that the oracle's FP64
geometry (three fixed-point steps) is checked against a converged solution.
"""
import mpmath as mp

mp.mp.dps = 50
C = mp.mpf(299792458)


def vec(a):
    return [mp.mpf(v) for v in a]


def pos(ant, t):
    return [mp.mpf(ant["pos0"][i]) + mp.mpf(ant["vel"][i]) * t for i in range(3)]


def norm(v):
    return mp.sqrt(sum(x * x for x in v))


def sub(a, b):
    return [a[i] - b[i] for i in range(3)]


def dot(a, b):
    return sum(a[i] * b[i] for i in range(3))


def pulse(desc, n, c):
    """Transmit time, Tx position, bounce time, Rx time / position at the scene
    centre for pulse n and channel c (converged fixed point)."""
    t = mp.mpf(n) / mp.mpf(desc["prf_hz"])
    ptx = pos(desc["tx"], t)
    rt = norm(ptx)
    ts = t + rt / C
    trx = ts
    for _ in range(40):
        trx = ts + norm(pos(desc["rx"][c], trx)) / C
    prx = pos(desc["rx"][c], trx)
    return {"t": t, "ts": ts, "trx": trx, "ptx": ptx, "prx": prx, "rt": rt, "rr": norm(prx)}


def range_start(desc, c):
    g = pulse(desc, desc["n_pulses"] // 2, c)
    return g["rt"] + g["rr"] - mp.mpf(desc["n_range"]) / 2 * C / mp.mpf(desc["fs_hz"])


def facet_xy(desc, f):
    nx, ny, d = desc["nx"], desc["ny"], mp.mpf(desc["facet_m"])
    ix, iy = f % nx, f // nx
    return (mp.mpf(ix) + mp.mpf(1) / 2 - mp.mpf(nx) / 2) * d, \
        (mp.mpf(iy) + mp.mpf(1) / 2 - mp.mpf(ny) / 2) * d


def wrap(x):
    """Wrap a phase to (-pi, pi]."""
    x = mp.mpf(x)
    two_pi = 2 * mp.pi
    y = x - two_pi * mp.floor(x / two_pi + mp.mpf(1) / 2)
    return float(y)
