"""Pins of the oracle's FP64 adjoint (gradients of the IQ misfit with respect to
per-cell NRCS and current) against the oracle's forward, which is pinned
separately:

* NRCS: IQ is a sum over cells of sqrt(sigma_cell)-scaled partial echoes (the
  per-cell facet subsets), so dL/dsigma_c = Re <r, IQ_c> / sigma_c exactly, with
  IQ_c the echo of cell c's facets alone.
* Current: central finite differences of L (h = 1e-4 m/s).
* Dot product: <grad L, d> against the directional finite difference along d.
"""
import math

import numpy as np
import pytest

import harm_scenes as hs
import oracle


def _scene(n_pulses=12, nx=40, ny=30, cell_m=20.0, taps=8, seed=3):
    d = hs.ati_scene(n_pulses=n_pulses, nx=nx, ny=ny, n_range=256)
    d["taps"] = taps
    ncx = int(math.ceil(nx * d["facet_m"] / cell_m))
    ncy = int(math.ceil(ny * d["facet_m"] / cell_m))
    rng = np.random.default_rng(seed)
    d["cells"] = {"ncx": ncx, "ncy": ncy, "cell_m": cell_m,
                  "sigma0": 0.02 * (1 + 0.3 * rng.random((ncy, ncx))),
                  "uv": np.stack([0.5 + 0.1 * rng.standard_normal((ncy, ncx)),
                                  0.2 + 0.1 * rng.standard_normal((ncy, ncx))], axis=-1)}
    return d


def _target(d, pulses, seed=4):
    rng = np.random.default_rng(seed)
    t = {k: v for k, v in d.items()}
    cells = dict(d["cells"])
    cells["sigma0"] = d["cells"]["sigma0"] * (1 + 0.2 * rng.random(d["cells"]["sigma0"].shape))
    cells["uv"] = d["cells"]["uv"] + 0.1 * rng.standard_normal(d["cells"]["uv"].shape)
    t["cells"] = cells
    return oracle.echo(t, pulses)


def _with_cells(d, sigma0=None, uv=None):
    e = dict(d)
    c = dict(d["cells"])
    if sigma0 is not None:
        c["sigma0"] = sigma0
    if uv is not None:
        c["uv"] = uv
    e["cells"] = c
    return e


def _cell_of_facets(d):
    nx, ny, dx = d["nx"], d["ny"], d["facet_m"]
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny))
    x = (ix + 0.5 - nx / 2) * dx + nx * dx / 2
    y = (iy + 0.5 - ny / 2) * dx + ny * dx / 2
    cx = np.clip(np.floor(x / d["cells"]["cell_m"]).astype(int), 0, d["cells"]["ncx"] - 1)
    cy = np.clip(np.floor(y / d["cells"]["cell_m"]).astype(int), 0, d["cells"]["ncy"] - 1)
    return (cy * d["cells"]["ncx"] + cx).ravel()


@pytest.mark.parametrize("taps", [8, 1])
def test_sigma_gradient_exact_by_cell_linearity(taps):
    d = _scene(taps=taps)
    pulses = list(range(0, 12, 2))
    tgt = _target(d, pulses)
    iq = oracle.echo(d, pulses)
    r = iq - tgt
    gs, _ = oracle.adjoint(d, pulses, r)
    cell = _cell_of_facets(d)
    ncx = d["cells"]["ncx"]
    total = np.zeros_like(iq)
    for q in range(d["cells"]["ncx"] * d["cells"]["ncy"]):
        fac = np.nonzero(cell == q)[0]
        part = oracle.echo(d, pulses, facets=fac)
        total += part
        want = float(np.real(np.vdot(r, part))) / d["cells"]["sigma0"][q // ncx, q % ncx]
        assert abs(gs[q // ncx, q % ncx] - want) <= 1e-9 * max(1e-30, np.abs(gs).max())
    assert np.abs(total - iq).max() < 1e-12 * np.abs(iq).max()


def test_current_gradient_matches_finite_differences():
    d = _scene()
    pulses = [1, 6, 11]
    tgt = _target(d, pulses)
    r = oracle.echo(d, pulses) - tgt
    _, guv = oracle.adjoint(d, pulses, r)
    h = 1e-4
    gmax = np.abs(guv).max()
    for (cy, cx, comp) in [(0, 0, 0), (1, 3, 1), (2, 1, 0), (0, 2, 1), (1, 1, 1)]:
        up = d["cells"]["uv"].copy()
        dn = d["cells"]["uv"].copy()
        up[cy, cx, comp] += h
        dn[cy, cx, comp] -= h
        lp, _ = oracle.misfit(_with_cells(d, uv=up), pulses, tgt)
        lm, _ = oracle.misfit(_with_cells(d, uv=dn), pulses, tgt)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - guv[cy, cx, comp]) <= 1e-5 * gmax + 1e-6 * abs(fd)


def test_sigma_gradient_matches_finite_differences():
    d = _scene(n_pulses=8)
    pulses = [3, 7]
    tgt = _target(d, pulses)
    r = oracle.echo(d, pulses) - tgt
    gs, _ = oracle.adjoint(d, pulses, r)
    gmax = np.abs(gs).max()
    for (cy, cx) in [(0, 0), (2, 3), (1, 2)]:
        s0 = d["cells"]["sigma0"]
        h = 1e-6 * s0[cy, cx]
        up, dn = s0.copy(), s0.copy()
        up[cy, cx] += h
        dn[cy, cx] -= h
        lp, _ = oracle.misfit(_with_cells(d, sigma0=up), pulses, tgt)
        lm, _ = oracle.misfit(_with_cells(d, sigma0=dn), pulses, tgt)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gs[cy, cx]) <= 1e-5 * gmax


def test_directional_derivative_dot_product():
    d = _scene(n_pulses=8)
    pulses = [0, 5]
    tgt = _target(d, pulses)
    r = oracle.echo(d, pulses) - tgt
    gs, guv = oracle.adjoint(d, pulses, r)
    rng = np.random.default_rng(11)
    ds = 1e-3 * rng.standard_normal(gs.shape)
    duv = rng.standard_normal(guv.shape)
    # eps large enough that the FP64 rounding of the 2e8-rad phases (~2e-8 rad per
    # contribution) stays far below the directional change of L
    eps = 1e-2
    lp, _ = oracle.misfit(_with_cells(d, sigma0=d["cells"]["sigma0"] + eps * ds,
                                      uv=d["cells"]["uv"] + eps * duv), pulses, tgt)
    lm, _ = oracle.misfit(_with_cells(d, sigma0=d["cells"]["sigma0"] - eps * ds,
                                      uv=d["cells"]["uv"] - eps * duv), pulses, tgt)
    fd = (lp - lm) / (2 * eps)
    an = float(np.sum(gs * ds) + np.sum(guv * duv))
    assert abs(fd - an) <= 2e-5 * abs(an)
