"""Golden fixtures (tests/golden/):

* frame_constants.json -- hand-derived constants of the workload frame (carrier,
  sampling, platform geometry and the bistatic range gradient at the scene
  centre), checked against the oracle's pulse state and bin positions;
* oracle_regression.json -- oracle IQ samples written by
  tests/golden/make_oracle_fixtures.py (which calls only the oracle): a change of
  the oracle's arithmetic fails here until the fixture is rewritten on purpose.
"""
import json
import math
import os

import numpy as np
import pytest

import harm_scenes as hs
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
C = 299792458.0


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_frame_constants():
    g = _load("frame_constants.json")
    d = hs.ati_scene()
    lam = C / d["f0_hz"]
    assert lam == pytest.approx(g["lambda_m"][0], abs=g["lambda_m"][1])
    assert 2 * math.pi / lam == pytest.approx(g["k0_rad_per_m"][0], abs=g["k0_rad_per_m"][1])
    assert C / d["fs_hz"] == pytest.approx(g["range_bin_m"][0], abs=g["range_bin_m"][1])
    mid = (d["n_pulses"] - 1) // 2
    st = oracle.pulse_state(d, mid, 1)  # Harmony A, centre phase centre
    assert st["ptx"][1] == pytest.approx(g["tx_ground_range_m"][0], abs=g["tx_ground_range_m"][1])
    assert st["rt_ref"] == pytest.approx(g["tx_range_to_centre_m"][0], abs=g["tx_range_to_centre_m"][1])
    p = st["prx"]
    r = np.linalg.norm(p)
    assert math.degrees(math.acos(p[2] / r)) == pytest.approx(g["rx_incidence_deg"][0], abs=g["rx_incidence_deg"][1])
    assert math.degrees(math.asin(abs(p[0]) / r)) == pytest.approx(g["rx_squint_deg"][0], abs=g["rx_squint_deg"][1])


@pytest.mark.parametrize("channel,key", [(1, "bistatic_range_gradient_harmony_a"),
                                         (4, "bistatic_range_gradient_harmony_b")])
def test_bistatic_range_gradient_at_the_centre(channel, key):
    # central differences of the oracle's bin position over one facet in x and y
    g = _load("frame_constants.json")
    (gx, gy), tol = g[key]
    d = hs.ati_scene(n_pulses=2048, nx=101, ny=101, n_range=4096)
    d.update(static_surface=1, n_omega=0, n_theta=0)
    n = (d["n_pulses"] - 1) // 2
    dr = C / d["fs_hz"]
    centre = 50 * d["nx"] + 50

    def p(f):
        return oracle.contribution(d, n, channel, f, [0.0, 0.0, 0.0])[1]

    grad_x = (p(centre + 1) - p(centre - 1)) * dr / (2 * d["facet_m"])
    grad_y = (p(centre + d["nx"]) - p(centre - d["nx"])) * dr / (2 * d["facet_m"])
    assert grad_x == pytest.approx(gx, abs=tol)
    assert grad_y == pytest.approx(gy, abs=tol)


def test_oracle_regression_fixture():
    import tests.golden.make_oracle_fixtures as mk
    fx = _load("oracle_regression.json")
    for name, d, pulses in mk.cases():
        iq = oracle.echo(d, pulses)
        scale = np.abs(iq).max()
        for c, n, k, re, im in fx[name]:
            got = iq[c, pulses.index(n), k]
            assert abs(got - complex(re, im)) <= 1e-10 * scale, (name, c, n, k)
