"""Pins of the oracle's surface and scattering variants (Sec. III) against
closed forms, invariants, special cases and finite differences: the AR(1)
speckle of Eq. 10 with the intra-facet Doppler shift of Eq. 7, the u-v antenna
gain grids of Sec. III-B, the heterogeneous sea state of Eq. 1 and Eq. 2, and
the Choppy Wave Model."""
import math

import numpy as np
import pytest

import harm_scenes as hs
import oracle

C = 299792458.0


def _tiny(**kw):
    d = hs.ati_scene(n_pulses=64, nx=40, ny=24, n_range=1024)
    d.update(kw)
    return d


# ----------------------------------------------------------------------------
# AR(1) speckle (Eq. 10) and intra-facet Doppler (Eq. 7)
# ----------------------------------------------------------------------------
def test_ar1_beta_from_tau_and_epoch():
    # epoch of 34 pulses at 1700 Hz = 20 ms; tau_s = 20 ms -> beta = 1/e
    d = _tiny(epoch_pulses=34, speckle_tau_s=0.02)
    assert oracle.speckle_beta(d) == pytest.approx(math.exp(-1.0), rel=1e-15)
    assert oracle.speckle_beta(_tiny(epoch_pulses=34, speckle_tau_s=0.0)) == 0.0
    assert oracle.speckle_beta(_tiny(epoch_pulses=0, speckle_tau_s=0.02)) == 0.0


def test_ar1_special_cases_independent_and_frozen():
    for e in (0, 1, 5, 17):
        assert oracle.speckle_ar1(3, 77, e, 0.0) == oracle.speckle(3, 77, e)
        assert oracle.speckle_ar1(3, 77, e, 1.0) == oracle.speckle(3, 77, 0)


def test_ar1_unrolled_closed_form():
    # s_3 = b^3 w_0 + sqrt(1 - b^2) (b^2 w_1 + b w_2 + w_3)
    b = 0.83
    w = [oracle.speckle(9, 1234, e) for e in range(4)]
    want = b ** 3 * w[0] + math.sqrt(1 - b * b) * (b * b * w[1] + b * w[2] + w[3])
    got = oracle.speckle_ar1(9, 1234, 3, b)
    assert abs(got - want) < 1e-14


def test_ar1_statistics_stationary_with_exponential_correlation():
    b = 0.7
    n = 20000
    z5 = np.array([oracle.speckle_ar1(5, f, 5, b) for f in range(n)])
    z7 = np.array([oracle.speckle_ar1(5, f, 7, b) for f in range(n)])
    se = 1.0 / math.sqrt(n)
    assert abs(np.mean(z7)) < 4 * se
    assert abs(np.mean(np.abs(z7) ** 2) - 1.0) < 5 * se
    # R and I each of variance 1/2 (Sec. III-A, reading of Eq. 10's R')
    assert abs(np.mean(z7.real ** 2) - 0.5) < 4 * se
    assert abs(np.mean(z7.imag ** 2) - 0.5) < 4 * se
    # lag-2 correlation E[s_7 conj(s_5)] = beta^2, no cross term
    r = np.mean(z7 * np.conj(z5))
    assert abs(r.real - b * b) < 5 * se
    assert abs(r.imag) < 5 * se


def test_doppler_shift_rotates_contribution_by_2pi_fs_t():
    d0 = _tiny(static_surface=0, n_omega=0, n_theta=0)
    d1 = dict(d0, speckle_doppler_hz=37.5)
    f = 5 * d0["nx"] + 7
    for n in (0, 13, 63):
        s0, p0 = oracle.contribution(d0, n, 0, f, [0.0, 0.0, 0.0])
        s1, p1 = oracle.contribution(d1, n, 0, f, [0.0, 0.0, 0.0])
        t = n / d0["prf_hz"]
        assert p1 == p0
        # the two-way phase is ~2e8 rad: its FP64 rounding (~3e-8 rad) bounds the match
        assert abs(s1 - s0 * np.exp(2j * math.pi * 37.5 * t)) < 1e-7 * abs(s0)


def test_ar1_enters_contribution_through_the_epoch_draws():
    d = hs.ar1_speckle(_tiny(), tau_s=0.01, doppler_hz=0.0, epoch_pulses=8)
    b = oracle.speckle_beta(d)
    f = 3 * d["nx"] + 11
    n = 29  # epoch 3
    s_ar1, _ = oracle.contribution(d, n, 2, f, [0.0, 0.0, 0.0])
    s_ind, _ = oracle.contribution(dict(d, speckle_tau_s=0.0), n, 2, f, [0.0, 0.0, 0.0])
    z_ar1 = oracle.speckle_ar1(d["speckle_seed"], f, 3, b)
    z_ind = oracle.speckle(d["speckle_seed"], f, 3)
    assert abs(s_ar1 - s_ind * z_ar1 / z_ind) < 1e-12 * abs(s_ind)


# ----------------------------------------------------------------------------
# u-v antenna gain grids (Sec. III-B)
# ----------------------------------------------------------------------------
def _pat(gain, u0=-0.01, du=0.001, v0=-0.004, dv=0.0005):
    return {"u0": u0, "du": du, "v0": v0, "dv": dv, "gain": np.asarray(gain)}


def test_lut_node_values_exact():
    rng = np.random.default_rng(0)
    g = rng.standard_normal((17, 21)) + 1j * rng.standard_normal((17, 21))
    p = _pat(g)
    for (iv, iu) in [(0, 0), (16, 20), (3, 7), (16, 0), (0, 20), (9, 12)]:
        u = p["u0"] + iu * p["du"]
        v = p["v0"] + iv * p["dv"]
        assert abs(oracle.lut_gain(p, u, v) - g[iv, iu]) < 1e-12


def test_lut_reproduces_bilinear_function_and_axes():
    # g(u, v) = a + b u + c v + d u v is reproduced exactly; distinct
    # coefficients on u and v catch swapped axes or a transposed grid
    a, b, c, dd = 0.3 + 0.1j, 40.0 - 7j, -90.0 + 20j, 3000.0 + 1000j
    p = _pat(np.zeros((17, 21)))
    uu = p["u0"] + p["du"] * np.arange(21)
    vv = p["v0"] + p["dv"] * np.arange(17)
    U, V = np.meshgrid(uu, vv)
    p["gain"] = a + b * U + c * V + dd * U * V
    rng = np.random.default_rng(1)
    for _ in range(50):
        u = rng.uniform(uu[0], uu[-1])
        v = rng.uniform(vv[0], vv[-1])
        want = a + b * u + c * v + dd * u * v
        assert abs(oracle.lut_gain(p, u, v) - want) < 1e-12


def test_lut_outside_grid_is_zero():
    p = _pat(np.ones((17, 21)))
    assert oracle.lut_gain(p, -0.0101, 0.0) == 0
    assert oracle.lut_gain(p, 0.0101, 0.0) == 0
    assert oracle.lut_gain(p, 0.0, -0.0041) == 0
    assert oracle.lut_gain(p, 0.0, 0.0041) == 0
    assert oracle.lut_gain(p, 0.01, 0.004) == 1.0  # last node is inside


def test_lut_of_sampled_sinc2_matches_analytic_pattern_within_bilinear_bound():
    d = _tiny(static_surface=1)
    lam = C / d["f0_hz"]
    nu, nv = 801, 401
    span_u, span_v = 0.02, 0.02
    u = np.linspace(-span_u / 2, span_u / 2, nu)
    v = np.linspace(-span_v / 2, span_v / 2, nv)

    def grid(ant):
        su = np.sinc(ant["len_az"] * u / lam) ** 2
        sv = np.sinc(ant["len_el"] * v / lam) ** 2
        return _pat(np.outer(sv, su).astype(complex), u0=u[0], du=u[1] - u[0], v0=v[0], dv=v[1] - v[0])

    dl = dict(d, patterns={"tx": grid(d["tx"]), 0: grid(d["rx"][0])})
    # bilinear error <= (h_u^2 max|g_uu| + h_v^2 max|g_vv|) / 8 per antenna;
    # max |d^2 sinc^2(a u)/du^2| = (2 pi^2 / 3) a^2
    def bound(ant):
        au, av = ant["len_az"] / lam, ant["len_el"] / lam
        return ((u[1] - u[0]) ** 2 * 2 * math.pi ** 2 / 3 * au ** 2
                + (v[1] - v[0]) ** 2 * 2 * math.pi ** 2 / 3 * av ** 2) / 8
    tol = bound(d["tx"]) + bound(d["rx"][0])
    rng = np.random.default_rng(2)
    for _ in range(20):
        f = int(rng.integers(0, d["nx"] * d["ny"]))
        n = int(rng.integers(0, d["n_pulses"]))
        s_a, p_a = oracle.contribution(d, n, 0, f, [0.0, 0.0, 0.0])
        s_l, p_l = oracle.contribution(dl, n, 0, f, [0.0, 0.0, 0.0])
        assert p_a == p_l
        # s = A G_t G_r: |G_t' G_r' - G_t G_r| <= eps_t + eps_r for gains <= 1
        gt, gr = _analytic_gains(d, n, 0, f)
        assert abs(s_l - s_a) <= tol * abs(s_a) / (gt * gr) + 1e-300


def _analytic_gains(d, n, c, f):
    g = oracle.pulse_state(d, n, c)
    lam = C / d["f0_hz"]
    ix, iy = f % d["nx"], f // d["nx"]
    x = np.array([(ix + 0.5 - 0.5 * d["nx"]) * d["facet_m"], (iy + 0.5 - 0.5 * d["ny"]) * d["facet_m"], 0.0])
    ut = (x - g["ptx"]) / np.linalg.norm(x - g["ptx"])
    ur = (x - g["prx"]) / np.linalg.norm(x - g["prx"])
    gt = oracle.pattern(d["tx"]["len_az"], d["tx"]["len_el"], lam, ut, g["atx"], g["etx"])
    gr = oracle.pattern(d["rx"][c]["len_az"], d["rx"][c]["len_el"], lam, ur, g["arx"], g["erx"])
    return gt, gr


def test_lut_complex_gain_multiplies_the_field():
    # constant complex gains c_t, c_r replace G_t G_r by c_t c_r
    d = _tiny(static_surface=1)
    ct, cr = 0.8 * np.exp(0.4j), 0.5 * np.exp(-1.1j)
    dl = dict(d, patterns={"tx": _pat(np.full((17, 21), ct)), 0: _pat(np.full((17, 21), cr))})
    f = 7 * d["nx"] + 20
    gt, gr = _analytic_gains(d, 5, 0, f)
    s_a, _ = oracle.contribution(d, 5, 0, f, [0.0, 0.0, 0.0])
    s_l, _ = oracle.contribution(dl, 5, 0, f, [0.0, 0.0, 0.0])
    assert abs(s_l - s_a / (gt * gr) * ct * cr) < 1e-12 * abs(s_l)


# ----------------------------------------------------------------------------
# Heterogeneous sea state (Eq. 1, Eq. 2)
# ----------------------------------------------------------------------------
def _het(tile_m=16.0, nx=40, ny=24, **kw):
    d = _tiny(nx=nx, ny=ny)
    d.update(kw)
    return hs.hetero_sea(d, tile_m=tile_m)


def test_hetero_weights_squares_sum_to_one():
    d = _het()
    ncy, ncx = d["hetero"]["u10"].shape
    lx, ly = d["nx"] * 2.0, d["ny"] * 2.0
    rng = np.random.default_rng(3)
    for _ in range(200):
        x = rng.uniform(-lx / 2, lx / 2)
        y = rng.uniform(-ly / 2, ly / 2)
        w = np.array([[oracle.hetero_weight(d, cx, cy, x, y) for cx in range(ncx)] for cy in range(ncy)])
        assert abs(np.sum(w ** 2) - 1.0) < 1e-14
        assert np.count_nonzero(w) <= 4


def test_hetero_weight_is_one_at_own_corner():
    d = _het()
    ncy, ncx = d["hetero"]["u10"].shape
    lx, ly = d["nx"] * 2.0, d["ny"] * 2.0
    for cy in range(ncy):
        for cx in range(ncx):
            x = -lx / 2 + cx * 16.0
            y = -ly / 2 + cy * 16.0
            if x > lx / 2 or y > ly / 2:
                continue
            w = np.array([[oracle.hetero_weight(d, i, j, x, y) for i in range(ncx)] for j in range(ncy)])
            assert w[cy, cx] == pytest.approx(1.0, abs=1e-15)
            assert np.sum(w) == pytest.approx(1.0, abs=1e-15)


def test_hetero_corner_tables_follow_corner_spectra_with_own_phases():
    d = _het()
    ncy, ncx = d["hetero"]["u10"].shape
    phases = []
    for ci in range(ncx * ncy):
        cy, cx = divmod(ci, ncx)
        tab = oracle.wave_table_corner(d, ci)
        hom = oracle.wave_table(dict(d, u10=float(d["hetero"]["u10"][cy, cx]),
                                     wind_dir_rad=float(d["hetero"]["wind_dir"][cy, cx])))
        for k in ("kx", "ky", "omega", "amp"):
            np.testing.assert_array_equal(tab[k], hom[k])
        phases.append(tab["phase"])
    # uncorrelated tiles: no two corners share their phases
    for i in range(len(phases)):
        for j in range(i + 1, len(phases)):
            assert not np.allclose(phases[i], phases[j])


def test_hetero_state_is_the_weighted_sum_of_corner_tiles():
    # Eq. 1 at one facet: the facet-state routine against the corner tables and
    # weights evaluated separately
    d = _het(nx=40, ny=24)
    ncy, ncx = d["hetero"]["u10"].shape
    n = 9
    st = oracle.facet_states(d, n, fields=3)
    g = oracle.pulse_state(d, n, 0)
    for ix, iy in [(13, 17), (0, 0), (39, 23), (8, 3)]:
        x = (ix + 0.5 - 0.5 * d["nx"]) * 2.0
        y = (iy + 0.5 - 0.5 * d["ny"]) * 2.0
        want = np.zeros(3)
        wsum2 = 0.0
        for ci in range(ncx * ncy):
            cy, cx = divmod(ci, ncx)
            w = oracle.hetero_weight(d, cx, cy, x, y)
            if w == 0.0:
                continue
            wsum2 += w * w
            want += w * oracle.surface(oracle.wave_table_corner(d, ci), x, y, g["ts"])
        assert wsum2 == pytest.approx(1.0, abs=1e-14)
        np.testing.assert_allclose(st[:, iy, ix], want, rtol=0, atol=1e-12)


def test_hetero_variance_is_preserved_across_tiles():
    # identical corner spectra, independent phases: var(eta) = sum W_i^2 m0 = m0
    # everywhere (with W_i not square-rooted the tile centres would drop to m0/4)
    m0 = None
    vals = []
    for seed in range(120):
        d = _het(tile_m=16.0, nx=16, ny=16, wave_seed=100 + seed)
        d["hetero"]["u10"][:] = 8.0
        d["hetero"]["wind_dir"][:] = math.radians(30.0)
        if m0 is None:
            tab = oracle.wave_table(dict(d, u10=8.0, wind_dir_rad=math.radians(30.0)))
            m0 = float(np.sum(tab["amp"] ** 2) / 2)
        st = oracle.facet_states(d, 0, fields=1)[0]
        vals.append(st[[0, 4, 8, 12], :][:, [0, 4, 8, 12]].ravel())
    v = np.array(vals)  # [seeds, 16 points]
    ratio = np.mean(v ** 2) / m0
    assert abs(ratio - 1.0) < 0.12
    # points (ix, iy) = (4, 4) and (12, 12) sit 1 m from TL-tile centres, where all
    # four weights are ~1/2: the variance is still m0 there (it would be ~m0/4
    # with bilinear weights that are not square-rooted)
    centres = v[:, [5, 15]]
    assert np.mean(centres ** 2) / m0 > 0.6


# ----------------------------------------------------------------------------
# Choppy Wave Model
# ----------------------------------------------------------------------------
def _single_wave(kx=0.05, ky=0.03, a=1.3, om=None, ph=0.4):
    k = math.hypot(kx, ky)
    om = math.sqrt(9.80665 * k) if om is None else om
    return {"kx": np.array([kx]), "ky": np.array([ky]), "omega": np.array([om]),
            "amp": np.array([a]), "phase": np.array([ph])}


def test_cwm_single_wave_moves_points_on_circles():
    tab = _single_wave()
    rng = np.random.default_rng(4)
    for _ in range(30):
        x, y, t = rng.uniform(-500, 500), rng.uniform(-500, 500), rng.uniform(0, 10)
        s = oracle.surface_cwm(tab, x, y, t)
        assert s[3] ** 2 + s[4] ** 2 + s[0] ** 2 == pytest.approx(1.3 ** 2, rel=1e-13)
        # the displacement is along the wave vector
        assert abs(s[3] * 0.03 - s[4] * 0.05) < 1e-13


def test_cwm_single_wave_jacobian_closed_form():
    kx, ky, a, ph = 0.05, 0.03, 1.3, 0.4
    tab = _single_wave(kx, ky, a, ph=ph)
    k = math.hypot(kx, ky)
    for x, y, t in [(3.0, -7.0, 0.5), (100.0, 40.0, 2.0), (-250.0, 10.0, 7.7)]:
        s = oracle.surface_cwm(tab, x, y, t)
        th = kx * x + ky * y - tab["omega"][0] * t + ph
        det = (1 + s[5]) * (1 + s[7]) - s[6] ** 2
        assert det == pytest.approx(1 - a * k * math.cos(th), abs=1e-13)


def test_cwm_derivative_fields_match_finite_differences_of_the_displaced_surface():
    d = choppy_tiny = hs.choppy(_tiny())
    tab = oracle.wave_table(choppy_tiny)
    h = 1e-3
    for x, y, t in [(1.0, 2.0, 0.3), (-31.0, 17.0, 1.1)]:
        s = oracle.surface_cwm(tab, x, y, t)
        px = (oracle.surface_cwm(tab, x + h, y, t) - oracle.surface_cwm(tab, x - h, y, t)) / (2 * h)
        py = (oracle.surface_cwm(tab, x, y + h, t) - oracle.surface_cwm(tab, x, y - h, t)) / (2 * h)
        # value fields 0 (eta), 3 (D_x), 4 (D_y) differentiated numerically
        assert s[1] == pytest.approx(px[0], abs=1e-7)
        assert s[2] == pytest.approx(py[0], abs=1e-7)
        assert s[5] == pytest.approx(px[3], abs=1e-7)
        assert s[6] == pytest.approx(py[3], abs=1e-7)
        assert s[6] == pytest.approx(px[4], abs=1e-7)
        assert s[7] == pytest.approx(py[4], abs=1e-7)
    assert d["cwm"] == 1


def test_cwm_eulerian_mean_height_is_minus_half_a2k():
    # 1-D single wave along x: the mean of the displaced surface's height over one
    # wavelength in the Eulerian (fixed x) sense is -a^2 k / 2 (the CWM lowers the
    # mean level; the opposite displacement sign would raise it)
    a, k = 0.9, 0.08
    tab = _single_wave(kx=k, ky=0.0, a=a, ph=0.0)
    lam = 2 * math.pi / k
    xs = np.linspace(0.0, lam, 512, endpoint=False)
    acc = 0.0
    for x in xs:
        s = oracle.surface_cwm(tab, x, 0.0, 0.0)
        acc += s[0] * (1 + s[5])  # eta dx = eta (1 + dD_x/dxbar) dxbar
    mean = acc * (lam / len(xs)) / lam
    assert mean == pytest.approx(-a * a * k / 2, rel=1e-10)


def test_cwm_off_is_the_linear_surface():
    d = _tiny()
    st8 = oracle.facet_states(d, 3, fields=8)
    assert np.all(st8[3:] == 0.0)
    dc = hs.choppy(d)
    st8c = oracle.facet_states(dc, 3, fields=8)
    np.testing.assert_array_equal(st8c[:3], st8[:3])
    assert np.any(st8c[3:] != 0.0)


def test_cwm_displacement_moves_the_facet_in_range():
    d = _tiny(static_surface=1)
    n, c = 20, 1
    f = 9 * d["nx"] + 4
    ix, iy = f % d["nx"], f // d["nx"]
    g = oracle.pulse_state(d, n, c)
    r0 = oracle.range_start(d, c)
    dr = C / d["fs_hz"]
    Dx, Dy, eta = 0.7, -1.9, 0.3
    st = [eta, 0.0, 0.0, Dx, Dy, 0.0, 0.0, 0.0]
    _, p = oracle.contribution(d, n, c, f, st)
    x = np.array([(ix + 0.5 - 0.5 * d["nx"]) * 2.0 + Dx, (iy + 0.5 - 0.5 * d["ny"]) * 2.0 + Dy, eta])
    want = (np.linalg.norm(x - g["ptx"]) + np.linalg.norm(x - g["prx"]) - r0) / dr
    assert p == pytest.approx(want, abs=1e-9)


def test_cwm_compression_scales_the_facet_area():
    d = _tiny(static_surface=0, n_omega=0, n_theta=0, wind_mod=0.0)
    f = 9 * d["nx"] + 4
    s0, _ = oracle.contribution(d, 4, 0, f, [0, 0, 0, 0, 0, 0, 0, 0])
    s1, _ = oracle.contribution(d, 4, 0, f, [0, 0, 0, 0, 0, -0.2, 0, 0])
    # flat facet, horizontal area x 0.8: amplitude x sqrt(0.8), same phase
    assert abs(s1 - s0 * math.sqrt(0.8)) < 1e-13 * abs(s0)


def test_cwm_normal_from_tangents():
    # tilted tangents: sigma0 tilt uses n = T_x x T_y of the displaced surface
    d = _tiny(static_surface=0, wind_mod=0.0)
    rt = np.array([0.1, 0.5, -0.86])
    rt /= np.linalg.norm(rt)
    rr = np.array([-0.2, 0.6, -0.77])
    rr /= np.linalg.norm(rr)
    jxx, jxy, jyy, ex, ey = 0.1, -0.05, 0.2, 0.12, -0.07
    tx = np.array([1 + jxx, jxy, ex])
    ty = np.array([jxy, 1 + jyy, ey])
    nvec = np.cross(tx, ty)
    q = -(rt + rr)
    want = 0.02 * max(0.0, nvec @ q) / (np.linalg.norm(nvec) * q[2])
    assert oracle.sigma0_normal(d, 0.02, rt, rr, nvec) == pytest.approx(want, rel=1e-14)
    # the linear-surface form is the special case n = (-eta_x, -eta_y, 1)
    assert oracle.sigma0(d, 0.02, rt, rr, ex, ey) == pytest.approx(
        oracle.sigma0_normal(d, 0.02, rt, rr, [-ex, -ey, 1.0]), rel=1e-15)
