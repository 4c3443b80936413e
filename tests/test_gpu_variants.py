"""GPU parity of the surface and scattering variants (Sec. III) against the FP64
oracle, through the C ABI: AR(1) speckle (Eq. 10) with the intra-facet Doppler
shift (Eq. 7), u-v antenna gain grids (Sec. III-B), heterogeneous sea states
(Eq. 1, 2) and the Choppy Wave Model, alone and combined, on both precisions,
plus the facet generator's CWM fields and the adjoint of a variant scene.

Scenes are 150 x 70 facets (ragged against the 32 x 16 tiles), 400 pulses (two
256-pulse time-Taylor windows, the second ragged), 6 channels; tolerances as in the base
parity tests: 1e-7 (FP64 path) and 1e-4 (mixed path) IQ relative RMS."""
import math

import numpy as np
import pytest

import harm_scenes as hs
import oracle
from paper_2405_09938_b300 import harm
from tests.gpu_util import assert_iq, rel_rms, run_echo

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-7
TOL_MIXED = 1e-4
PULSES = [0, 77, 255, 256, 399]  # both windows, their shared edge and the tail


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _base(n_pulses=400):
    return hs.ati_scene(n_pulses=n_pulses, nx=150, ny=70, n_range=1024)


VARIANTS = {
    "ar1_doppler": lambda d: hs.ar1_speckle(d, tau_s=0.03, doppler_hz=12.0, epoch_pulses=8),
    "uv_grids": lambda d: hs.uv_patterns(d),
    "hetero": lambda d: hs.hetero_sea(d, tile_m=100.0),
    "cwm": lambda d: hs.choppy(d),
    "all": lambda d: hs.uv_patterns(hs.choppy(hs.hetero_sea(
        hs.ar1_speckle(d, tau_s=0.03, doppler_hz=12.0, epoch_pulses=8), tile_m=100.0))),
}


def _check(d, prec, tol):
    got = run_echo(d, prec, 0, d["n_pulses"], "c128")[:, PULSES, :]
    want = oracle.echo(d, PULSES)
    assert_iq(got, want, tol)
    for c in range(len(d["rx"])):
        assert_iq(got[c], want[c], tol)


@pytest.mark.parametrize("name", list(VARIANTS))
def test_variant_mixed_matches_oracle(name):
    _check(VARIANTS[name](_base()), harm.HARM_PREC_MIXED, TOL_MIXED)


@pytest.mark.parametrize("name", ["uv_grids", "cwm", "all"])
def test_variant_mixed_three_channels(name):
    # one receive antenna: the variant kernels' general channel loop (six-channel
    # scenes run instantiations with a compile-time channel count)
    d = _base()
    tx, rx = hs.geometry(d["n_pulses"], ("A",), (-hs.PHASE_CENTRE_SPACING_M, 0.0, hs.PHASE_CENTRE_SPACING_M))
    d["tx"], d["rx"] = tx, rx
    _check(VARIANTS[name](d), harm.HARM_PREC_MIXED, TOL_MIXED)


@pytest.mark.parametrize("name", list(VARIANTS))
def test_variant_fp64_matches_oracle(name):
    d = VARIANTS[name](_base(n_pulses=48))
    got = run_echo(d, harm.HARM_PREC_FP64, 0, 48, "c128")
    pulses = [0, 17, 47]
    want = oracle.echo(d, pulses)
    assert_iq(got[:, pulses, :], want, TOL_FP64)


@pytest.mark.parametrize("name", list(VARIANTS))
def test_variant_fp32_plain_matches_oracle(name):
    # the plain FP32 path runs the FP64 path's template in float: every variant,
    # within the plain FP32 path's own error on this 300 x 140 m scene (measured
    # 2e-4 without variants; the bound is that of the plain FP32 parity tests)
    d = VARIANTS[name](_base(n_pulses=48))
    got = run_echo(d, harm.HARM_PREC_FP32, 0, 48, "c128")
    pulses = [0, 17, 47]
    want = oracle.echo(d, pulses)
    assert_iq(got[:, pulses, :], want, 1e-3)


def test_variant_changes_the_echo():
    # each variant moves the IQ well beyond the tolerance (the parity above is not vacuous)
    d = _base(n_pulses=48)
    base = oracle.echo(d, [17])
    for name, f in VARIANTS.items():
        assert rel_rms(oracle.echo(f(d), [17]), base) > 1e-2, name


def test_ar1_truncated_restart_mid_burst():
    # beta = exp(-(8/1700)/0.003) = 0.21: the mixed path restarts the recurrence
    # from the last 19 epochs at a window that starts at epoch 128; the oracle runs
    # it from epoch 0
    d = hs.ar1_speckle(_base(n_pulses=1100), tau_s=0.003, doppler_hz=-7.0, epoch_pulses=8)
    n0, np_ = 1024, 76
    got = run_echo(d, harm.HARM_PREC_MIXED, n0, np_, "c128")
    pulses = [1024, 1060, 1099]
    want = oracle.echo(d, pulses)
    assert_iq(got[:, [p - n0 for p in pulses], :], want, TOL_MIXED)


def test_cwm_generator_fields():
    import torch
    d = hs.hetero_sea(hs.choppy(_base(n_pulses=100)), tile_m=100.0)
    # FP32: four corner tables of 256 components each are summed (heights ~1 m)
    for prec, dt, tol in [(harm.HARM_PREC_FP64, torch.float64, 1e-11),
                          (harm.HARM_PREC_MIXED, torch.float32, 6e-6)]:
        scene = harm.harm_scene_create(d, prec)
        st = torch.zeros((6, 8, d["ny"], d["nx"]), dtype=dt, device="cuda")
        harm.harm_facets_generate(scene, 40, 6, st)
        harm.harm_scene_sync(scene)
        got = st.cpu().numpy().astype(np.float64)
        scene.close()
        for i, n in [(0, 40), (5, 45)]:
            want = oracle.facet_states(d, n, fields=8)
            assert np.abs(got[i] - want).max() < tol


@pytest.mark.parametrize("nx", [152, 150])
def test_hetero_generator_fields(nx):
    """Three-field states of a heterogeneous sea (Eq. 1, 2) from the mixed
    generator, every pulse of a window that starts and ends off the 256-pulse
    time-Taylor windows. A width nx % 4 == 0 takes the generator whose states
    leave shared memory by bulk tensor stores (clipped at the scene's edges),
    other widths the one with direct stores."""
    import torch
    d = hs.hetero_sea(hs.ati_scene(n_pulses=300, nx=nx, ny=70, n_range=1024), tile_m=100.0)
    n0, np_ = 17, 263
    scene = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    st = torch.full((np_, 3, 70, nx), float("nan"), dtype=torch.float32, device="cuda")
    harm.harm_facets_generate(scene, n0, np_, st)
    harm.harm_scene_sync(scene)
    got = st.cpu().numpy().astype(np.float64)
    scene.close()
    assert not np.isnan(got).any()
    for n in (17, 18, 255, 256, 257, 279):
        want = oracle.facet_states(d, n)
        assert np.abs(got[n - n0] - want).max() < 6e-6


def test_uv_grid_set_and_removed():
    import torch
    d = _base(n_pulses=48)
    dl = hs.uv_patterns(d)
    scene = harm.harm_scene_create(dl, harm.HARM_PREC_MIXED)
    iq = torch.zeros((6, 48, 1024), dtype=torch.complex128, device="cuda")
    harm.harm_echo_accumulate(scene, 0, 48, iq)
    harm.harm_scene_sync(scene)
    with_grid = iq.cpu().numpy()
    harm.harm_scene_set_pattern(scene, -1, None)
    for c in range(6):
        harm.harm_scene_set_pattern(scene, c, None)
    harm.harm_echo_accumulate(scene, 0, 48, iq)
    harm.harm_scene_sync(scene)
    without = iq.cpu().numpy()
    scene.close()
    assert_iq(with_grid[:, [17], :], oracle.echo(dl, [17]), TOL_MIXED)
    assert_iq(without[:, [17], :], oracle.echo(d, [17]), TOL_MIXED)
    # channel 6 does not exist; a grid with one node per axis is rejected
    other = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    with pytest.raises(harm.HarmError):
        harm.harm_scene_set_pattern(other, 6, dl["patterns"]["tx"])
    with pytest.raises(harm.HarmError):
        harm.harm_scene_set_pattern(other, 0, dict(dl["patterns"]["tx"], gain=np.ones((1, 5))))
    other.close()


def test_variant_adjoint_matches_oracle_adjoint():
    import torch
    d = VARIANTS["all"](hs.ati_scene(n_pulses=40, nx=96, ny=64, n_range=512))
    cell_m = 16.0
    ncx, ncy = int(math.ceil(96 * 2 / cell_m)), int(math.ceil(64 * 2 / cell_m))
    rng = np.random.default_rng(5)
    d["cells"] = {"ncx": ncx, "ncy": ncy, "cell_m": cell_m,
                  "sigma0": 0.02 * (1 + 0.3 * rng.random((ncy, ncx))),
                  "uv": np.stack([0.5 + 0.1 * rng.standard_normal((ncy, ncx)),
                                  0.2 + 0.1 * rng.standard_normal((ncy, ncx))], axis=-1)}
    pulses = list(range(40))
    resid = (rng.standard_normal((6, 40, 512)) + 1j * rng.standard_normal((6, 40, 512))) * 1e-3
    want_s, want_uv = oracle.adjoint(d, pulses, resid)
    scene = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    c = d["cells"]
    s0 = torch.tensor(c["sigma0"], dtype=torch.float64, device="cuda")
    uv = torch.tensor(c["uv"], dtype=torch.float64, device="cuda")
    harm.harm_scene_set_cells(scene, ncx, ncy, cell_m, s0, uv)
    r = torch.tensor(resid, dtype=torch.complex64, device="cuda")
    gs, guv = torch.zeros_like(s0), torch.zeros_like(uv)
    harm.harm_echo_adjoint(scene, 0, 40, r, gs, guv)
    harm.harm_scene_sync(scene)
    got_s, got_uv = gs.cpu().numpy(), guv.cpu().numpy()
    scene.close()
    assert np.abs(got_s - want_s).max() < 2e-3 * np.abs(want_s).max()
    assert np.abs(got_uv - want_uv).max() < 2e-3 * np.abs(want_uv).max()


def test_batch_of_variant_scenes():
    import torch
    descs = []
    for i, (nx, ny, npul) in enumerate([(90, 40, 96), (64, 70, 270), (40, 33, 50)]):
        d = hs.ati_scene(n_pulses=npul, nx=nx, ny=ny, n_range=1024)
        d["speckle_seed"] = 400 + i
        descs.append(hs.choppy(hs.hetero_sea(hs.ar1_speckle(d, tau_s=0.02, epoch_pulses=8), tile_m=60.0)))
    scenes = [harm.harm_scene_create(d, harm.HARM_PREC_MIXED) for d in descs]
    b = harm.harm_batch_create(scenes)
    iqs = [torch.zeros((6, d["n_pulses"], 1024), dtype=torch.complex64, device="cuda") for d in descs]
    harm.harm_batch_run(b, iqs)
    torch.cuda.synchronize()
    for d, t in zip(descs, iqs):
        pulses = [0, d["n_pulses"] - 1]
        assert_iq(t.cpu().numpy()[:, pulses, :], oracle.echo(d, pulses), TOL_MIXED)
    b.close()
    # scenes of different surface models do not batch together
    plain = harm.harm_scene_create(hs.ati_scene(n_pulses=50, nx=40, ny=33, n_range=1024), harm.HARM_PREC_MIXED)
    with pytest.raises(harm.HarmError):
        harm.harm_batch_create([scenes[0], plain])
    for s in scenes + [plain]:
        s.close()
