"""Parity at the full sizes of the measured workloads, in the launch
configuration the bench times, on outputs the FP64 oracle can compute one by one:

* the headline ATI scene (2000 x 1000 facets, 2048 pulses, 6 channels, complex64,
  one launch over the whole burst): IQ relative RMS and ATI phase bias on 3
  sampled pulses, all channels and range samples, and the error of the FP32
  accumulation stage (complex64 against complex128 output of the same run);
* the 48-scene batch (one persistent graph-replayed launch after tuning): one
  pulse of the smallest and of the largest scene;
* the differentiable scene (1000 x 500 facets, 6 channels, 100 m cells): the
  adjoint of an 8-pulse window inside the burst against the oracle's FP64
  adjoint of the same window.
"""
import numpy as np
import pytest

import harm_scenes as hs
import oracle
from paper_2405_09938_b300 import harm
from tests.gpu_util import assert_iq, ati_phase_bias, rel_rms, take_pulses

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-4
TOL_GRAD = 2e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_headline_scene_full_burst_sampled_pulses():
    import torch
    d = hs.ati_scene()
    sc = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    iq = torch.zeros((6, d["n_pulses"], d["n_range"]), dtype=torch.complex64, device="cuda")
    harm.harm_echo_accumulate(sc, 0, d["n_pulses"], iq)
    harm.harm_scene_sync(sc)
    pulses = [0, 1023, 2047]
    got = take_pulses(iq, pulses)
    sc.close()
    del iq
    want = oracle.echo(d, pulses)
    err, pe = assert_iq(got, want, TOL_MIXED)
    print("headline scene: IQ rel RMS %.3e, per-element error %.3e of the row peak" % (err, pe))
    for c in range(6):
        assert_iq(got[c], want[c], TOL_MIXED)
    for a, b in ((0, 1), (1, 2), (3, 4), (4, 5)):
        assert abs(ati_phase_bias(got, want, a, b)) < 1e-4


def test_headline_scene_plain_fp32_error():
    """The plain method in FP32 (HARM_PREC_FP32) on the full headline scene, one
    launch over the burst: its IQ error against the FP64 oracle on sampled pulses,
    recorded to show why the mixed path keeps the reference ranges in FP64. FP32
    rounding of the ~2 km range offsets (1.2e-4 m) and of the ~2e5 rad phase
    (1.6e-2 rad) spreads every contribution's phase by ~1e-2 rad, so the IQ error
    is ~1e-2 (measured on a B300: 5.4e-3, worst ATI bias 4.6e-4 rad): two orders
    above the mixed path on the same scene."""
    import torch
    d = hs.ati_scene()
    sc = harm.harm_scene_create(d, harm.HARM_PREC_FP32)
    iq = torch.zeros((6, d["n_pulses"], d["n_range"]), dtype=torch.complex64, device="cuda")
    harm.harm_echo_accumulate(sc, 0, d["n_pulses"], iq)
    harm.harm_scene_sync(sc)
    pulses = [0, 1023, 2047]
    got = take_pulses(iq, pulses)
    sc.close()
    del iq
    want = oracle.echo(d, pulses)
    err = rel_rms(got, want)
    bias = max(abs(ati_phase_bias(got, want, a, b)) for a, b in ((0, 1), (1, 2), (3, 4), (4, 5)))
    print("headline scene, plain FP32: IQ rel RMS %.3e, worst ATI bias %.3e rad" % (err, bias))
    assert err < 2e-2
    assert bias < 5e-3
    # the plain FP32 form cannot hold the mixed path's 1e-4 bound on this scene
    assert err > 10 * TOL_MIXED


def test_headline_complex64_accumulation_error():
    # the FP32 warp and tile sums are common to both outputs; the complex64 output
    # also adds the tiles into the IQ in FP32 (atomics), the complex128 output in
    # FP64: their difference bounds the error of the FP32 accumulation stage
    import torch
    d = hs.ati_scene()
    sc = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    pulses = [5, 1500]
    outs = []
    for dt in (torch.complex64, torch.complex128):
        iq = torch.zeros((6, d["n_pulses"], d["n_range"]), dtype=dt, device="cuda")
        harm.harm_echo_accumulate(sc, 0, d["n_pulses"], iq)
        harm.harm_scene_sync(sc)
        outs.append(take_pulses(iq, pulses).astype(np.complex128))
        del iq
    sc.close()
    err = rel_rms(outs[0], outs[1])
    print("complex64 vs complex128 accumulation: rel RMS %.3e" % err)
    assert err < 2e-6


def test_batch_of_48_scenes_full_size_sampled():
    import torch
    descs = hs.batch_scenes()
    scenes = [harm.harm_scene_create(d, harm.HARM_PREC_MIXED) for d in descs]
    iqs = [torch.empty((6, d["n_pulses"], d["n_range"]), dtype=torch.complex64, device="cuda") for d in descs]
    b = harm.harm_batch_create(scenes)
    harm.harm_batch_tune(b, iqs)
    harm.harm_batch_run(b, iqs)
    torch.cuda.synchronize()
    sizes = [hs.n_facets(d) for d in descs]
    for s in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        d = descs[s]
        n = d["n_pulses"] // 3
        got = take_pulses(iqs[s], [n])
        want = oracle.echo(d, [n])
        err, pe = assert_iq(got, want, TOL_MIXED)
        print("batch scene %d (%d facets): IQ rel RMS %.3e, per-element %.3e" % (s, sizes[s], err, pe))
    b.close()
    for sc in scenes:
        sc.close()


def test_adjoint_scene_full_size_window():
    import torch
    d = hs.adjoint_scene()
    c = d["cells"]
    n0, nw = 600, 8
    rng = np.random.default_rng(41)
    resid = (rng.standard_normal((6, nw, d["n_range"])) + 1j * rng.standard_normal((6, nw, d["n_range"]))) * 1e-3
    want_s, want_uv = oracle.adjoint(d, list(range(n0, n0 + nw)), resid)
    sc = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    s0 = torch.tensor(c["sigma0"], dtype=torch.float64, device="cuda")
    uv = torch.tensor(c["uv"], dtype=torch.float64, device="cuda")
    harm.harm_scene_set_cells(sc, c["ncx"], c["ncy"], c["cell_m"], s0, uv)
    r = torch.tensor(resid, dtype=torch.complex64, device="cuda")
    gs, guv = torch.zeros_like(s0), torch.zeros_like(uv)
    harm.harm_echo_adjoint(sc, n0, nw, r, gs, guv)
    harm.harm_scene_sync(sc)
    got_s, got_uv = gs.cpu().numpy(), guv.cpu().numpy()
    sc.close()
    es = np.abs(got_s - want_s).max() / np.abs(want_s).max()
    eu = np.abs(got_uv - want_uv).max() / np.abs(want_uv).max()
    print("adjoint window: sigma0 %.3e, current %.3e (relative to the largest component)" % (es, eu))
    assert es < TOL_GRAD
    assert eu < TOL_GRAD
