"""Batched persistent launch (harm_batch_*): every scene of an uneven batch must
match its single-scene accumulator and the oracle; tuning and CUDA-graph replay
must not change results."""
import numpy as np
import pytest

import harm_scenes as hs
import oracle
from paper_2405_09938_b300 import harm
from tests.gpu_util import assert_iq, rel_rms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _uneven_scenes():
    specs = [(90, 40, 96, 1024, 5.0, 0.3), (37, 70, 64, 512, 12.0, 2.0), (128, 64, 40, 1024, 8.0, 4.0),
             (20, 17, 33, 256, 3.5, 5.5), (64, 96, 70, 1024, 14.0, 1.0)]
    out = []
    for i, (nx, ny, npul, nr, u10, wd) in enumerate(specs):
        d = hs.ati_scene(n_pulses=npul, nx=nx, ny=ny, n_range=nr)
        d["u10"], d["wind_dir_rad"], d["speckle_seed"] = u10, wd, 100 + i
        out.append(d)
    return out


def _single(d):
    import torch
    sc = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    iq = torch.zeros((len(d["rx"]), d["n_pulses"], d["n_range"]), dtype=torch.complex64, device="cuda")
    harm.harm_echo_accumulate(sc, 0, d["n_pulses"], iq)
    harm.harm_scene_sync(sc)
    out = iq.cpu().numpy()
    sc.close()
    return out


def _batch_outputs(descs):
    import torch
    return [torch.full((len(d["rx"]), d["n_pulses"], d["n_range"]), 3.0, dtype=torch.complex64, device="cuda")
            for d in descs]


def test_batch_matches_single_scene_and_oracle():
    import torch
    descs = _uneven_scenes()
    scenes = [harm.harm_scene_create(d, harm.HARM_PREC_MIXED) for d in descs]
    b = harm.harm_batch_create(scenes)
    iqs = _batch_outputs(descs)
    harm.harm_batch_run(b, iqs, zero_first=True)
    torch.cuda.synchronize()
    for d, t in zip(descs, iqs):
        got = t.cpu().numpy()
        assert_iq(got, _single(d), 1e-5)
    for i in (1, 3):
        d = descs[i]
        pulses = [0, d["n_pulses"] // 2, d["n_pulses"] - 1]
        want = oracle.echo(d, pulses)
        assert_iq(iqs[i].cpu().numpy()[:, pulses, :], want, 1e-4)
    b.close()
    for s in scenes:
        s.close()


def test_batch_tune_and_graph_replay():
    import torch
    descs = _uneven_scenes()
    scenes = [harm.harm_scene_create(d, harm.HARM_PREC_MIXED) for d in descs]
    b = harm.harm_batch_create(scenes)
    iqs = _batch_outputs(descs)
    harm.harm_batch_tune(b, iqs)
    rows = harm.harm_batch_tile_rows(b)
    assert all(r in (8, 16) for r in rows)
    harm.harm_batch_run(b, iqs)
    torch.cuda.synchronize()
    first = [t.cpu().numpy() for t in iqs]
    # the tuned tile heights (8-row tiles run one facet per thread) against the
    # single-scene accumulator
    print("tuned tile rows:", rows)
    for d, a in zip(descs, first):
        assert_iq(a, _single(d), 1e-5)
    harm.harm_batch_run(b, iqs)  # graph replay
    torch.cuda.synchronize()
    for a, t in zip(first, iqs):
        assert_iq(t.cpu().numpy(), a, 1e-5)
    # new output buffers: the graph is captured again
    iqs2 = _batch_outputs(descs)
    harm.harm_batch_run(b, iqs2)
    torch.cuda.synchronize()
    for a, t in zip(first, iqs2):
        assert_iq(t.cpu().numpy(), a, 1e-5)
    # accumulate without clearing: doubles
    harm.harm_batch_run(b, iqs2, zero_first=False)
    torch.cuda.synchronize()
    for a, t in zip(first, iqs2):
        assert_iq(t.cpu().numpy(), 2 * a, 1e-5)
    b.close()
    for s in scenes:
        s.close()


def test_batch_eight_row_tiles():
    # 8-row tiles (one facet per thread) pinned on every scene: same echo as the
    # single-scene accumulator (16-row tiles) and as the oracle
    import torch
    descs = _uneven_scenes()
    scenes = [harm.harm_scene_create(d, harm.HARM_PREC_MIXED) for d in descs]
    b = harm.harm_batch_create(scenes)
    with pytest.raises(harm.HarmError):
        harm.harm_batch_set_tile_rows(b, [8, 12, 8, 8, 8])
    harm.harm_batch_set_tile_rows(b, [8] * len(descs))
    assert harm.harm_batch_tile_rows(b) == [8] * len(descs)
    iqs = _batch_outputs(descs)
    harm.harm_batch_run(b, iqs)
    torch.cuda.synchronize()
    for d, t in zip(descs, iqs):
        assert_iq(t.cpu().numpy(), _single(d), 1e-5)
    d = descs[3]
    pulses = [0, d["n_pulses"] - 1]
    assert_iq(iqs[3].cpu().numpy()[:, pulses, :], oracle.echo(d, pulses), 1e-4)
    harm.harm_batch_set_tile_rows(b, [16, 8, 16, 8, 16])  # mixed heights, graph captured again
    harm.harm_batch_run(b, iqs)
    torch.cuda.synchronize()
    for d, t in zip(descs, iqs):
        assert_iq(t.cpu().numpy(), _single(d), 1e-5)
    b.close()
    for s in scenes:
        s.close()


def test_batch_config_windows_and_ctas():
    """Half-length time-Taylor windows on some scenes and one CTA per SM: the same
    echo as the single-scene accumulator (full windows, two CTAs per SM) within
    the Taylor truncation of the longer window; bad shapes are refused."""
    import time

    import torch
    descs = _uneven_scenes()
    scenes = [harm.harm_scene_create(d, harm.HARM_PREC_MIXED) for d in descs]
    pb = harm.harm_scene_query(scenes[0])["pulse_batch"]
    b = harm.harm_batch_create(scenes)
    cfg = harm.harm_batch_config(b)
    assert cfg == {"rows": [16] * 5, "windows": [pb] * 5, "ctas_per_sm": 2}
    for bad in (([16] * 5, [pb] * 4 + [pb // 4], 2), ([16] * 5, [pb] * 5, 3), ([16] * 5, [pb] * 5, 0),
                ([16, 16, 16, 16, 4], [pb] * 5, 1)):
        with pytest.raises(harm.HarmError):
            harm.harm_batch_set_config(b, *bad)
    harm.harm_batch_set_config(b, [16, 8, 16, 8, 16], [pb // 2, pb, pb // 2, pb // 2, pb], 1)
    assert harm.harm_batch_config(b) == {"rows": [16, 8, 16, 8, 16], "windows": [pb // 2, pb, pb // 2, pb // 2, pb],
                                         "ctas_per_sm": 1}
    iqs = _batch_outputs(descs)
    harm.harm_batch_run(b, iqs)
    torch.cuda.synchronize()
    for d, t in zip(descs, iqs):
        assert_iq(t.cpu().numpy(), _single(d), 1e-5)
    # the tuner's choices are kept for the process: a second batch of the same kind
    # is configured without timing, to the same shape
    harm.harm_batch_tune(b, iqs)
    first = harm.harm_batch_config(b)
    b2 = harm.harm_batch_create(scenes)
    t0 = time.perf_counter()
    harm.harm_batch_tune(b2, iqs)
    dt = time.perf_counter() - t0
    assert harm.harm_batch_config(b2) == first
    print("tuned shape:", first, "second tune %.3f s" % dt)
    assert dt < 0.5
    harm.harm_batch_run(b2, iqs)
    torch.cuda.synchronize()
    for d, t in zip(descs, iqs):
        assert_iq(t.cpu().numpy(), _single(d), 1e-5)
    b.close()
    b2.close()
    for s in scenes:
        s.close()


def test_batch_rejects_bad_inputs():
    descs = _uneven_scenes()[:2]
    s64 = harm.harm_scene_create(descs[0], harm.HARM_PREC_FP64)
    smx = harm.harm_scene_create(descs[1], harm.HARM_PREC_MIXED)
    with pytest.raises(harm.HarmError) as ei:
        harm.harm_batch_create([s64, smx])
    assert ei.value.status == harm.HARM_E_UNSUPPORTED
    d1 = hs.small_static()  # one channel
    s1 = harm.harm_scene_create(d1, harm.HARM_PREC_MIXED)
    with pytest.raises(harm.HarmError):
        harm.harm_batch_create([smx, s1])
    b = harm.harm_batch_create([smx])
    import torch
    with pytest.raises(harm.HarmError):
        harm.harm_batch_run(b, [torch.zeros(4, device="cuda")])
    b.close()
    for s in (s64, smx, s1):
        s.close()
