"""harm_batch_run_noalloc: the allocation-free batched run (for callers that cannot
allocate device memory where they run the echo) must give the same IQ as the
allocating entry point harm_batch_run, on two calls in a row that share the
library's fixed scratch array. Collected last on purpose (file name), and it
does not depend on state left by other tests."""
import pytest

import harm_scenes as hs
from paper_2405_09938_b300 import harm
from tests.gpu_util import assert_iq, rel_rms

pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative RMS between two runs of the same batched computation


def _scenes():
    specs = [(70, 33, 48, 512, 6.0, 0.4), (40, 64, 40, 1024, 11.0, 2.5), (96, 48, 64, 1024, 9.0, 5.0)]
    out = []
    for i, (nx, ny, npul, nr, u10, wd) in enumerate(specs):
        d = hs.ati_scene(n_pulses=npul, nx=nx, ny=ny, n_range=nr)
        d["u10"], d["wind_dir_rad"], d["speckle_seed"] = u10, wd, 300 + i
        out.append(d)
    return out


def test_noalloc_matches_batch_run_twice():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    descs = _scenes()
    scenes = [harm.harm_scene_create(d, harm.HARM_PREC_MIXED) for d in descs]
    shapes = [(len(d["rx"]), d["n_pulses"], d["n_range"]) for d in descs]
    ref = [torch.zeros(s, dtype=torch.complex64, device="cuda") for s in shapes]
    b = harm.harm_batch_create(scenes)
    harm.harm_batch_run(b, ref)
    torch.cuda.synchronize()
    want = [t.cpu().numpy() for t in ref]
    b.close()
    for call in range(2):
        out = [torch.full(s, 5.0 + call, dtype=torch.complex64, device="cuda") for s in shapes]
        harm.harm_batch_run_noalloc(scenes, out, zero_first=True)
        torch.cuda.synchronize()
        for w, t in zip(want, out):
            assert_iq(t.cpu().numpy(), w, TOL)
    for s in scenes:
        s.close()


def test_noalloc_64_scenes_and_accumulation():
    """The largest call (64 scenes: every argument slot and the ends of the work
    tables in the fixed array) against harm_batch_run, then a call with
    zero_first = 0 into prefilled outputs: prefill + echo."""
    import numpy as np
    import torch
    descs = []
    for i in range(64):
        d = hs.ati_scene(n_pulses=12 + (i % 5) * 4, nx=20 + (i % 7) * 6, ny=17 + (i % 3) * 9, n_range=256)
        d["speckle_seed"], d["u10"] = 500 + i, 4.0 + 0.15 * i
        descs.append(d)
    scenes = [harm.harm_scene_create(d, harm.HARM_PREC_MIXED) for d in descs]
    shapes = [(len(d["rx"]), d["n_pulses"], d["n_range"]) for d in descs]
    ref = [torch.zeros(s, dtype=torch.complex64, device="cuda") for s in shapes]
    b = harm.harm_batch_create(scenes)
    harm.harm_batch_run(b, ref)
    torch.cuda.synchronize()
    want = [t.cpu().numpy() for t in ref]
    b.close()
    out = [torch.full(s, 2.0, dtype=torch.complex64, device="cuda") for s in shapes]
    harm.harm_batch_run_noalloc(scenes, out, zero_first=True)
    torch.cuda.synchronize()
    for w, t in zip(want, out):
        assert_iq(t.cpu().numpy(), w, TOL)
    rng = np.random.default_rng(9)
    pre = [(rng.standard_normal(s) + 1j * rng.standard_normal(s)).astype(np.complex64) for s in shapes]
    out = [torch.tensor(p, device="cuda") for p in pre]
    harm.harm_batch_run_noalloc(scenes, out, zero_first=False)
    torch.cuda.synchronize()
    for w, p, t in zip(want, pre, out):
        assert_iq(t.cpu().numpy(), p + w, TOL)
    for s in scenes:
        s.close()


def test_noalloc_rejects_more_than_64_scenes():
    import torch
    d = _scenes()[0]
    sc = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    iq = torch.zeros((len(d["rx"]), d["n_pulses"], d["n_range"]), dtype=torch.complex64, device="cuda")
    with pytest.raises(harm.HarmError) as ei:
        harm.harm_batch_run_noalloc([sc] * 65, [iq] * 65)
    assert ei.value.status == harm.HARM_E_INVALID
    assert "64" in str(ei.value)
    sc.close()
