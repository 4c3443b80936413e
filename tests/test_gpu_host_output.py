"""Echo into host memory (harm_echo_accumulate_host): pulse blocks computed into
the scene's device ring and copied to a page-locked host array on a second
stream. Checked against the device-output call on the same scene (same kernels,
same work items; only the atomic order differs) and against the FP64 oracle on
sampled pulses, for ragged blocks, an offset window, both output types, a ring
that grows between calls, and pageable memory (rejected).
"""
import numpy as np
import pytest

import harm_scenes as hs
import oracle
from paper_2405_09938_b300 import harm
from tests.gpu_util import assert_iq, rel_rms, run_echo

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-4
TOL_SAME_KERNEL = 2e-6  # two runs of the mixed path: FP32 atomic order only


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _scene():
    return hs.ati_scene(n_pulses=300, nx=40, ny=32, n_range=1024)


def _host_echo(scene, d, n0, np_, dtype, block):
    import torch
    out = torch.empty((len(d["rx"]), np_, d["n_range"]), dtype=dtype, pin_memory=True)
    out.fill_(complex(float("nan"), 0.0))  # every element must be written
    harm.harm_echo_accumulate_host(scene, n0, np_, out, block_pulses=block)
    harm.harm_scene_sync(scene)
    return out.numpy().copy()


@pytest.mark.parametrize("block", [100, 64, 0])
def test_host_output_matches_device_output_ragged_blocks(block):
    import torch
    d = _scene()
    n0, np_ = 20, 250
    sc = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    got = _host_echo(sc, d, n0, np_, torch.complex64, block)
    want = run_echo(d, harm.HARM_PREC_MIXED, n0, np_, dtype="c64", scene=sc)
    sc.close()
    assert np.isfinite(got).all()
    err, pe = assert_iq(got, want, TOL_SAME_KERNEL)
    print("block %d: host vs device output rel RMS %.2e, per-element %.2e" % (block, err, pe))
    for c in range(len(d["rx"])):
        assert_iq(got[c], want[c], TOL_SAME_KERNEL)


def test_host_output_complex128_against_oracle():
    import torch
    d = _scene()
    n0, np_ = 0, 300
    sc = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    got = _host_echo(sc, d, n0, np_, torch.complex128, 0)
    sc.close()
    pulses = [0, 127, 128, 255, 256, 299]  # inside and at the edge of the default 256-pulse block, and the tail
    want = oracle.echo(d, pulses)
    err, pe = assert_iq(got[:, pulses, :], want, TOL_MIXED)
    print("host output (complex128) vs oracle: rel RMS %.2e, per-element %.2e" % (err, pe))


def test_host_output_ring_grows_and_is_reused():
    import torch
    d = _scene()
    sc = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    a = _host_echo(sc, d, 10, 40, torch.complex64, 16)     # small ring
    b = _host_echo(sc, d, 0, 300, torch.complex64, 200)    # grows it
    c = _host_echo(sc, d, 10, 40, torch.complex64, 16)     # reuses the large ring
    sc.close()
    assert_iq(a, c, TOL_SAME_KERNEL)
    assert_iq(b[:, 10:50, :], a, TOL_SAME_KERNEL)


def test_host_output_rejects_pageable_memory():
    import torch
    d = _scene()
    sc = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    out = torch.empty((len(d["rx"]), 8, d["n_range"]), dtype=torch.complex64)  # not pinned
    with pytest.raises(harm.HarmError) as e:
        harm.harm_echo_accumulate_host(sc, 0, 8, out)
    assert e.value.status == harm.HARM_E_INVALID
    assert "page-locked" in str(e.value)
    # the scene stays usable
    pinned = torch.empty_like(out).pin_memory()
    harm.harm_echo_accumulate_host(sc, 0, 8, pinned)
    harm.harm_scene_sync(sc)
    sc.close()
    assert np.isfinite(pinned.numpy()).all()


def test_host_output_fp64_scene():
    import torch
    d = hs.small_static()
    sc = harm.harm_scene_create(d, harm.HARM_PREC_FP64)
    got = _host_echo(sc, d, 0, 64, torch.complex128, 24)
    sc.close()
    want = oracle.echo(d, list(range(64)))
    assert_iq(got, want, 1e-7)


def test_host_output_window_checks():
    import torch
    d = _scene()
    sc = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    out = torch.empty((len(d["rx"]), 8, d["n_range"]), dtype=torch.complex64, pin_memory=True)
    with pytest.raises(harm.HarmError) as e:
        harm.harm_echo_accumulate_host(sc, d["n_pulses"] - 4, 8, out)  # runs past the burst
    assert e.value.status == harm.HARM_E_INVALID
    out.fill_(complex(7.0, 7.0))
    harm.harm_echo_accumulate_host(sc, 0, 0, out)  # empty window: nothing written
    harm.harm_scene_sync(sc)
    sc.close()
    assert (out.numpy() == np.complex64(7 + 7j)).all()
