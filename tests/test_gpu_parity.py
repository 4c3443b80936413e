"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded scenes, element by element.

Tolerances (IQ relative RMS over all compared samples):
  * FP64 path: 1e-7. The only differences are rounding order, the offset form of
    the ranges and the wave phasor tables; the bound on the path is 1e-5.
  * Mixed path: 1e-4 (FP32 phase, patterns, taps and accumulation).
"""
import numpy as np
import pytest

import harm_scenes as hs
import oracle
from paper_2405_09938_b300 import harm
from tests.gpu_util import assert_iq, ati_phase_bias, rel_rms, run_echo, run_states

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-7
TOL_MIXED = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()


def small_wave_scene(n_pulses=64, nx=48, ny=40, n_range=1024):
    return hs.ati_scene(n_pulses=n_pulses, nx=nx, ny=ny, n_range=n_range)


# ------------------------------------------------------------------ generator
def test_generator_fp64_matches_oracle():
    d = small_wave_scene(n_pulses=64, nx=37, ny=23)
    got = run_states(d, harm.HARM_PREC_FP64, 10, 5)
    for i, n in enumerate(range(10, 15)):
        want = oracle.facet_states(d, n)
        assert np.abs(got[i] - want).max() < 1e-11


def test_generator_mixed_matches_oracle():
    d = small_wave_scene(n_pulses=100, nx=70, ny=33)
    got = run_states(d, harm.HARM_PREC_MIXED, 30, 40)
    for i, n in [(0, 30), (1, 31), (17, 47), (39, 69)]:
        want = oracle.facet_states(d, n)
        err = np.abs(got[i] - want)
        assert err[0].max() < 2e-6      # height [m]
        assert err[1:].max() < 2e-6     # slopes


def test_generator_mixed_many_items_per_cta():
    """More work items (tiles x pulse windows) than twice the persistent grid of
    the linear-surface generator: CTAs take three items in turn, so both
    coefficient buffers are filled, released and refilled. Ragged tiles (300 x
    170 facets) and a ragged first and last window (pulses 5 .. 1294)."""
    import torch
    from tests.gpu_util import take_pulses
    d = small_wave_scene(n_pulses=1300, nx=300, ny=170)
    n0, np_ = 5, 1290
    scene = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    nb = harm.harm_scene_query(scene)["pulse_batch"]
    tiles = -(-300 // 32) * -(-170 // 16)
    windows = (n0 + np_ - 1) // nb - n0 // nb + 1
    assert tiles * windows > 2 * 2 * torch.cuda.get_device_properties(0).multi_processor_count
    st = torch.full((np_, 3, 170, 300), float("nan"), dtype=torch.float32, device="cuda")
    harm.harm_facets_generate(scene, n0, np_, st)
    harm.harm_scene_sync(scene)
    pulses = [5, nb - 1, nb, 700, 1024, 1294]
    got = take_pulses(st.reshape(np_, 1, -1).transpose(0, 1), [p - n0 for p in pulses])
    scene.close()
    assert not torch.isnan(st).any()
    for i, n in enumerate(pulses):
        want = oracle.facet_states(d, n).reshape(3, -1)
        err = np.abs(got[0, i].reshape(3, -1).astype(np.float64) - want)
        assert err[0].max() < 2e-6
        assert err[1:].max() < 2e-6


@pytest.mark.parametrize("nx,ny,n0,np_", [(4, 3, 3, 1), (4, 3, 250, 9), (68, 21, 0, 37)])
def test_generator_tensor_store_kernel_edges(nx, ny, n0, np_):
    """The tensor-store generator (nx % 4 == 0) on a scene smaller than one tile,
    a single pulse, a request that crosses a 256-pulse window, and ragged tiles;
    then the same request into a state array that starts 4 bytes into its
    allocation, which takes the direct-store kernel: the two kernels run the same
    arithmetic, so their states agree bit for bit."""
    import torch
    d = small_wave_scene(n_pulses=300, nx=nx, ny=ny)
    scene = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    n = np_ * 3 * ny * nx
    st = torch.full((np_, 3, ny, nx), float("nan"), dtype=torch.float32, device="cuda")
    harm.harm_facets_generate(scene, n0, np_, st)
    flat = torch.full((n + 1,), float("nan"), dtype=torch.float32, device="cuda")
    off = flat[1:]
    assert off.data_ptr() % 16 == 4
    harm.harm_facets_generate(scene, n0, np_, off)
    harm.harm_scene_sync(scene)
    got = st.cpu().numpy()
    other = off.cpu().numpy().reshape(np_, 3, ny, nx)
    scene.close()
    assert not np.isnan(got).any()
    assert np.array_equal(got.view(np.uint32), other.view(np.uint32))
    for p in sorted({0, np_ // 2, np_ - 1}):
        want = oracle.facet_states(d, n0 + p)
        assert np.abs(got[p].astype(np.float64) - want).max() < 2e-6


def test_generator_static_surface_is_flat():
    """A static surface (100 x 100 facets, nx % 4 == 0: the tensor-store kernel)
    has zero height and slopes at every pulse: every state written, every one 0."""
    import torch
    d = hs.small_static()
    scene = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    st = torch.full((7, 3, d["ny"], d["nx"]), float("nan"), dtype=torch.float32, device="cuda")
    harm.harm_facets_generate(scene, 20, 7, st)
    harm.harm_scene_sync(scene)
    got = st.cpu().numpy()
    scene.close()
    assert np.array_equal(got, np.zeros_like(got))


# ------------------------------------------------------------------ FP64 path
@pytest.mark.parametrize("taps", [8, 1])
def test_static_patch_fp64(taps):
    d = hs.small_static()
    d["taps"] = taps
    got = run_echo(d, harm.HARM_PREC_FP64, 0, 64, "c128")
    want = oracle.echo(d, list(range(64)))
    assert_iq(got, want, TOL_FP64)


def test_wave_scene_fp64_all_channels():
    d = small_wave_scene()
    got = run_echo(d, harm.HARM_PREC_FP64, 0, 64, "c128")
    want = oracle.echo(d, list(range(64)))
    assert got.shape == want.shape == (6, 64, 1024)
    assert_iq(got, want, TOL_FP64)
    for c in range(6):
        assert_iq(got[c], want[c], TOL_FP64)


def test_fp64_path_c64_output():
    d = hs.small_static()
    got = run_echo(d, harm.HARM_PREC_FP64, 0, 64, "c64")
    want = oracle.echo(d, list(range(64)))
    assert_iq(got, want, 1e-6)


# ------------------------------------------------------------------ plain FP32 path
def test_wave_scene_fp32_plain_error():
    """The plain method in FP32: same kernel structure as the FP64 path, every
    per-facet step in float. Its error is set by FP32 rounding of the range offsets
    and of the phase K0 (r - R) over this 96 x 80 m patch (measured on a B300:
    2.2e-4); the bound below is that figure with margin, not the mixed path's."""
    d = small_wave_scene()
    got = run_echo(d, harm.HARM_PREC_FP32, 0, 64, "c64")
    want = oracle.echo(d, list(range(64)))
    err = rel_rms(got, want)
    print("small wave scene, plain FP32: IQ rel RMS %.3e" % err)
    assert err < 1e-3


def test_fp32_plain_states_and_window():
    # the plain FP32 generator against the oracle's states, and a ragged grid with
    # an unaligned pulse window through the FP32 accumulator (c128 output)
    d = small_wave_scene(n_pulses=100, nx=45, ny=19)
    got = run_states(d, harm.HARM_PREC_FP32, 30, 4)
    for i, n in enumerate(range(30, 34)):
        want = oracle.facet_states(d, n)
        assert np.abs(got[i] - want).max() < 2e-5
    n0, np_ = 41, 23
    got = run_echo(d, harm.HARM_PREC_FP32, n0, np_, "c128")
    want = oracle.echo(d, list(range(n0, n0 + np_)))
    assert rel_rms(got, want) < 1e-3


# ------------------------------------------------------------------ mixed path
@pytest.mark.parametrize("taps", [8, 1])
def test_static_patch_mixed(taps):
    d = hs.small_static()
    d["taps"] = taps
    got = run_echo(d, harm.HARM_PREC_MIXED, 0, 64, "c64")
    want = oracle.echo(d, list(range(64)))
    assert_iq(got, want, TOL_MIXED)


def test_wave_scene_mixed_errors():
    d = small_wave_scene()
    got = run_echo(d, harm.HARM_PREC_MIXED, 0, 64, "c64")
    want = oracle.echo(d, list(range(64)))
    assert_iq(got, want, TOL_MIXED)
    for sat in (0, 3):
        for a, b in ((0, 1), (1, 2), (0, 2)):
            assert abs(ati_phase_bias(got, want, sat + a, sat + b)) < 1e-4


def test_mixed_c128_output():
    d = small_wave_scene(n_pulses=40)
    got = run_echo(d, harm.HARM_PREC_MIXED, 0, 40, "c128")
    want = oracle.echo(d, list(range(40)))
    assert_iq(got, want, TOL_MIXED)


# ------------------------------------------------------------------ edges
def test_ragged_grid_and_unaligned_pulse_window():
    # grid not a multiple of the tiles; the pulse window crosses the edge of the
    # 256-pulse time-Taylor windows (256) and two speckle epoch edges (238, 272)
    d = small_wave_scene(n_pulses=300, nx=45, ny=19)
    n0, np_ = 233, 45
    want = oracle.echo(d, list(range(n0, n0 + np_)))
    for prec, tol, dt in ((harm.HARM_PREC_FP64, TOL_FP64, "c128"), (harm.HARM_PREC_MIXED, TOL_MIXED, "c64")):
        got = run_echo(d, prec, n0, np_, dt)
        assert_iq(got, want, tol)


def test_sixteen_channels_maximum():
    # the channel maximum: Harmony A and B with 8 phase centres each (a 16-channel
    # scene needs more shared memory per CTA than two CTAs per SM allow)
    pcs = tuple(5.0 * (i - 3.5) for i in range(8))
    d = small_wave_scene(n_pulses=40, nx=70, ny=33, n_range=1024)
    d["tx"], d["rx"] = hs.geometry(40, ("A", "B"), pcs)
    assert len(d["rx"]) == harm.HARM_MAX_CHANNELS
    pulses = [0, 17, 39]
    want = oracle.echo(d, pulses)
    for prec, tol, dt in ((harm.HARM_PREC_FP64, TOL_FP64, "c128"), (harm.HARM_PREC_MIXED, TOL_MIXED, "c64")):
        got = run_echo(d, prec, 0, 40, dt)[:, pulses, :]
        assert_iq(got, want, tol)
        for c in range(16):
            assert_iq(got[c], want[c], tol)


def test_six_channels_without_shared_antennas():
    # six channels whose phase centres are 100 m apart (more than the 50 m that
    # makes them one antenna): no pattern / NRCS sharing, the six-channel
    # instantiation with the sharing mask read at run time
    pcs = (-100.0, 0.0, 100.0)
    d = small_wave_scene(n_pulses=40, nx=70, ny=33, n_range=1024)
    d["tx"], d["rx"] = hs.geometry(40, ("A", "B"), pcs)
    pulses = [0, 17, 39]
    want = oracle.echo(d, pulses)
    got = run_echo(d, harm.HARM_PREC_MIXED, 0, 40, "c64")[:, pulses, :]
    assert_iq(got, want, TOL_MIXED)
    for c in range(6):
        assert_iq(got[c], want[c], TOL_MIXED)


def test_echo_partly_outside_range_window():
    # a short range window cuts the echo: taps outside [0, n_range) are dropped
    d = small_wave_scene(n_pulses=16, nx=64, ny=64, n_range=1024)
    full = oracle.echo(d, list(range(16)))
    nz = np.nonzero(np.abs(full).sum(axis=(0, 1)))[0]
    lo, hi = nz.min(), nz.max()
    # a window narrower than the echo (R0 = R_ref - n_range/2 dr stays centred)
    cut = dict(d, n_range=max(8, int((hi - lo) // 2)))
    want = oracle.echo(cut, list(range(16)))
    assert np.abs(want[:, :, 0]).max() > 0 and np.abs(want[:, :, -1]).max() > 0
    for prec, tol, dt in ((harm.HARM_PREC_FP64, TOL_FP64, "c128"), (harm.HARM_PREC_MIXED, TOL_MIXED, "c64")):
        got = run_echo(cut, prec, 0, 16, dt)
        assert_iq(got, want, tol)


def test_single_facet_and_single_pulse():
    d = hs.small_static(n_pulses=3)
    d.update(nx=1, ny=1)
    want = oracle.echo(d, [2])
    for prec, tol, dt in ((harm.HARM_PREC_FP64, TOL_FP64, "c128"), (harm.HARM_PREC_MIXED, TOL_MIXED, "c64")):
        got = run_echo(d, prec, 2, 1, dt)
        assert_iq(got, want, tol)


def test_scene_query_reports_the_scene():
    d = small_wave_scene(n_pulses=300, nx=45, ny=19)
    for prec, batch in ((harm.HARM_PREC_MIXED, 256), (harm.HARM_PREC_FP64, 0)):
        sc = harm.harm_scene_create(d, prec)
        info = harm.harm_scene_query(sc)
        sc.close()
        assert (info["n_facets"], info["n_pulses"], info["n_range"]) == (45 * 19, 300, d["n_range"])
        assert (info["n_channels"], info["n_waves"]) == (len(d["rx"]), d["n_omega"] * d["n_theta"])
        assert (info["precision"], info["pulse_batch"]) == (prec, batch)
        assert abs(info["range_bin_m"] - 299792458.0 / d["fs_hz"]) < 1e-12
        want = [oracle.range_start(d, c) for c in range(len(d["rx"]))]
        assert np.allclose(info["range_start_m"], want, rtol=0, atol=1e-6)


def test_empty_window_is_noop():
    import torch
    d = hs.small_static()
    scene = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    iq = torch.full((1, 1, 512), 7.0, dtype=torch.complex64, device="cuda")
    harm.harm_echo_accumulate(scene, 5, 0, iq)
    harm.harm_scene_sync(scene)
    assert torch.all(iq == 7.0)
    scene.close()


def test_accumulate_without_zeroing_adds():
    import torch
    d = hs.small_static()
    scene = harm.harm_scene_create(d, harm.HARM_PREC_FP64)
    iq = torch.zeros((1, 8, 512), dtype=torch.complex128, device="cuda")
    harm.harm_echo_accumulate(scene, 0, 8, iq, zero_first=True)
    harm.harm_echo_accumulate(scene, 0, 8, iq, zero_first=False)
    harm.harm_scene_sync(scene)
    want = oracle.echo(d, list(range(8)))
    assert_iq(iq.cpu().numpy(), 2 * want, TOL_FP64)
    scene.close()


def test_bad_calls_raise():
    import torch
    d = hs.small_static()
    scene = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    iq = torch.zeros((1, 4, 512), dtype=torch.complex64, device="cuda")
    with pytest.raises(harm.HarmError):
        harm.harm_echo_accumulate(scene, 62, 4, iq)  # beyond the burst
    with pytest.raises(harm.HarmError):
        harm.harm_echo_accumulate(scene, 0, 4, iq.cpu())
    with pytest.raises(harm.HarmError):
        harm.harm_echo_accumulate(scene, 0, 4, torch.zeros((1, 4, 512), device="cuda"))
    with pytest.raises(harm.HarmError):
        harm.harm_echo_adjoint(scene, 0, 4, iq)  # no cells set
    scene.close()


def test_repeat_runs_agree():
    d = small_wave_scene(n_pulses=32)
    a = run_echo(d, harm.HARM_PREC_MIXED, 0, 32, "c64")
    b = run_echo(d, harm.HARM_PREC_MIXED, 0, 32, "c64")
    assert_iq(a, b, 1e-6)


# ------------------------------------------------------------------ deterministic sums
def _det_run(d, prec, n0, np_, scene=None, zero_first=True, iq=None):
    import torch
    sc = scene or harm.harm_scene_create(d, prec)
    harm.harm_scene_set_deterministic(sc, True)
    if iq is None:
        iq = torch.zeros((len(d["rx"]), np_, d["n_range"]), dtype=torch.complex128, device="cuda")
    harm.harm_echo_accumulate(sc, n0, np_, iq, zero_first=zero_first)
    harm.harm_scene_sync(sc)
    out = iq.cpu().numpy()
    if scene is None:
        sc.close()
    return out, iq


@pytest.mark.parametrize("prec", [harm.HARM_PREC_FP64, harm.HARM_PREC_FP32])
def test_deterministic_sums_are_bit_identical(prec):
    """Fixed-point (integer-atomic) sums of the plain paths: two runs give the same
    bits, the second of two accumulating runs is exactly twice the first, and the
    result keeps the path's accuracy against the oracle. This is the run-to-run
    race check of the accumulator (floating-point atomics agree only to rounding)."""
    import torch
    d = small_wave_scene(n_pulses=48, nx=45, ny=37)
    want = oracle.echo(d, list(range(5, 37)))
    sc = harm.harm_scene_create(d, prec)
    a, _ = _det_run(d, prec, 5, 32, scene=sc)
    b, iq = _det_run(d, prec, 5, 32, scene=sc)
    assert a.tobytes() == b.tobytes()
    c, _ = _det_run(d, prec, 5, 32, scene=sc, zero_first=False, iq=iq)
    assert c.tobytes() == (2 * a).tobytes()
    tol = TOL_FP64 if prec == harm.HARM_PREC_FP64 else 1e-3
    assert_iq(a, want, tol)
    # the floating-point atomics of the default mode: same result to rounding (the
    # fixed point rounds each of the ~700 contributions of a bin by up to 2^-41,
    # ~1e-11 of the bin's magnitude after the random walk; measured 5.2e-12)
    harm.harm_scene_set_deterministic(sc, False)
    f = run_echo(d, prec, 5, 32, "c128", scene=sc)
    assert rel_rms(f, a) < (1e-10 if prec == harm.HARM_PREC_FP64 else 1e-6)
    # complex64 output cannot hold the fixed-point sums
    harm.harm_scene_set_deterministic(sc, True)
    with pytest.raises(harm.HarmError) as e:
        harm.harm_echo_accumulate(sc, 5, 32, torch.zeros((6, 32, d["n_range"]), dtype=torch.complex64, device="cuda"))
    assert e.value.status == harm.HARM_E_UNSUPPORTED
    # the host-output path runs the same deterministic accumulator per block
    host = torch.zeros((6, 32, d["n_range"]), dtype=torch.complex128, pin_memory=True)
    harm.harm_echo_accumulate_host(sc, 5, 32, host, block_pulses=12)
    harm.harm_scene_sync(sc)
    assert host.numpy().tobytes() == a.tobytes()
    sc.close()


def test_deterministic_mode_refused_for_mixed_scene():
    sc = harm.harm_scene_create(small_wave_scene(n_pulses=8, nx=16, ny=16), harm.HARM_PREC_MIXED)
    with pytest.raises(harm.HarmError) as e:
        harm.harm_scene_set_deterministic(sc, True)
    assert e.value.status == harm.HARM_E_UNSUPPORTED
    harm.harm_scene_set_deterministic(sc, False)
    sc.close()
