"""Bit-exact parity of the accumulator's integer work (harm_probe_indices) with the
FP64 oracle: the Philox4x32-10 words of every speckle draw (Eq. 7), the facet's
first range bin in every channel (Eq. 17 with the 8-tap or box kernel) and its cell
index. The probe runs the accumulator's own per-facet code (the same work items,
tile references, surface and ranges) up to the scatter.

Where the two sides take an integer from a real number (the range bin from the
fractional position p), they use different arithmetic (FP32 offsets from FP64
tile references against a direct FP64 range sum), so the bins agree exactly
except where p lies within the mixed path's position error of an integer; there
both floors are correct (the 8-tap kernel is zero at its ends, so the sum does
not depend on the choice) and the test checks that the GPU took one of them."""
import numpy as np
import pytest

import harm_scenes as hs
import oracle
from paper_2405_09938_b300 import harm

pytestmark = pytest.mark.gpu

# mixed path bin-position error: ~1e-6 m of range error (the 1e-4 rad phase
# budget over K0) is 2e-7 bins; 1e-5 bins leaves a wide margin
EPS_BIN = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _probe(d, n0, np_):
    sc = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    c = d.get("cells")
    if c is not None:
        import torch
        s0 = torch.tensor(c["sigma0"], dtype=torch.float64, device="cuda")
        uv = torch.tensor(c["uv"], dtype=torch.float64, device="cuda")
        harm.harm_scene_set_cells(sc, c["ncx"], c["ncy"], c["cell_m"], s0, uv)
    bins, spk, words, cells = harm.harm_probe_indices(sc, n0, np_)
    harm.harm_scene_sync(sc)
    out = (bins.cpu().numpy(), spk.cpu().numpy(), words.cpu().numpy().view(np.uint32), cells.cpu().numpy())
    sc.close()
    return out


def _check_bins(got, p, taps, eps=EPS_BIN):
    """got[i, c, iy, ix] against floor(p) - 3 (8 taps) or floor(p) (box): equal
    wherever p is further than eps from an integer, one of the two floors
    otherwise. Returns the number of such near-integer positions."""
    off = 3 if taps == 8 else 0
    want = np.floor(p).astype(np.int64) - off
    near = np.abs(p - np.rint(p)) < eps
    exact = ~near
    assert np.array_equal(got[exact], want[exact]), \
        "bins differ at %d of %d positions" % (int(np.sum(got[exact] != want[exact])), int(exact.sum()))
    lo = np.floor(p - eps).astype(np.int64) - off
    hi = np.floor(p + eps).astype(np.int64) - off
    g = got[near]
    assert np.all((g == lo[near]) | (g == hi[near]))
    return int(near.sum())


def _check_words_and_speckle(d, n0, np_, spk, words):
    nx, ny = d["nx"], d["ny"]
    ep = d["epoch_pulses"]
    fid = np.arange(nx * ny, dtype=np.uint32)
    for i in range(np_):
        e = (n0 + i) // ep if ep > 0 else 0
        want = oracle.speckle_words(d["speckle_seed"], fid, e)
        assert np.array_equal(words[i].reshape(-1, 4), want), "Philox words differ at pulse %d" % (n0 + i)
    # the FP32 Box-Muller draw against the oracle's FP64 draw (a sample of facets)
    for i in (0, np_ - 1):
        e = (n0 + i) // ep if ep > 0 else 0
        for f in range(0, nx * ny, max(1, nx * ny // 97)):
            z = oracle.speckle(d["speckle_seed"], f, e)
            assert abs(complex(spk[i].reshape(-1)[f]) - z) < 2e-6 * max(1.0, abs(z))


def test_indices_wave_scene_six_channels():
    # headline instantiation (six channels, two antennas of three phase centres),
    # a grid ragged in both directions, a new speckle epoch every pulse (so the
    # window draws 150 x 200 x 40 = 1.2e6 Philox counters) and a pulse window
    # crossing the edge of the 256-pulse time-Taylor windows
    d = hs.ati_scene(n_pulses=300, nx=200, ny=150, n_range=2048)
    d["epoch_pulses"] = 1
    n0, np_ = 236, 40
    bins, spk, words, cells = _probe(d, n0, np_)
    p, cells_o = oracle.bin_positions(d, list(range(n0, n0 + np_)))
    near = _check_bins(bins, p, 8)
    print("6-channel wave scene: %d bins compared, %d within %.0e of an integer" % (bins.size, near, EPS_BIN))
    _check_words_and_speckle(d, n0, np_, spk, words)
    assert np.array_equal(cells, cells_o)  # -1: no cells


def test_indices_box_taps_three_channels_and_cells():
    # the Eq. 17 box, the general channel loop (one antenna, three phase centres)
    # and per-cell fields on 14 m cells (not a multiple of the 2 m facets)
    d = hs.ati_scene(n_pulses=64, nx=70, ny=45, n_range=1024)
    tx, rx = hs.geometry(d["n_pulses"], ("A",), (-5.0, 0.0, 5.0))
    d["tx"], d["rx"] = tx, rx
    d["taps"] = 1
    ncx, ncy = 10, 7
    d["cells"] = {"ncx": ncx, "ncy": ncy, "cell_m": 14.0, "sigma0": np.full((ncy, ncx), 0.02),
                  "uv": np.tile(np.array([0.5, 0.2]), (ncy, ncx, 1))}
    n0, np_ = 0, 64
    bins, spk, words, cells = _probe(d, n0, np_)
    p, cells_o = oracle.bin_positions(d, list(range(n0, n0 + np_)))
    _check_bins(bins, p, 1)
    _check_words_and_speckle(d, n0, np_, spk, words)
    assert np.array_equal(cells, cells_o)
    assert cells.min() == 0 and cells.max() == ncx * ncy - 1


def test_indices_static_patch_one_channel():
    d = hs.small_static()
    bins, spk, words, cells = _probe(d, 0, 64)
    p, _ = oracle.bin_positions(d, list(range(64)))
    _check_bins(bins, p, 8)
    _check_words_and_speckle(d, 0, 64, spk, words)


@pytest.mark.parametrize("prec,eps", [("fp64", 1e-9), ("fp32", 2e-3)])
def test_indices_plain_paths(prec, eps):
    """The plain accumulators' integer work: Philox words bit-exact, bins exact
    away from the path's own position error (FP64: ~1e-12 bins; FP32: rounding of
    the range offsets, ~1e-4 bins here), cells exact."""
    p_ = harm.HARM_PREC_FP64 if prec == "fp64" else harm.HARM_PREC_FP32
    d = hs.ati_scene(n_pulses=80, nx=70, ny=45, n_range=1024)
    d["epoch_pulses"] = 3
    ncx, ncy = 9, 6
    d["cells"] = {"ncx": ncx, "ncy": ncy, "cell_m": 16.0, "sigma0": np.full((ncy, ncx), 0.02),
                  "uv": np.tile(np.array([0.5, 0.2]), (ncy, ncx, 1))}
    sc = harm.harm_scene_create(d, p_)
    import torch
    s0 = torch.tensor(d["cells"]["sigma0"], dtype=torch.float64, device="cuda")
    uv = torch.tensor(d["cells"]["uv"], dtype=torch.float64, device="cuda")
    harm.harm_scene_set_cells(sc, ncx, ncy, 16.0, s0, uv)
    n0, np_ = 17, 30
    bins, spk, words, cells = harm.harm_probe_indices(sc, n0, np_)
    harm.harm_scene_sync(sc)
    bins, spk = bins.cpu().numpy(), spk.cpu().numpy()
    words, cells = words.cpu().numpy().view(np.uint32), cells.cpu().numpy()
    sc.close()
    p, cells_o = oracle.bin_positions(d, list(range(n0, n0 + np_)))
    near = _check_bins(bins, p, 8, eps)
    print("plain %s: %d bins, %d within %.0e of an integer" % (prec, bins.size, near, eps))
    _check_words_and_speckle(d, n0, np_, spk, words)
    assert np.array_equal(cells, cells_o)
