"""Host-side logic of bench.py (no GPU): the traffic figure is tied to the kernel
code it was captured on, not to its comments, and the uploaded-bytes count of the
end-to-end leg follows the scene."""
import bench
import harm_scenes as hs
from paper_2405_09938_b300 import harm


def test_code_lines_ignore_comments_and_blank_lines():
    a = b"int x = 1;  // one\n\n// a comment line\nint y = 2;\n"
    b = b"int x = 1;\nint y = 2;   // two\n"
    assert bench._code_lines(a) == bench._code_lines(b)
    assert bench._code_lines(b"int x = 1;\n") != bench._code_lines(b"int x = 2;\n")


def test_traffic_only_for_the_captured_launch():
    assert bench.captured_traffic(bench.TRAFFIC_PULSES + 1) is None
    t = bench.captured_traffic(bench.TRAFFIC_PULSES)
    assert t is None or t == float(bench.TRAFFIC_BYTES)


def test_uploaded_bytes_follow_the_scene():
    mixed, fp64 = harm.HARM_PREC_MIXED, harm.HARM_PREC_FP64
    d = hs.ati_scene(n_pulses=256, nx=64, ny=32, n_range=512)
    nw = d["n_omega"] * d["n_theta"]
    base = bench._scene_table_bytes(d, mixed, 256)
    # the mixed path's time-Taylor tables: one complex64 batch-centre phasor per
    # window and wave, 3 fields x 6 orders of float32 factors per wave, tau per pulse
    assert base - bench._scene_table_bytes(d, fp64, 256) == nw * 8 + nw * 3 * 6 * 4 + 256 * 4
    # half-length windows add one more phasor table
    assert bench._scene_table_bytes(d, mixed, 128) - base == nw * 8
    # 256 more pulses: a pulse record (2 + 10 doubles), 6 receive records
    # (10 + 2 doubles), tau, and one more window
    d2 = hs.ati_scene(n_pulses=512, nx=64, ny=32, n_range=512)
    assert bench._scene_table_bytes(d2, mixed, 256) - base == 256 * (96 + 6 * 96 + 4) + nw * 8
    # the Choppy Wave Model carries 8 fields
    assert bench._scene_table_bytes(hs.choppy(d), mixed, 256) - base == nw * 5 * 6 * 4
    # a heterogeneous sea state uploads one wave set per corner of its tile grid
    h = hs.hetero_sea(d, tile_m=100.0)
    sets = h["hetero"]["u10"].size
    assert sets > 1
    assert bench._scene_table_bytes(h, fp64, 256) - bench._scene_table_bytes(d, fp64, 256) == (sets - 1) * nw * 72
