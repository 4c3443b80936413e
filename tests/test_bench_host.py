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


def test_uploaded_bytes_grow_with_pulses():
    d = hs.ati_scene(n_pulses=256, nx=64, ny=32, n_range=512)
    small = bench._scene_table_bytes(d, harm.HARM_PREC_MIXED)
    d2 = hs.ati_scene(n_pulses=512, nx=64, ny=32, n_range=512)
    assert bench._scene_table_bytes(d2, harm.HARM_PREC_MIXED) > small > 0
