"""CPU checks of the C ABI: the library builds and loads, exports every function
include/harm.h declares, and the ctypes mirror of every struct has the C layout."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2405_09938_b300 import build as harm_build
from paper_2405_09938_b300 import harm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "harm.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(harm_[a-z_]+)\s*\(", src)))


def test_library_builds_and_loads():
    path = harm_build.build()
    assert os.path.exists(path)
    lib = harm.load_library(path)
    assert lib is not None


def test_every_declared_symbol_exported():
    lib = ctypes.CDLL(harm_build.build())
    names = _declared_functions()
    assert "harm_echo_accumulate" in names and "harm_scene_create" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(harm.SIGNATURES), "binding and header disagree"


def test_last_error_without_gpu_work():
    lib = harm.load_library(harm_build.build())
    assert isinstance(lib.harm_last_error(), bytes)


def _c_layout(struct, fields):
    code = ['#include <stdio.h>', '#include <stddef.h>', '#include "harm.h"', 'int main(void){',
            '  printf("%%zu\\n", sizeof(%s));' % struct]
    for f in fields:
        code.append('  printf("%%zu\\n", offsetof(%s, %s));' % (struct, f))
    code.append("  return 0; }")
    return "\n".join(code)


@pytest.mark.parametrize("name,cls", [("harm_scene_desc", harm.harm_scene_desc),
                                      ("harm_antenna", harm.harm_antenna),
                                      ("harm_scene_info", harm.harm_scene_info)])
def test_struct_layout_matches_header(tmp_path, name, cls):
    fields = [f[0] for f in cls._fields_]
    src = tmp_path / "layout.c"
    src.write_text(_c_layout(name, fields))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(cls)
    for f, off in zip(fields, out[1:]):
        assert getattr(cls, f).offset == off, f


def test_invalid_descriptor_rejected_without_device_work():
    """Validation runs on the host before any CUDA call."""
    import harm_scenes as hs
    lib = harm.load_library(harm_build.build())
    d = hs.small_static()
    s, keep = harm.make_desc(d, harm.HARM_PREC_FP64)
    s.struct_size = 12
    out = ctypes.c_void_p()
    st = lib.harm_scene_create(ctypes.byref(s), None, ctypes.byref(out))
    assert st == harm.HARM_E_INVALID
    assert b"struct_size" in lib.harm_last_error()
    assert out.value is None
    s, keep = harm.make_desc(d, harm.HARM_PREC_FP64)
    s.taps = 5
    assert lib.harm_scene_create(ctypes.byref(s), None, ctypes.byref(out)) == harm.HARM_E_UNSUPPORTED
    s, keep = harm.make_desc(d, harm.HARM_PREC_FP64)
    s.n_channels = 0
    assert lib.harm_scene_create(ctypes.byref(s), None, ctypes.byref(out)) == harm.HARM_E_INVALID
    s, keep = harm.make_desc(d, harm.HARM_PREC_FP64)
    s.tx.pos0[2] = -1.0
    assert lib.harm_scene_create(ctypes.byref(s), None, ctypes.byref(out)) == harm.HARM_E_INVALID
    assert lib.harm_scene_create(None, None, ctypes.byref(out)) == harm.HARM_E_INVALID
    # NULL scene handles
    assert lib.harm_echo_accumulate(None, 0, 1, None, 0, 1) == harm.HARM_E_INVALID
    assert lib.harm_scene_sync(None) == harm.HARM_E_INVALID
    assert lib.harm_scene_destroy(None) == harm.HARM_OK


def test_version_1_descriptor_and_variant_validation():
    """A version-1 descriptor (the prefix before the variant fields) passes
    validation; bad variant fields are rejected, all before any CUDA call."""
    import harm_scenes as hs
    lib = harm.load_library(harm_build.build())
    d = hs.small_static()
    out = ctypes.c_void_p()
    s, keep = harm.make_desc(d, harm.HARM_PREC_FP64)
    s.abi_version = 1
    s.struct_size = harm.harm_scene_desc.speckle_tau_s.offset
    st = lib.harm_scene_create(ctypes.byref(s), None, ctypes.byref(out))
    assert st != harm.HARM_E_INVALID, lib.harm_last_error()
    s.struct_size = ctypes.sizeof(harm.harm_scene_desc)  # a version-1 caller cannot send the longer struct
    assert lib.harm_scene_create(ctypes.byref(s), None, ctypes.byref(out)) == harm.HARM_E_INVALID
    s, keep = harm.make_desc(d, harm.HARM_PREC_FP64)
    s.abi_version = 3
    assert lib.harm_scene_create(ctypes.byref(s), None, ctypes.byref(out)) == harm.HARM_E_INVALID
    for field, value in [("speckle_tau_s", -1.0), ("cwm", 2), ("speckle_doppler_hz", float("nan"))]:
        s, keep = harm.make_desc(d, harm.HARM_PREC_FP64)
        setattr(s, field, value)
        assert lib.harm_scene_create(ctypes.byref(s), None, ctypes.byref(out)) == harm.HARM_E_INVALID, field
    # a corner grid that does not cover the patch (200 m patch, 2 x 2 corners of 150 m)
    dh = hs.hetero_sea(d, tile_m=150.0)
    dh["hetero"]["u10"] = dh["hetero"]["u10"][:2, :2]
    dh["hetero"]["wind_dir"] = dh["hetero"]["wind_dir"][:2, :2]
    s, keep = harm.make_desc(dh, harm.HARM_PREC_FP64)
    assert lib.harm_scene_create(ctypes.byref(s), None, ctypes.byref(out)) == harm.HARM_E_INVALID
    assert b"cover" in lib.harm_last_error()
    dh = hs.hetero_sea(d, tile_m=100.0)
    dh["hetero"]["u10"][0, 0] = 0.0
    s, keep = harm.make_desc(dh, harm.HARM_PREC_FP64)
    assert lib.harm_scene_create(ctypes.byref(s), None, ctypes.byref(out)) == harm.HARM_E_INVALID
    assert out.value is None
    # pattern setter on a NULL scene
    assert lib.harm_scene_set_pattern(None, -1, 2, 2, 0.0, 1.0, 0.0, 1.0, None) == harm.HARM_E_INVALID


def test_binding_rejects_bad_host_and_device_arguments():
    # argument marshalling checks of the binding run before any library call
    import torch
    harm.load_library(harm_build.build())

    class _NoScene:
        @property
        def handle(self):
            raise AssertionError("the scene must not be touched")

    sc = _NoScene()
    with pytest.raises(harm.HarmError) as e:
        harm.harm_echo_accumulate_host(sc, 0, 1, "not a tensor")
    assert e.value.status == harm.HARM_E_INVALID
    strided = torch.zeros((2, 4, 8), dtype=torch.complex64)[:, ::2, :]
    with pytest.raises(harm.HarmError) as e:
        harm.harm_echo_accumulate_host(sc, 0, 2, strided)
    assert "contiguous" in str(e.value)


    class _NullScene:
        handle = None  # the device-pointer check fails before the library is called

    with pytest.raises(harm.HarmError) as e:
        harm.harm_echo_accumulate(_NullScene(), 0, 1, torch.zeros(4, dtype=torch.complex64))  # a CPU tensor
    assert "CUDA" in str(e.value)


class _FakeCuda(__import__("torch").Tensor):
    """A CPU tensor that reports itself as a CUDA tensor on cuda:0, so that the
    binding's size and device checks can run without a GPU (the library is never
    called: every case below must be refused first)."""

    @property
    def is_cuda(self):
        return True

    @property
    def device(self):
        import torch
        return torch.device("cuda", 0)


def _fake(shape, dtype):
    import torch
    return torch.zeros(shape, dtype=dtype).as_subclass(_FakeCuda)


def test_binding_refuses_wrong_sized_or_misplaced_buffers():
    """Output and input tensors must hold exactly the elements the call touches,
    on the scene's device, before anything reaches the library (an undersized
    buffer would otherwise be written past its end on the device)."""
    import torch

    import harm_scenes as hs
    harm.load_library(harm_build.build())
    d = hs.ati_scene(n_pulses=16, nx=40, ny=20, n_range=256)

    class _Scene:
        desc = d
        precision = harm.HARM_PREC_MIXED
        device = 0
        _ncells = 8

        @property
        def handle(self):
            raise AssertionError("the library must not be called")

    sc = _Scene()
    nc, nr = len(d["rx"]), d["n_range"]
    cases = [
        lambda: harm.harm_echo_accumulate(sc, 0, 4, _fake((nc, 3, nr), torch.complex64)),
        lambda: harm.harm_echo_accumulate(sc, 0, 4, _fake((nc, 4, nr + 1), torch.complex128)),
        lambda: harm.harm_facets_generate(sc, 0, 2, _fake((2, 3, 20 * 40 - 1), torch.float32)),
        lambda: harm.harm_facets_generate(sc, 0, 2, _fake((2, 3, 20 * 40), torch.float64)),
        lambda: harm.harm_echo_adjoint(sc, 0, 4, _fake((nc, 4, nr - 1), torch.complex64)),
        lambda: harm.harm_echo_adjoint(sc, 0, 4, _fake((nc, 4, nr), torch.complex64),
                                       grad_sigma0=_fake((7,), torch.float64)),
        lambda: harm.harm_echo_adjoint(sc, 0, 4, _fake((nc, 4, nr), torch.complex64),
                                       grad_uv=_fake((8,), torch.float64)),
        lambda: harm.harm_scene_set_cells(sc, 4, 2, 10.0, _fake((9,), torch.float64), None),
        lambda: harm.harm_batch_run_noalloc([sc], [_fake((nc, 15, nr), torch.complex64)]),
        lambda: harm.harm_batch_run_noalloc([sc, sc], [_fake((nc, 16, nr), torch.complex64)]),
    ]
    for i, case in enumerate(cases):
        with pytest.raises(harm.HarmError) as e:
            case()
        assert e.value.status == harm.HARM_E_INVALID, i
    # a buffer of the right size on another device
    sc.device = 1
    with pytest.raises(harm.HarmError) as e:
        harm.harm_echo_accumulate(sc, 0, 4, _fake((nc, 4, nr), torch.complex64))
    assert "cuda:1" in str(e.value)


def test_peaks_library_exports_its_header():
    lib = ctypes.CDLL(harm_build.build_peaks())
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "harm_peaks.h")).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(harm_peak_[a-z_]+)\s*\(", src)))
    assert names == ["harm_peak_launch", "harm_peak_ops"]
    for name in names:
        assert hasattr(lib, name), name
    from paper_2405_09938_b300 import peaks
    pl = peaks.load_library()
    # operation counts of a launch: blocks x 256 threads x 8 chains x iterations
    assert pl.harm_peak_ops(0, 2, 3) == 2 * 2 * 256 * 8 * 3
    assert pl.harm_peak_ops(1, 2, 3) == 4 * 2 * 256 * 8 * 3
    assert pl.harm_peak_ops(3, 1, 1) == 256 * 8
    assert pl.harm_peak_ops(9, 1, 1) == 0
    assert pl.harm_peak_launch(0, 0, 1, None, None) == 1  # bad arguments: refused before any launch
