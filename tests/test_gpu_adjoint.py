"""GPU adjoint (harm_echo_adjoint and the torch.autograd wrapper) against the
oracle's FP64 adjoint and against central finite differences of the oracle's
FP64 forward (h = 1e-4 m/s) on 16 cells."""
import math

import numpy as np
import pytest

import harm_scenes as hs
import oracle
from paper_2405_09938_b300 import harm

pytestmark = pytest.mark.gpu

TOL_GRAD = 2e-3  # relative to the largest gradient component (FP32 forward / adjoint)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _scene(n_pulses=40, nx=96, ny=64, cell_m=16.0, taps=8, seed=5):
    d = hs.ati_scene(n_pulses=n_pulses, nx=nx, ny=ny, n_range=512)
    d["taps"] = taps
    ncx = int(math.ceil(nx * d["facet_m"] / cell_m))
    ncy = int(math.ceil(ny * d["facet_m"] / cell_m))
    rng = np.random.default_rng(seed)
    d["cells"] = {"ncx": ncx, "ncy": ncy, "cell_m": cell_m,
                  "sigma0": 0.02 * (1 + 0.3 * rng.random((ncy, ncx))),
                  "uv": np.stack([0.5 + 0.1 * rng.standard_normal((ncy, ncx)),
                                  0.2 + 0.1 * rng.standard_normal((ncy, ncx))], axis=-1)}
    return d


def _perturbed(d, seed=6):
    rng = np.random.default_rng(seed)
    t = dict(d)
    c = dict(d["cells"])
    c["sigma0"] = d["cells"]["sigma0"] * (1 + 0.2 * rng.random(c["sigma0"].shape))
    c["uv"] = d["cells"]["uv"] + 0.1 * rng.standard_normal(c["uv"].shape)
    t["cells"] = c
    return t


def _gpu_adjoint(d, n0, np_, resid, rdtype=None):
    import torch
    rdtype = rdtype or torch.complex64
    scene = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    c = d["cells"]
    s0 = torch.tensor(c["sigma0"], dtype=torch.float64, device="cuda")
    uv = torch.tensor(c["uv"], dtype=torch.float64, device="cuda")
    harm.harm_scene_set_cells(scene, c["ncx"], c["ncy"], c["cell_m"], s0, uv)
    r = torch.tensor(resid, dtype=rdtype, device="cuda")
    gs = torch.zeros_like(s0)
    guv = torch.zeros_like(uv)
    harm.harm_echo_adjoint(scene, n0, np_, r, gs, guv)
    harm.harm_scene_sync(scene)
    out = gs.cpu().numpy(), guv.cpu().numpy()
    scene.close()
    return out


@pytest.mark.parametrize("taps", [8, 1])
def test_adjoint_matches_oracle_adjoint(taps):
    d = _scene(taps=taps)
    pulses = list(range(0, 40))
    tgt = oracle.echo(_perturbed(d), pulses)
    r = oracle.echo(d, pulses) - tgt
    gs_o, guv_o = oracle.adjoint(d, pulses, r)
    gs_g, guv_g = _gpu_adjoint(d, 0, 40, r)
    assert np.abs(gs_g - gs_o).max() <= TOL_GRAD * np.abs(gs_o).max()
    assert np.abs(guv_g - guv_o).max() <= TOL_GRAD * np.abs(guv_o).max()
    # relative 2-norm error
    assert np.linalg.norm(guv_g - guv_o) <= 1e-3 * np.linalg.norm(guv_o)


def test_adjoint_three_channels():
    # one receive antenna (3 phase centres): the general channel loop of the
    # adjoint (six-channel scenes run a fully unrolled instantiation)
    d = _scene(n_pulses=40, nx=64, ny=48)
    tx, rx = hs.geometry(d["n_pulses"], ("A",), (-hs.PHASE_CENTRE_SPACING_M, 0.0, hs.PHASE_CENTRE_SPACING_M))
    d["tx"], d["rx"] = tx, rx
    pulses = list(range(40))
    r = oracle.echo(d, pulses) - oracle.echo(_perturbed(d), pulses)
    gs_o, guv_o = oracle.adjoint(d, pulses, r)
    gs_g, guv_g = _gpu_adjoint(d, 0, 40, r)
    assert np.abs(gs_g - gs_o).max() <= TOL_GRAD * np.abs(gs_o).max()
    assert np.abs(guv_g - guv_o).max() <= TOL_GRAD * np.abs(guv_o).max()


def test_adjoint_complex128_residual():
    import torch
    d = _scene(n_pulses=24, nx=64, ny=48)
    pulses = list(range(24))
    r = oracle.echo(d, pulses) - oracle.echo(_perturbed(d), pulses)
    gs_o, guv_o = oracle.adjoint(d, pulses, r)
    gs_g, guv_g = _gpu_adjoint(d, 0, 24, r, torch.complex128)
    assert np.abs(gs_g - gs_o).max() <= TOL_GRAD * np.abs(gs_o).max()
    assert np.abs(guv_g - guv_o).max() <= TOL_GRAD * np.abs(guv_o).max()


def test_adjoint_unaligned_window():
    d = _scene(n_pulses=100, nx=45, ny=30)
    pulses = list(range(17, 70))
    r = oracle.echo(d, pulses) - oracle.echo(_perturbed(d), pulses)
    gs_o, guv_o = oracle.adjoint(d, pulses, r)
    gs_g, guv_g = _gpu_adjoint(d, 17, len(pulses), r)
    assert np.abs(gs_g - gs_o).max() <= TOL_GRAD * np.abs(gs_o).max()
    assert np.abs(guv_g - guv_o).max() <= TOL_GRAD * np.abs(guv_o).max()


def test_adjoint_matches_fd_on_16_cells():
    d = _scene(n_pulses=24, nx=64, ny=48, cell_m=16.0)
    pulses = list(range(24))
    tgt = oracle.echo(_perturbed(d), pulses)
    r = oracle.echo(d, pulses) - tgt
    _, guv_g = _gpu_adjoint(d, 0, 24, r)
    h = 1e-4
    ncy, ncx = d["cells"]["ncy"], d["cells"]["ncx"]
    cells = [(q // ncx, q % ncx) for q in np.linspace(0, ncx * ncy - 1, 16).astype(int)]
    gmax = np.abs(guv_g).max()
    for (cy, cx) in cells:
        for comp in (0, 1):
            up = d["cells"]["uv"].copy()
            dn = d["cells"]["uv"].copy()
            up[cy, cx, comp] += h
            dn[cy, cx, comp] -= h
            du = dict(d, cells=dict(d["cells"], uv=up))
            dd = dict(d, cells=dict(d["cells"], uv=dn))
            lp, _ = oracle.misfit(du, pulses, tgt)
            lm, _ = oracle.misfit(dd, pulses, tgt)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - guv_g[cy, cx, comp]) <= TOL_GRAD * gmax


def test_adjoint_sigma0_matches_fd_on_8_cells():
    """dL/dsigma0 of the GPU adjoint against central differences of the oracle's
    FP64 misfit (the IQ goes as sqrt(sigma0), so the misfit is not linear in it;
    step 1e-7 on sigma0 ~ 0.02, truncation ~1e-10 relative)."""
    d = _scene(n_pulses=24, nx=64, ny=48, cell_m=16.0)
    pulses = list(range(24))
    tgt = oracle.echo(_perturbed(d), pulses)
    r = oracle.echo(d, pulses) - tgt
    gs_g, _ = _gpu_adjoint(d, 0, 24, r)
    h = 1e-7
    ncy, ncx = d["cells"]["ncy"], d["cells"]["ncx"]
    gmax = np.abs(gs_g).max()
    for q in np.linspace(0, ncx * ncy - 1, 8).astype(int):
        cy, cx = q // ncx, q % ncx
        up = d["cells"]["sigma0"].copy()
        dn = d["cells"]["sigma0"].copy()
        up[cy, cx] += h
        dn[cy, cx] -= h
        lp, _ = oracle.misfit(dict(d, cells=dict(d["cells"], sigma0=up)), pulses, tgt)
        lm, _ = oracle.misfit(dict(d, cells=dict(d["cells"], sigma0=dn)), pulses, tgt)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gs_g[cy, cx]) <= TOL_GRAD * gmax, (cy, cx, fd, gs_g[cy, cx])


def test_autograd_complex128_gradient_kept():
    """A complex128 IQ (iq_dtype) and its complex128 incoming gradient go through
    the adjoint without a cast to complex64."""
    import torch
    from paper_2405_09938_b300 import autograd as hag
    d = _scene(n_pulses=16, nx=64, ny=40)
    c = d["cells"]
    scene = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    s0 = torch.tensor(c["sigma0"], dtype=torch.float64, device="cuda", requires_grad=True)
    uv = torch.tensor(c["uv"], dtype=torch.float64, device="cuda", requires_grad=True)
    tgt = torch.tensor(oracle.echo(_perturbed(d), list(range(16))), dtype=torch.complex128, device="cuda")
    iq = hag.echo(s0, uv, scene, 0, 16, c["cell_m"], iq_dtype=torch.complex128)
    assert iq.dtype == torch.complex128
    loss = torch.sum(torch.abs(iq - tgt) ** 2)
    loss.backward()
    r = (iq.detach() - tgt).cpu().numpy()
    gs_o, guv_o = oracle.adjoint(d, list(range(16)), r)
    assert np.abs(s0.grad.cpu().numpy() - gs_o).max() <= TOL_GRAD * np.abs(gs_o).max()
    assert np.abs(uv.grad.cpu().numpy() - guv_o).max() <= TOL_GRAD * np.abs(guv_o).max()
    scene.close()


def test_autograd_function_gradients():
    import torch
    from paper_2405_09938_b300 import autograd as hag
    d = _scene(n_pulses=32, nx=64, ny=40)
    c = d["cells"]
    scene = harm.harm_scene_create(d, harm.HARM_PREC_MIXED)
    s0 = torch.tensor(c["sigma0"], dtype=torch.float64, device="cuda", requires_grad=True)
    uv = torch.tensor(c["uv"], dtype=torch.float64, device="cuda", requires_grad=True)
    tgt = torch.tensor(oracle.echo(_perturbed(d), list(range(32))), dtype=torch.complex64, device="cuda")
    iq = hag.echo(s0, uv, scene, 0, 32, c["cell_m"])
    loss = torch.sum(torch.abs(iq - tgt) ** 2)
    loss.backward()
    r = (iq.detach() - tgt).cpu().numpy().astype(np.complex128)
    gs_o, guv_o = oracle.adjoint(d, list(range(32)), r)
    assert np.abs(s0.grad.cpu().numpy() - gs_o).max() <= TOL_GRAD * np.abs(gs_o).max()
    assert np.abs(uv.grad.cpu().numpy() - guv_o).max() <= TOL_GRAD * np.abs(guv_o).max()
    scene.close()


def test_adjoint_rejects_fp64_scene_and_missing_cells():
    import torch
    d = _scene(n_pulses=8, nx=16, ny=16)
    scene = harm.harm_scene_create(d, harm.HARM_PREC_FP64)
    r = torch.zeros((6, 8, 512), dtype=torch.complex128, device="cuda")
    with pytest.raises(harm.HarmError):
        harm.harm_echo_adjoint(scene, 0, 8, r)  # no cells
    s0 = torch.full((d["cells"]["ncy"], d["cells"]["ncx"]), 0.02, dtype=torch.float64, device="cuda")
    harm.harm_scene_set_cells(scene, d["cells"]["ncx"], d["cells"]["ncy"], 16.0, s0, None)
    with pytest.raises(harm.HarmError) as ei:
        harm.harm_echo_adjoint(scene, 0, 8, r, torch.zeros_like(s0), None)
    assert ei.value.status == harm.HARM_E_UNSUPPORTED
    scene.close()
