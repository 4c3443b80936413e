"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the oracle."""
import numpy as np

from paper_2405_09938_b300 import harm


def run_echo(desc, precision, n0, np_, dtype="c128", scene=None):
    import torch
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    own = scene is None
    if own:
        scene = harm.harm_scene_create(desc, precision)
    iq = torch.zeros((len(desc["rx"]), np_, desc["n_range"]), dtype=tdt, device="cuda")
    harm.harm_echo_accumulate(scene, n0, np_, iq, zero_first=True)
    harm.harm_scene_sync(scene)
    out = iq.cpu().numpy()
    if own:
        scene.close()
    return out


def run_states(desc, precision, n0, np_):
    import torch
    scene = harm.harm_scene_create(desc, precision)
    tdt = torch.float64 if precision == harm.HARM_PREC_FP64 else torch.float32
    st = torch.zeros((np_, 3, desc["ny"], desc["nx"]), dtype=tdt, device="cuda")
    harm.harm_facets_generate(scene, n0, np_, st)
    harm.harm_scene_sync(scene)
    out = st.cpu().numpy().astype(np.float64)
    scene.close()
    return out


def take_pulses(iq, pulses):
    """Pulse rows [:, pulses, :] of an IQ tensor on the device, as a numpy array.
    The indices are checked on the host first: an out-of-range index into a CUDA
    tensor would trip a device-side assert and lose the context."""
    n = iq.shape[1]
    bad = [p for p in pulses if not 0 <= p < n]
    assert not bad, "pulses %s outside [0, %d)" % (bad, n)
    return iq[:, list(pulses), :].cpu().numpy()


def rel_rms(got, want):
    num = np.sum(np.abs(got - want) ** 2)
    den = np.sum(np.abs(want) ** 2)
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))


def ati_phase_bias(got, want, a, b):
    """wrap(arg sum IQ_a conj IQ_b (GPU) - same (oracle)) in rad."""
    g = np.sum(got[a] * np.conj(got[b]))
    w = np.sum(want[a] * np.conj(want[b]))
    d = np.angle(g) - np.angle(w)
    return float((d + np.pi) % (2 * np.pi) - np.pi)


def peak_err(got, want):
    """Largest per-element error, each normalised by the peak magnitude of its
    (channel, pulse) row of the reference: max_k |got - want| / max_k |want|.
    Unlike the relative RMS, this does not let one facet's misplaced bin or tap
    disappear in the sum over a large scene (rows without signal are skipped)."""
    g = np.asarray(got).reshape(-1, np.asarray(got).shape[-1])
    w = np.asarray(want).reshape(-1, np.asarray(want).shape[-1])
    peak = np.abs(w).max(axis=1)
    rows = peak > 0
    if not rows.any():
        return float(np.abs(g).max())
    return float((np.abs(g - w).max(axis=1)[rows] / peak[rows]).max())


# Per-element bound relative to the RMS bound: the largest error of a row is a few
# times its RMS error, and a row's peak a few times its RMS value.
ELEM_FACTOR = 10.0


def assert_iq(got, want, tol, elem_tol=None):
    """IQ relative RMS below tol and every element within elem_tol (default
    ELEM_FACTOR x tol) of its row's peak; returns (rel_rms, peak_err)."""
    err, pe = rel_rms(got, want), peak_err(got, want)
    lim = ELEM_FACTOR * tol if elem_tol is None else elem_tol
    assert err < tol, "IQ rel RMS %.3e >= %.1e" % (err, tol)
    assert pe < lim, "per-element error %.3e of the row peak >= %.1e (rel RMS %.3e)" % (pe, lim, err)
    return err, pe
