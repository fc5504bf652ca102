"""Host logic of the W-snapshot calls (no GPU): psc_snapshot_components moves
components to the snapshot frame and rescales their fluxes by the beam ratio,
on the host; it must equal the oracle's ``wsnap.snapshot_sources``."""
import numpy as np
import pytest

from paper_1709_08681_gb300 import _abi, inputs as I
from oracle import wsnap


@pytest.mark.parametrize("kind", ["disk", "gauss"])
def test_snapshot_components_match_oracle(kind):
    rng = np.random.default_rng(4)
    n = 37
    src = np.stack([rng.uniform(-0.006, 0.006, n), rng.uniform(-0.006, 0.006, n), rng.uniform(0.1, 2.0, n)], axis=1)
    alpha = I.ALPHA_PER_DLAMBDA_DISK
    for a, b in ((0.0, -1.7320508), (0.31, -0.07), (-2.0, 0.5)):
        got = _abi.psc_snapshot_components(src, a, b, kind, 25.0, alpha, 1.4e9)
        ref = wsnap.snapshot_sources(src, a, b, kind, 1.4e9, 25.0, alpha)
        assert np.allclose(got[:, :2], ref[:, :2], rtol=0, atol=1e-15)
        assert np.allclose(got[:, 2], ref[:, 2], rtol=1e-11, atol=0)


def test_snapshot_components_arguments():
    src = np.array([[0.001, 0.0, 1.0]])
    with pytest.raises(_abi.PscError):
        _abi.psc_snapshot_components(np.array([[0.8, 0.7, 1.0]]), 0.1, 0.1, "disk", 25.0, 1.0, 1.4e9)  # |lm| >= 1
    with pytest.raises(_abi.PscError):
        _abi.psc_snapshot_components(src, 0.1, 0.1, "disk", -1.0, 1.0, 1.4e9)
    with pytest.raises(_abi.PscError):
        _abi.psc_snapshot_components(src, float("nan"), 0.1, "gauss", 25.0, 1.0, 1.4e9)


@pytest.mark.parametrize("kind", ["disk", "gauss"])
def test_wstack_components_match_oracle(kind):
    """psc_wstack_components = the snapshot components plus n - 1 of each true
    direction (``wstack.stack_sources``; the oracle forms n - 1 by a plain
    subtraction, so it agrees to its cancellation error, about 1e-16 absolute)."""
    from oracle import wstack
    rng = np.random.default_rng(5)
    n = 29
    src = np.stack([rng.uniform(-0.01, 0.01, n), rng.uniform(-0.01, 0.01, n), rng.uniform(0.1, 2.0, n)], axis=1)
    alpha = I.ALPHA_PER_DLAMBDA_DISK
    for a, b in ((0.0, -1.7320508), (0.31, -0.07)):
        got = _abi.psc_wstack_components(src, a, b, kind, 25.0, alpha, 1.4e9)
        ref = wstack.stack_sources(src, a, b, kind, 1.4e9, 25.0, alpha)
        assert got.shape == (n, 4)
        assert np.array_equal(got[:, :3], _abi.psc_snapshot_components(src, a, b, kind, 25.0, alpha, 1.4e9))
        assert np.allclose(got[:, 3], ref[:, 3], rtol=0, atol=1e-15)
        assert np.all(got[:, 3] < 0)
    with pytest.raises(_abi.PscError):
        _abi.psc_wstack_components(np.array([[0.8, 0.7, 1.0]]), 0.1, 0.1, kind, 25.0, alpha, 1.4e9)
    import ctypes
    buf = np.zeros((4, 4))                                   # output overlapping the input
    ap = _abi.psc_aperture(_abi.PSC_AP_DISK if kind == "disk" else _abi.PSC_AP_GAUSS, 25.0, alpha, 1)
    assert _abi.lib().psc_wstack_components(3, buf.ctypes.data_as(_abi._D), 0.0, 0.0, ctypes.byref(ap), 1.4e9,
                                            buf.ctypes.data_as(_abi._D)) == _abi.PSC_ERR_ARG
