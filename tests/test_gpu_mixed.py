"""Batched solves over mixed intervals (three array types, uneven lengths,
offsets of 10-60 arcsec with 2 arcmin outliers), at a reduced count and length.

* The GPU prediction of one interval per array type is compared with the
  FP64 oracle on sampled visibilities (oracle grid from the sky components,
  which the oracle pins equal to the image transform).
* One batched solve over all intervals (one persistent launch per LM
  iteration, autotuned shapes refitted per interval length) must equal the
  intervals' individual solves, and recover the true offsets, outliers
  included."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi, inputs as I
from paper_1709_08681_gb300.session import MixedSession
from oracle import model_grid, psc

import cases


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def mixed():
    A = I.mixed_arrays(0)
    ivs = I.mixed_intervals(A, 10, seed=2, t_range=(30, 70))
    assert {iv.array for iv in ivs} == set(A)
    s = MixedSession(A, ivs)
    vis = s.simulate()
    yield A, ivs, s, vis
    s.close()


def test_mixed_predict_matches_oracle_on_samples(mixed):
    A, ivs, s, vis = mixed
    rng = np.random.default_rng(5)
    seen = set()
    for k, iv in enumerate(ivs):
        if iv.array in seen:
            continue
        seen.add(iv.array)
        arr = A[iv.array]
        du = 1.0 / (arr.n_grid * arr.cell_rad)
        grid = model_grid.grid_from_components(arr.sky, arr.n_grid, du)
        m = psc.Model(uvw_m=I.mixed_uvw(arr, iv), freq_hz=arr.freq_hz, n_ant=arr.n_ant, grid=grid,
                      cell_rad=arr.cell_rad, support=arr.support, oversample=arr.oversample, ap_kind=arr.ap_kind,
                      diam_m=arr.diam_m, alpha_per_dlambda=arr.alpha_per_dlambda, decorrelation=arr.decorrelation)
        del grid
        n = 200
        ti = rng.integers(0, iv.n_time, n)
        bi = rng.integers(0, arr.n_bl, n)
        ci = rng.integers(0, len(arr.freq_hz), n)
        Vo, dVo = psc.predict_points(m, iv.lm_true, ti, bi, ci)
        vg = torch.empty(s.shape(k), dtype=torch.complex64, device="cuda")
        dg = torch.empty((4,) + s.shape(k), dtype=torch.complex64, device="cuda")
        s.ctxs[k].psc_predict(iv.lm_true, vg, dg)
        V, dV = vg.cpu().numpy()[ti, bi, ci], dg.cpu().numpy()[:, ti, bi, ci]
        assert cases.rel_l2(V, Vo) < 1e-5, iv.array
        for p in range(4):
            assert cases.rel_l2(dV[p], dVo[p]) < 1e-5, (iv.array, p)
    assert seen == set(A)


def test_mixed_batch_equals_individual_solves_and_recovers_offsets(mixed):
    A, ivs, s, vis = mixed
    w_scale = [1.0 / A[iv.array].sigma_noise ** 2 for iv in ivs]
    b = _abi.Batch(s.ctxs, vis, None, w_scale=w_scale)
    tiling = b.psc_batch_autotune()
    # refitted shapes may be narrower than the batch's block (the widest one);
    # c_group 0 marks flat bricks of tt items, (-1, 0) the track kernel, which
    # then serves every context
    track = [tt == -1 and cg == 0 for tt, cg, kv, st in tiling]
    assert all(track) or not any(track)
    assert all((1 <= tt * cg <= 256 or (cg == 0 and tt in (-1, 64, 128, 192, 256))) and kv in (1, 2) and st in (0, 1)
               for tt, cg, kv, st in tiling)
    b.close()
    sols, reps = _abi.psc_solve_batch(s.ctxs, vis, None, w_scale=w_scale)
    for k, iv in enumerate(ivs):
        ref, rep = s.ctxs[k].psc_solve_offsets(vis[k], None, w_scale[k])
        assert np.max(np.abs(sols[k] - ref)) < 1e-3 * I.ARCSEC, k
        assert _abi.STOP_REASONS[reps[k].reason] in ("step", "chi2"), (k, reps[k].reason)
        d = np.abs(sols[k] - iv.lm_true) / I.ARCSEC
        assert np.sqrt(np.mean(d ** 2)) < 1.0, (k, iv.array)
        if len(iv.outliers):
            assert np.max(d[iv.outliers]) < 1.0, (k, iv.array)
