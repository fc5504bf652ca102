"""Batched solves (one persistent fused launch per LM iteration over several
solution intervals, graph-replayed) against per-interval solves and the
oracle.  Intervals differ in array size, length, channel set and aperture."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi, inputs as I
from oracle import lm as LM, psc

import cases
from gpu_cases import GpuProblem


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


SPECS = [  # (aperture/grid, n_ant, n_time, freqs, seed)
    (cases.DISK_SMALL, 5, 10, (1.4e9,), 1),
    (cases.GAUSS_SMALL, 6, 37, (1.3e9, 1.35e9, 1.45e9), 2),
    (cases.DISK_SMALL, 7, 20, (1.2e9, 1.3e9, 1.4e9, 1.5e9, 1.6e9), 3),
]


def _intervals():
    out = []
    for spec, n_ant, nt, freqs, seed in SPECS:
        m, _, lmt, img = cases.problem(spec, n_ant=n_ant, n_time=nt, freqs=freqs, n_src=8, seed=seed)
        V, _ = psc.predict(m, lmt, False)
        vobs = (V + I.complex_noise(V.shape, 1e-3, seed + 10)).astype(np.complex64)
        w = np.full(V.shape, 1e6, dtype=np.float32)
        gp = GpuProblem(m, img)
        out.append(dict(m=m, lmt=lmt, vobs=vobs, w=w, gp=gp, dv=gp.upload(vobs), dw=gp.upload(w, torch.float32)))
    return out


def test_batch_solve_equals_single_solves_and_oracle():
    ivs = _intervals()
    single = [iv["gp"].ctx.psc_solve_offsets(iv["dv"], iv["dw"], 1.0) for iv in ivs]
    sols, reps = _abi.psc_solve_batch([iv["gp"].ctx for iv in ivs], [iv["dv"] for iv in ivs],
                                      [iv["dw"] for iv in ivs])
    for k, iv in enumerate(ivs):
        assert np.array_equal(sols[k], single[k][0]), k
        assert reps[k].n_iter == single[k][1].n_iter and reps[k].reason == single[k][1].reason
    # one interval against the oracle's full LM
    iv = ivs[2]
    m = iv["m"]

    def ev(p):
        c, g, H, X = psc.chi2_grad_normal(m, p, iv["vobs"], iv["w"])
        G, A = psc.assemble_full(m.n_ant, g, H, X)
        return c, G, A
    so, _ = LM.solve_full(ev, np.zeros((m.n_ant, 2)))
    assert np.max(np.abs(sols[2] - so)) < 0.1 * I.ARCSEC


def test_batch_graph_replay_with_restart_matches_solve():
    ivs = _intervals()
    sols, reps = _abi.psc_solve_batch([iv["gp"].ctx for iv in ivs], [iv["dv"] for iv in ivs],
                                      [iv["dw"] for iv in ivs])
    b = _abi.Batch([iv["gp"].ctx for iv in ivs], [iv["dv"] for iv in ivs], [iv["dw"] for iv in ivs])
    zeros = [np.zeros((iv["m"].n_ant, 2)) for iv in ivs]
    b.psc_batch_begin(zeros)
    b.psc_batch_iterate(3)
    b.psc_batch_restart()
    b.psc_batch_iterate(60)
    got, greps = b.psc_batch_end()
    for k in range(len(ivs)):
        assert np.array_equal(got[k], sols[k])
        assert greps[k].n_iter == reps[k].n_iter
    b.close()


def test_batch_autotune_keeps_results():
    ivs = _intervals()
    b = _abi.Batch([iv["gp"].ctx for iv in ivs], [iv["dv"] for iv in ivs], [iv["dw"] for iv in ivs])
    tiles = b.psc_batch_autotune()
    # c_group 0 marks flat bricks of tt items
    assert all((1 <= tt * cg <= 256 or (cg == 0 and tt in (64, 128, 192, 256))) and kv in (1, 2) and st in (0, 1)
               for tt, cg, kv, st in tiles)
    b.psc_batch_begin([np.zeros((iv["m"].n_ant, 2)) for iv in ivs])
    b.psc_batch_iterate(60)
    got, reps = b.psc_batch_end()
    for k, iv in enumerate(ivs):
        ref, _ = iv["gp"].ctx.psc_solve_offsets(iv["dv"], iv["dw"], 1.0)
        assert np.max(np.abs(got[k] - ref)) < 1e-3 * I.ARCSEC
        assert _abi.STOP_REASONS[reps[k].reason] in ("step", "chi2")
    b.close()


def test_autotune_in_the_middle_of_a_solve_leaves_it_undisturbed():
    """psc_batch_autotune times whole-batch launches at zero offsets; it saves
    and restores every context's trial offsets and solver state around them.
    Small apertures, so that the track kernel is among the candidates."""
    small_ap = ("disk", 512, 5.0, 1024)
    ivs = []
    for n_ant, nt, freqs, seed in ((5, 40, (1.3e9, 1.4e9), 4), (6, 64, (1.3e9, 1.4e9, 1.5e9), 5)):
        m, _, lmt, img = cases.problem(small_ap, n_ant=n_ant, n_time=nt, freqs=freqs, sigma_arcsec=30.0, seed=seed)
        V, _ = psc.predict(m, lmt, False)
        vobs = (V + I.complex_noise(V.shape, 1e-3, seed + 10)).astype(np.complex64)
        gp = GpuProblem(m, img)
        ivs.append(dict(m=m, gp=gp, dv=gp.upload(vobs)))
    ctxs = [iv["gp"].ctx for iv in ivs]
    zeros = [np.zeros((iv["m"].n_ant, 2)) for iv in ivs]
    b = _abi.Batch(ctxs, [iv["dv"] for iv in ivs], None, w_scale=[1e6, 1e6])
    b.psc_batch_autotune()
    b.psc_batch_begin(zeros)
    b.psc_batch_iterate(2)
    lm_a, rep_a = b.psc_batch_end()
    b.psc_batch_autotune()                             # mid-solve (its choice may differ: timing)
    lm_b, rep_b = b.psc_batch_end()
    for x, y in zip(lm_a, lm_b):
        assert np.array_equal(x, y)
    for x, y in zip(rep_a, rep_b):
        assert (x.n_iter, x.n_eval, x.reason, x.chi2, x.lam) == (y.n_iter, y.n_eval, y.reason, y.chi2, y.lam)
    b.psc_batch_iterate(40)
    got, reps = b.psc_batch_end()
    b.close()
    # the same minimum as a solve without the interruption: each may stop up to
    # ten step tolerances (1e-3 arcsec) from it, along a different path (the
    # kernel chosen mid-solve may differ from the first choice)
    for k, iv in enumerate(ivs):
        assert _abi.STOP_REASONS[reps[k].reason] in ("step", "chi2"), k
        ref, _ = iv["gp"].ctx.psc_solve_offsets(iv["dv"], None, 1e6)
        assert np.max(np.abs(got[k] - ref)) < 5e-3 * I.ARCSEC, k


def test_batch_rejects_duplicates():
    ivs = _intervals()[:1]
    c = ivs[0]["gp"].ctx
    with pytest.raises(_abi.PscError):
        _abi.Batch([c, c], [ivs[0]["dv"], ivs[0]["dv"]])
