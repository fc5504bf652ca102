"""Learned initial estimate end to end on the GPU (reduced sizes): data
simulated by the predictor, features, training with the library's kernels,
and the comparison with plain LM from zero."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi, learned_init as LI


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_learned_init_is_consistent_with_features_and_network():
    sim = LI.Simulator(n_geom=1, seed=3)
    X, T = LI.make_dataset(sim, 4, time_stride=4)
    net = _abi.Mlp(512)
    net.psc_mlp_set_params(LI.init_params(X, 3))
    k, vis, lm = sim.draw()
    ctx = sim.sessions[k].ctxs[0]
    got = ctx.psc_learned_init(net, vis, None, sim.w_scale, LI.SIGMA_PRIOR, 4)
    feat = sim.features(k, vis, 4)
    ref = net.psc_mlp_forward(feat).double().cpu().numpy() * LI.SIGMA_PRIOR
    assert np.allclose(got, ref, rtol=1e-6, atol=1e-12)
    net.close()
    sim.close()


def test_trained_network_beats_the_zero_start():
    rep, params = LI.run(n_train=150, n_eval=6, steps=300, batch=512, n_geom=2, seed=1, log=None, n_eval_batched=4)
    assert rep["final_train_loss"] < 1.0                       # targets have unit variance
    assert rep["learned_init_rms_arcsec"] < 0.8 * 30.0
    assert rep["plain_reached"] == rep["n_eval"]
    assert np.all(np.isfinite(params))
    b = rep["batched"]
    assert b["plain_iters_all"] is not None and b["learned_iters_all"] is not None
    assert b["learned_init_rms_arcsec"] < 0.8 * 30.0
    assert b["t_batch_iter_ms"] > 0 and b["t_learned_init_ms"] > 0
