"""Learned initial estimate end to end on the GPU (reduced sizes of the
64-antenna workload): features in one batched launch, training with the
library's kernels on GPU-simulated intervals, and the measured comparison
with plain LM from zero on held-out intervals."""
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


def test_batched_features_equal_single_calls_and_kept_step_contexts():
    """psc_features_batch over several (context, data) pairs -- one context
    serving two pairs -- gives every pair's psc_features result bit for bit;
    and the features of a full interval at time stride 15 equal those of a
    context holding only its kept steps (what the training data uses)."""
    stream = torch.cuda.current_stream()
    pool = LI.GeometryPool("disk64_l16ch", [-1.0, 1.5], 2, stream, 15)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    rng = np.random.default_rng(9)
    ctxs = [pool.full[0], pool.full[1], pool.full[0]]
    vis = torch.empty((3, pool.n_time, pool.n_bl, pool.n_chan), dtype=torch.complex64, device="cuda")
    lms = [rng.normal(0.0, pool.wl.sigma_pt, (pool.n_ant, 2)) for _ in range(3)]
    pool.simulate(ctxs, lms, vis, gen)
    work = torch.empty(_abi.psc_features_batch_work(ctxs, 15), dtype=torch.uint8, device="cuda")
    out = torch.empty((3 * pool.n_ant, 52), dtype=torch.float32, device="cuda")
    _abi.psc_features_batch(ctxs, [vis[j] for j in range(3)], pool.w_scale, LI.SIGMA_PRIOR, 15, work, out)
    for j in range(3):
        one = ctxs[j].psc_features(vis[j], None, pool.w_scale, LI.SIGMA_PRIOR, 15)
        assert torch.equal(one, out[j * pool.n_ant:(j + 1) * pool.n_ant]), j
    kept = vis[0, ::15].contiguous()
    k1 = pool.kept[0].psc_features(kept, None, pool.w_scale, LI.SIGMA_PRIOR, 1)
    assert torch.equal(k1, out[:pool.n_ant])
    with pytest.raises(_abi.PscError):
        _abi.psc_features_batch(ctxs, [vis[j] for j in range(3)], pool.w_scale, LI.SIGMA_PRIOR, 15, work[:64], out)
    pool.close()


def test_trained_network_reaches_one_arcsec_in_fewer_iterations_and_less_time():
    """The network's estimate, trained on 6,000 simulated intervals over 64
    hour-angle windows, must bring 512 held-out intervals (on 16 windows
    between the training ones) to 1 arcsec RMS in fewer LM iterations than
    plain LM from zero, and in less measured time including its features and
    network."""
    rep = LI.run_at_scale(n_train=6000, n_eval=512, train_batch=1000, eval_batch=256, steps=3000, seed=0)
    p, l = rep["plain"], rep["learned"]
    assert rep["final_train_loss"] < 0.5                        # targets have unit variance
    assert rep["learned_init_rms_arcsec_median"] < 10.0         # against sigma = 30 arcsec per axis
    assert p["reached_fraction"] == 1.0 and l["reached_fraction"] == 1.0
    assert l["mean_iters_to_target"] < p["mean_iters_to_target"]
    assert l["batch_iters_to_target_mean"] < p["batch_iters_to_target_mean"]
    assert l["intervals_per_s"] > p["intervals_per_s"]
