"""Learned smoother parameters: the MLP's CUDA forward / backward / Adam kernels against
the numpy oracle (fp32 kernels vs fp64 oracle: relative 1e-5 forward, 1e-4 gradient),
and training by the kernels on a seeded regression."""
import numpy as np
import pytest

from oracle import mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _batch(B, seed):
    g = np.random.default_rng(seed)
    x = g.standard_normal((B, 6)).astype(np.float32)
    t = g.standard_normal((B, 2)).astype(np.float32)
    w = g.uniform(0.2, 2.0, B).astype(np.float32)
    return x, t, w


def test_mlp_forward_backward_adam_match_oracle():
    from paper_1603_02524_gb300.learned import SmootherMLP, init_theta
    theta = init_theta(3) + 0.05 * np.random.default_rng(1).standard_normal(4738).astype(np.float32)
    net = SmootherMLP(theta)
    for B in (1, 7, 300):
        x, t, w = _batch(B, B)
        y = net.forward(x)
        yr, _, _ = omlp.forward(theta.astype(np.float64), x.astype(np.float64))
        assert np.abs(y - yr).max() <= 1e-5 * max(1.0, np.abs(yr).max())
        loss, grad = net.loss_and_grad(x, t, w)
        gr = omlp.grad(theta.astype(np.float64), x.astype(np.float64), t.astype(np.float64), w)
        lr = omlp.loss(theta.astype(np.float64), x.astype(np.float64), t.astype(np.float64), w)
        assert abs(float(loss.item()) - lr) <= 1e-5 * abs(lr)
        assert np.abs(grad.cpu().numpy() - gr).max() <= 1e-4 * np.abs(gr).max()
    # one Adam step
    m = np.zeros(4738)
    v = np.zeros(4738)
    g = grad.cpu().numpy().astype(np.float64)
    ref, _, _ = omlp.adam(theta.astype(np.float64), g, m, v, 1, lr=1e-3)
    net.adam_step(grad, lr=1e-3)
    assert np.abs(net.theta.cpu().numpy() - ref).max() <= 1e-6


def test_mlp_training_reduces_loss():
    from paper_1603_02524_gb300.learned import SmootherMLP
    g = np.random.default_rng(5)
    x = g.uniform(-1, 1, (128, 6)).astype(np.float32)
    t = np.stack([np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2], np.cos(x[:, 3]) - x[:, 5]], 1).astype(np.float32)
    net = SmootherMLP()
    hist = net.train(x, t, steps=600, lr=3e-3)
    assert hist[-1] < 0.05 * hist[0]


def test_learned_parameters_beat_paper_parameters_on_heldout_grids(capsys):
    """Train the MLP on rates measured by the library's own MGCG runs (FA smoother with the
    variable V-cycle, 4^3 elements, P = 2, 4, 8, training aspect ratios and gradings), then
    on held-out aspect ratios and gradings:

    * the network's per-level (omega, tau) converge measurably faster on average than the
      paper's omega = tau = 1 (mean rate reduction above 1.15x);
    * the parameters the library hands out, judged by the measured rate with the paper's
      values as fallback (learned.judged_params), are never clearly worse on any grid.  The
      network alone can be: its training rates move in the last bits from run to run (the
      additive patch corrections are summed by atomics), and on one or two held-out grids its
      omega then lands just past the over-relaxation cliff."""
    import math

    from paper_1603_02524_gb300 import learned
    net, hist, records = learned.train_default()
    assert hist[-1] < 0.5 * hist[0]
    gains, rows = [], []
    held = learned.default_configs((2, 4, 8), learned.HELDOUT_ASPECTS, learned.HELDOUT_GRADINGS)
    for cfg in held:
        shape = cfg.aspect if cfg.grading == (1, 1, 1) else ("graded",) + tuple(cfg.grading)
        om, ta, kept, mlp, paper = learned.judged_params(net, cfg.P, cfg.n_elem, cfg.spacing())
        assert (om is not None) == kept
        gains.append(math.log(paper / mlp))
        rows.append((cfg.P, shape, paper, mlp, kept))
        # fresh runs with the handed-out parameters against fresh runs with the paper's
        handed = learned.measure_rate(cfg, om, ta)
        assert handed <= 1.10 * learned.measure_rate(cfg), rows[-1] + (handed,)
        if kept:                       # the kept parameters are the network's
            om2, ta2 = net.level_params(cfg.P, cfg.spacing())
            assert om == om2 and ta == ta2
    mean_gain = sum(gains) / len(gains)
    with capsys.disabled():
        for P, a, paper, mlp, kept in rows:
            print(f"  P={P} aspect={a}: rate paper {paper:.4f} learned {mlp:.4f} "
                  f"({'kept' if kept else 'paper parameters kept'})")
        print(f"  mean rate reduction of the network on held-out grids: x{math.exp(mean_gain):.2f}")
    assert mean_gain > math.log(1.15)      # the learned parameters converge measurably faster
