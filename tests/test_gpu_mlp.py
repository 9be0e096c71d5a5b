"""Learned early stop on the GPU: the training kernels against the oracle's
fp64 forward/backward/Adam, and what the trained stop gains over the plain
fixed-ef search at equal recall."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _data(n, seed):
    rng = np.random.default_rng(seed)
    P = (rng.standard_normal(5313) * 0.3).astype(np.float32)
    x = rng.standard_normal((n, 16)).astype(np.float32)
    y = (rng.uniform(size=n) > 0.4).astype(np.float32)
    w = rng.uniform(0.2, 3.0, size=n).astype(np.float32)
    return P, x, y, w


@pytest.mark.parametrize("n", [1, 127, 1000])
def test_mlp_gradient_matches_oracle(lib_built, oracle_mod, n):
    from paper_2411_12229_gb300 import learned_stop as L
    P, x, y, w = _data(n, n)
    loss, g = L.grad(torch.from_numpy(P).cuda(), torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                     torch.from_numpy(w).cuda())
    lref, gref = oracle_mod.mlp_loss_grad_f64(P.astype(np.float64), x, y, w)
    assert float(loss) == pytest.approx(lref, rel=1e-4)
    g = g.cpu().numpy().astype(np.float64)
    scale = np.abs(gref).max()
    assert np.abs(g - gref).max() <= 1e-4 * scale + 1e-7


def test_mlp_adam_matches_oracle(lib_built, oracle_mod):
    from paper_2411_12229_gb300 import learned_stop as L
    rng = np.random.default_rng(1)
    p = rng.standard_normal(5313)
    m = rng.standard_normal(5313) * 0.01
    v = np.abs(rng.standard_normal(5313)) * 0.01
    g = rng.standard_normal(5313)
    pd, md, vd, gd = (torch.from_numpy(a.astype(np.float32)).cuda() for a in (p, m, v, g))
    for t in (1, 7):
        L.adam(pd, gd, md, vd, t, 1e-3)
        oracle_mod.adam_step_f64(p, m, v, g, t, 1e-3)
        np.testing.assert_allclose(pd.cpu().numpy(), p, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(md.cpu().numpy(), m, rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(vd.cpu().numpy(), v, rtol=1e-5, atol=1e-7)


def test_mlp_forward_matches_oracle(lib_built, oracle_mod):
    from paper_2411_12229_gb300 import learned_stop as L
    P, x, _, _ = _data(300, 3)
    z = L.forward(torch.from_numpy(P).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    ref = np.array([oracle_mod.mlp_logit_f32(P, x[i]) for i in range(300)])
    np.testing.assert_allclose(z, ref, rtol=1e-5, atol=1e-5)


def test_training_lowers_the_loss(lib_built, oracle_mod):
    """A few hundred Adam steps with the library's kernels fit a separable
    toy labelling (loss well below log 2)."""
    from paper_2411_12229_gb300 import learned_stop as L
    rng = np.random.default_rng(4)
    x = rng.standard_normal((20000, 16)).astype(np.float32)
    y = ((x[:, 0] + 0.5 * x[:, 3] - x[:, 7]) > 0.2).astype(np.float32)
    P = L.train(x, y, steps=600, batch=4096, lr=3e-3)
    lref, _ = oracle_mod.mlp_loss_grad_f64(P.cpu().numpy().astype(np.float64), x, y, np.ones(20000, np.float32))
    assert lref < 0.2


@pytest.fixture(scope="module")
def stop_setup(tmp_path_factory, lib_built):
    """A 30,000-vertex index built on the GPU (Algorithm 2) with test and
    training queries and their exact ground truth."""
    from paper_2411_12229_gb300 import eval as E
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300 import synth
    from paper_2411_12229_gb300.api import Index
    w = synth.small(synth.BATCHED_1M_D128, 30_000, 1000)
    x = synth.base(w)
    p = tmp_path_factory.mktemp("stop") / "s.sqg"
    ib.build_index(p, x, 32, device=0, init="random", iterations=3, ef_build=64)
    q, tq = synth.queries(w), synth.train_queries(w, 6000)
    g, _ = E.ground_truth(x, q, 10, device=0)
    tg, _ = E.ground_truth(x, tq, 10, device=0)
    return Index(p, 0), q, g, tq, tg


def test_learned_stop_gain_over_fixed_ef(stop_setup):
    """What the trained stop gains over the plain fixed-ef search, held to
    bars that sampling noise does not pass.  The plain search reaches
    recall@10 0.95 at ef_t; the stop runs with twice that beam as its cap.
    Its threshold is chosen on held-out training queries (the most
    aggressive one whose recall still reaches 0.95), then the 1,000 test
    queries run once:
      * the stop ends searches early: it expands at least 5 % fewer vertices
        than the plain search at the same cap, and its recall is at least
        0.95 minus 2 standard errors of recall@10 over these queries;
      * the perfect stop at the cap (each query stopped at the first
        expansion holding its true top-10, from traces) saves at least as
        much and is printed beside it, with the plain frontier's expansions
        at the stop's recall.
    Whether that saving buys QPS at equal recall is measured by the
    benchmark (the network's evaluations cost time), not asserted here."""
    from paper_2411_12229_gb300 import learned_stop as L
    ix, q, g, tq, tg = stop_setup
    qd = torch.from_numpy(q).cuda()
    efs = (16, 24, 32, 40, 48, 56, 64, 80, 96, 128)
    plain = np.array([L.evaluate(ix, qd, g, 10, ef, reps=1) for ef in efs])  # recall, qps, hops
    ef_t = next((ef for ef, r in zip(efs, plain) if r[0] >= 0.95), 128)
    cap = 2 * ef_t
    model = L.fit(ix, tq, tg, 10, cap, 0.95, every=4, steps=2000, label="final")
    ids, _, st = ix.search(qd, 10, cap, stats=True, stop_mlp=model.params, stop_logit=model.logit, stop_every=4)
    per_q = L.hits_of(ids.cpu().numpy(), g, 10) / 10.0
    r_stop, hops_stop = float(per_q.mean()), float(st[:, 0].float().mean())
    se = float(per_q.std(ddof=1) / np.sqrt(len(per_q)))
    r_cap, _, hops_cap = L.evaluate(ix, qd, g, 10, cap, reps=1)
    bound = L.perfect_stop(ix, q, g, 10, cap)
    plain_hops_at_r = float(np.interp(r_stop, plain[:, 0], plain[:, 2]))
    print(f"cap {cap}: plain recall {r_cap:.4f} hops {hops_cap:.2f}; stop (logit {model.logit}) recall "
          f"{r_stop:.4f} (se {se:.4f}) hops {hops_stop:.2f}; perfect stop hops {bound['perfect_stop_hops']}; "
          f"plain frontier at the stop's recall: {plain_hops_at_r:.2f} hops")
    assert hops_stop <= 0.95 * hops_cap
    assert r_stop >= 0.95 - 2 * se
    assert bound["perfect_stop_hops"] <= hops_cap


def test_training_resumes_from_a_checkpoint(lib_built, tmp_path):
    """300 Adam steps in one run, and 120 steps, a state file, then the other
    180 resumed from it: the same minibatches and the same Adam moments, so
    the same parameters up to the float atomics' summation order."""
    from paper_2411_12229_gb300 import learned_stop as L
    rng = np.random.default_rng(9)
    x = rng.standard_normal((5000, 16)).astype(np.float32)
    y = ((x[:, 1] - x[:, 5]) > 0.0).astype(np.float32)
    full = L.train(x, y, steps=300, batch=1024, seed=3)
    ck = tmp_path / "state.npz"
    L.train(x, y, steps=300, batch=1024, seed=3, stop_after=120, checkpoint=str(ck))
    st = L.load_train_state(ck)
    assert st["step"] == 120 and np.any(st["m"] != 0)
    resumed = L.train(x, y, steps=300, batch=1024, seed=3, resume=str(ck))
    np.testing.assert_allclose(resumed.cpu().numpy(), full.cpu().numpy(), rtol=0, atol=2e-4)
    with pytest.raises(ValueError):
        L.train(x, y, steps=300, batch=1024, seed=4, resume=str(ck))
