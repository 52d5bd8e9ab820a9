"""The learned step-size proposer: its training kernels against the oracle (gradient,
forward pass, AdamW), bit reproducibility, and what the trained network gains: fewer
corrector stages per path than the plain controller on held-out paths, with every
accepted step judged by the oracle (replay) and the same end points."""
import numpy as np
import pytest

from gpu_util import torch_cuda
import oracle
from oracle import mlp as omlp
from paper_1109_0545_gb300 import hc, learn, synth

pytestmark = pytest.mark.gpu


def _batch(seed, B=1000):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, 12)).astype(np.float32)
    X[:, 7:11] = rng.uniform(-4, 0.5, size=(B, 4))
    r = rng.normal(0, 1, B).astype(np.float32)
    a = rng.integers(0, 2, B).astype(np.int32)
    p = learn.init_params(seed) + rng.normal(0, 0.02, hc.HC_MLP_NPARAM).astype(np.float32)
    return X, r, a, p.astype(np.float32)


def test_gradient_matches_oracle():
    torch = torch_cuda()
    X, r, a, p = _batch(1)
    d = lambda v: torch.from_numpy(v).cuda()
    g = torch.zeros(hc.HC_MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hc.hc_mlp_grad(d(p), len(r), d(X), d(r), d(a), learn.KAPPA, g, loss)
    torch.cuda.synchronize()
    go, lo = omlp.grad(p.astype(np.float64), X.astype(np.float64), r.astype(np.float64), a, learn.KAPPA)
    gg = g.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(gg - go) / np.linalg.norm(go)
    print(f"gradient rel err {err:.2e}, loss {loss.item():.8f} vs {lo:.8f}")
    assert err < 1e-4
    assert abs(loss.item() - lo) <= 1e-5 * lo
    # each block of parameters separately, so that no layer hides in the norm
    for name, sl in (("W1", slice(0, 768)), ("b1", slice(768, 832)), ("W2", slice(832, 4928)),
                     ("b2", slice(4928, 4992)), ("W3", slice(4992, 5056)), ("b3", slice(5056, 5057))):
        e = np.linalg.norm(gg[sl] - go[sl]) / max(np.linalg.norm(go[sl]), 1e-30)
        assert e < 1e-3, name


def test_gradient_is_reproducible():
    torch = torch_cuda()
    X, r, a, p = _batch(2, 5000)
    d = lambda v: torch.from_numpy(v).cuda()
    outs = []
    for _ in range(2):
        g = torch.zeros(hc.HC_MLP_NPARAM, dtype=torch.float32, device="cuda")
        hc.hc_mlp_grad(d(p), len(r), d(X), d(r), d(a), learn.KAPPA, g)
        torch.cuda.synchronize()
        outs.append(g.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_forward_and_adamw_match_oracle():
    torch = torch_cuda()
    X, r, a, p = _batch(3, 300)
    d = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    out = torch.zeros(300, dtype=torch.float32, device="cuda")
    hc.hc_mlp_forward(d(p), 300, d(X), out)
    torch.cuda.synchronize()
    mo, _ = omlp.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(out.cpu().numpy() - mo)) <= 1e-4 * max(1.0, np.max(np.abs(mo)))
    rng = np.random.default_rng(4)
    g = rng.normal(size=hc.HC_MLP_NPARAM).astype(np.float32)
    m1 = (rng.normal(size=hc.HC_MLP_NPARAM) * 0.01).astype(np.float32)
    m2 = (rng.uniform(size=hc.HC_MLP_NPARAM) * 0.01).astype(np.float32)
    pd, m1d, m2d = d(p), d(m1), d(m2)
    hc.hc_mlp_adamw(pd, m1d, m2d, d(g), 7, 1e-3, 0.9, 0.999, 1e-8, 1e-4)
    torch.cuda.synchronize()
    po, m1o, m2o = omlp.adamw(p.astype(np.float64), m1.astype(np.float64), m2.astype(np.float64),
                              g.astype(np.float64), 7, 1e-3)
    assert np.max(np.abs(pd.cpu().numpy() - po)) < 1e-6
    assert np.max(np.abs(m1d.cpu().numpy() - m1o)) < 1e-6
    # 1 - 0.999f differs from 0.001 by 1.3e-5 relative: float32 hyperparameters
    assert np.max(np.abs(m2d.cpu().numpy() - m2o) / np.abs(m2o)) < 1e-4


def test_trained_proposer_gains_over_the_plain_controller():
    """Train on the plain tracker's logs of 160 paths, evaluate on 64 held-out paths of
    the same family (regular variant of the uneven-path shape, n 10..20): the proposer
    takes fewer corrector stages per path, converges as often, reaches the same end
    points, and the oracle accepts every step it took."""
    torch = torch_cuda()
    train_fam = learn.regular_family(500, 160, 10, 20)
    test_fam = learn.regular_family(501, 64, 10, 20)
    plain = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE)
    X, r, a = learn.collect(torch, [f[0] for f in train_fam], [f[1] for f in train_fam], plain)
    params, losses = learn.train(torch, X, r, a, steps=600, batch=4096)
    systems, gammas = [f[0] for f in test_fam], [f[1] for f in test_fam]
    ev = learn.evaluate(torch, systems, gammas, params)
    pl, pr = ev["plain"], ev["proposer"]
    print(f"records {len(r)} accept rate {a.mean():.3f}; loss {losses[0]:.4f} -> {losses[-1]:.4f}")
    print(f"plain: {pl['mean_stages']:.1f} stages/path ({pl['mean_rejected']:.1f} rejected), "
          f"{pl['ok_paths']} ok; proposer: {pr['mean_stages']:.1f} stages/path "
          f"({pr['mean_rejected']:.1f} rejected), {pr['ok_paths']} ok")
    assert losses[-1] < losses[0]
    assert pr["ok_paths"] >= pl["ok_paths"]
    assert pr["mean_stages"] < pl["mean_stages"]
    same = 0
    for p in range(len(systems)):
        a_end, b_end = pl["ends"][p], pr["ends"][p]
        d = np.abs((a_end - b_end).sum(-1)).max() / max(1.0, np.abs(a_end.sum(-1)).max())
        same += d <= 1e-28
    print(f"same end point as the plain controller (1e-28): {same} of {len(systems)}")
    assert same >= 0.9 * len(systems)
    # the oracle replays the proposer's accepted steps of 4 paths: every step converges
    o = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE)
    o.proposer = params.data_ptr()
    st, ends, recs, _ = learn.run_tracker(torch, systems[:4], gammas[:4], o, log_cap=4096)
    oo = oracle.TrackOpts(lambda0=o.lambda0, lambda_min=o.lambda_min, lambda_max=o.lambda_max,
                          grow=o.grow, shrink=o.shrink, eps=o.eps, eps_x=o.eps_x, eps_end=o.eps_end,
                          eps_end_x=o.eps_end_x, div_bound=o.div_bound, max_it=o.max_it,
                          end_it=o.end_it, grow_after=o.grow_after, max_steps=o.max_steps,
                          predictor=o.predictor, lu_mode=o.lu_mode, max_refine=o.max_refine)
    for p in range(4):
        if st[p]["status"] != hc.HC_OK:
            continue
        lg = recs[p][:st[p]["n_corr"]]
        acc = np.nonzero(lg["accepted"] == 1)[0]
        tseq = [lg["t"][k + 1] if k + 1 < len(lg) else 1.0 for k in acc]
        s, g = systems[p], gammas[p]
        x1, status, fail = oracle.track_replay(s.as_dict(), s.coef_limbs(2), synth.limbs(np.ones(s.n), 2),
                                               np.array([g.real, g.imag]), oo, tseq)
        assert fail == -1 and status == 0
        d = np.abs((x1 - ends[p]).sum(-1)).max() / max(1.0, np.abs(x1.sum(-1)).max())
        assert d <= 1e-28
