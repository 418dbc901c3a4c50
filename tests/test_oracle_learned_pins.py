"""Pins of the learned-scorer oracle (CPU only): each checks it against
something other than itself -- a library routine, finite differences, a
closed form or an identity between independently computed quantities."""

import itertools

import numpy as np
import pytest

import oracle
from oracle import learned as ol
from workloads import make_problem

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _small(seed=11, n=80, m=14, planted=((2, 7, 11),), beta=((1.5, -0.8, 0.6),), sigma=0.05):
    return make_problem(n_samples=n, n_sis=m, seed=seed, planted=[list(planted[0])],
                        beta=[list(beta[0])], sigma=sigma, distinct=True)


def test_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.normal(size=2000), rng.normal(size=500) * 1e-20,
                        rng.normal(size=500) * 1e20, [0.0, -0.0, 1.0, -2.5]]).astype(np.float32)
    # exact ties: low 16 bits 0x8000, both parities of bit 16
    ties = (rng.integers(0, 2**15, size=200, dtype=np.uint32) << 17 | 0x8000
            | (rng.integers(0, 2, size=200, dtype=np.uint32) << 16)) + np.uint32(0x3F800000 & 0)
    tv = (ties | np.uint32(0x3F000000)).view(np.float32)
    v = np.concatenate([v, tv, -tv])
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ol.bf16(v), ref)


def test_pair_ranks_are_colex():
    P = ol.all_pairs(23)
    assert len(P) == 23 * 22 // 2
    np.testing.assert_array_equal(ol.pair_rank(P[:, 0], P[:, 1]), np.arange(len(P)))
    assert set(map(tuple, P.tolist())) == set(itertools.combinations(range(23), 2))


def test_pair_features_partial_correlation_identity():
    # R2 (two-feature QR fit) = r_i^2 + rho_j.i^2 (1 - r_i^2) / (1 - C_ij^2)
    # (the partial-correlation decomposition): R2 comes from Householder QR,
    # rho from explicit residual projections
    p = _small()
    F = ol.pair_features(p.X, p.y)
    ri, rj, c, rji, rij, f5 = F.T
    r2 = 1.0 - np.exp(8.0 * f5)
    np.testing.assert_allclose(r2, ri**2 + rji**2 * (1 - ri**2) / (1 - c**2), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(r2, rj**2 + rij**2 * (1 - rj**2) / (1 - c**2), rtol=1e-9, atol=1e-12)
    # r from Eq. 1 directly
    x = p.X[3] - p.X[3].mean()
    yy = p.y - p.y.mean()
    r3 = (x @ yy) / np.sqrt((x @ x) * (yy @ yy))
    q = int(ol.pair_rank(3, 5))
    assert F[q, 0] == pytest.approx(r3, rel=1e-12)


def test_residual_correlation_vanishes_for_collinear_column():
    p = _small()
    X = p.X.copy()
    X[5] = 3.0 * X[2] - 1.0
    F = ol.pair_features(X, p.y, pairs=np.array([[2, 5]], dtype=np.int32))
    assert abs(F[0, 3]) < 1e-12 and abs(F[0, 4]) < 1e-12
    assert abs(F[0, 2]) == pytest.approx(1.0, abs=1e-12)


def test_labels_bounded_by_pair_fit_and_by_global_best():
    p = _small()
    F = ol.pair_features(p.X, p.y)
    best = ol.best_completion(p.X, p.y)
    assert np.all(best <= np.exp(8.0 * F[:, 5]) * (1 + 1e-12))   # nesting
    ex = oracle.fit(p.X, p.y, 3, 1)
    syy = float(((p.y - p.y.mean()) ** 2).sum())
    assert np.min(best) == pytest.approx(ex["score"][0, 0] / syy, rel=1e-12)
    # the pairs of the planted triple complete it
    for (a, b) in itertools.combinations((2, 7, 11), 2):
        q = int(ol.pair_rank(a, b))
        assert best[q] == pytest.approx(ex["score"][0, 0] / syy, rel=1e-12)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    B = 24
    feats = rng.normal(size=(B, 6))
    target = rng.normal(size=B)
    flat = rng.normal(size=ol.N_PARAMS) * 0.1
    loss, g = ol.loss_and_grad(flat, feats, target, round_bf16=False)
    idx = np.concatenate([rng.choice(256 * 6, 8, replace=False),
                          256 * 6 + rng.choice(256, 4, replace=False),
                          256 * 7 + rng.choice(256 * 256, 12, replace=False),
                          256 * 263 + rng.choice(256, 4, replace=False),
                          256 * 264 + rng.choice(256, 4, replace=False), [ol.N_PARAMS - 1]])
    h = 1e-6
    for q in idx:
        e = np.zeros_like(flat)
        e[q] = h
        lp, _ = ol.loss_and_grad(flat + e, feats, target, round_bf16=False)
        lm, _ = ol.loss_and_grad(flat - e, feats, target, round_bf16=False)
        fd = (lp - lm) / (2 * h)
        assert g[q] == pytest.approx(fd, rel=1e-5, abs=1e-9), q


def test_rounded_forward_equals_exact_forward_on_bf16_values():
    # when every rounded quantity is already a BF16 value the two forms agree
    rng = np.random.default_rng(4)
    feats = ol.bf16(rng.normal(size=(5, 6)))
    flat = np.zeros(ol.N_PARAMS)
    p = ol.unpack(flat.copy())
    p["W1"][:] = ol.bf16(rng.normal(size=(256, 6)))
    p["W2"][:] = 0.0
    p["b2"][:] = 0.0
    p["w3"][:] = 0.0
    flat = ol.pack(p)
    a, _ = ol.forward(flat, feats, True)
    b, _ = ol.forward(flat, feats, False)
    np.testing.assert_array_equal(a, b)


def _torch_net(torch, flat):
    """A 6-256-256-1 ReLU network of torch.nn modules in FP64 holding the
    same parameters as the flat vector (W1 [256,6] | b1 | W2 [256,256] with
    rows = output units | b2 | w3 | b3)."""
    p = ol.unpack(flat)
    net = torch.nn.Sequential(torch.nn.Linear(6, 256), torch.nn.ReLU(),
                              torch.nn.Linear(256, 256), torch.nn.ReLU(),
                              torch.nn.Linear(256, 1)).double()
    with torch.no_grad():
        net[0].weight.copy_(torch.from_numpy(p["W1"]))
        net[0].bias.copy_(torch.from_numpy(p["b1"]))
        net[2].weight.copy_(torch.from_numpy(p["W2"]))
        net[2].bias.copy_(torch.from_numpy(p["b2"]))
        net[4].weight.copy_(torch.from_numpy(p["w3"][None, :]))
        net[4].bias.copy_(torch.from_numpy(p["b3"]))
    return net


def _dense_params(rng):
    # every tensor non-zero, biases of both signs so some units are off
    p = dict(W1=rng.normal(size=(256, 6)) * 0.6, b1=rng.normal(size=256) * 0.3,
             W2=rng.normal(size=(256, 256)) / 16.0, b2=rng.normal(size=256) * 0.2,
             w3=rng.normal(size=256) / 16.0, b3=np.array([0.37]))
    return ol.pack(p)


def test_unrounded_forward_matches_torch_nn_fp64():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(21)
    flat = _dense_params(rng)
    feats = rng.normal(size=(300, 6))
    out, c = ol.forward(flat, feats, round_bf16=False)
    net = _torch_net(torch, flat)
    with torch.no_grad():
        ref = net(torch.from_numpy(feats))[:, 0].numpy()
        h1 = net[1](net[0](torch.from_numpy(feats))).numpy()
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(c["h1"], h1, rtol=1e-12, atol=1e-14)
    # both ReLUs cut something on this input, so a dropped ReLU would show
    assert 0.1 < np.mean(c["pre1"] > 0) < 0.9
    assert 0.1 < np.mean(c["pre2"] > 0) < 0.9


def test_unrounded_gradient_matches_torch_autograd_fp64():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(22)
    flat = _dense_params(rng)
    feats = rng.normal(size=(64, 6))
    target = rng.normal(size=64)
    loss, g = ol.loss_and_grad(flat, feats, target, round_bf16=False)
    net = _torch_net(torch, flat)
    out = net(torch.from_numpy(feats))[:, 0]
    tl = torch.mean((out - torch.from_numpy(target)) ** 2)
    tl.backward()
    assert loss == pytest.approx(float(tl.detach()), rel=1e-12)
    ref = ol.pack(dict(W1=net[0].weight.grad.numpy(), b1=net[0].bias.grad.numpy(),
                       W2=net[2].weight.grad.numpy(), b2=net[2].bias.grad.numpy(),
                       w3=net[4].weight.grad.numpy()[0], b3=net[4].bias.grad.numpy()))
    np.testing.assert_allclose(g, ref, rtol=1e-10, atol=1e-14)


def test_adam_matches_torch_optim_over_several_steps():
    """Eight Adam steps with changing gradients against torch.optim.Adam in
    FP64: the bias corrections 1 - beta^t past the first step are checked."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(23)
    w0 = rng.normal(size=50)
    grads = [rng.normal(size=50) * (1.0 + 3.0 * t) for t in range(8)]
    w, m1, m2 = w0.copy(), np.zeros(50), np.zeros(50)
    tw = torch.nn.Parameter(torch.from_numpy(w0.copy()))
    opt = torch.optim.Adam([tw], lr=3e-2, betas=(0.8, 0.95), eps=1e-6)
    for t, g in enumerate(grads, start=1):
        w, m1, m2 = ol.adam_step(w, g, m1, m2, t, 3e-2, beta1=0.8, beta2=0.95, eps=1e-6)
        tw.grad = torch.from_numpy(g.copy())
        opt.step()
        np.testing.assert_allclose(w, tw.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_first_adam_step_is_sign_step():
    rng = np.random.default_rng(5)
    w = rng.normal(size=100)
    g = rng.normal(size=100)
    new, m1, m2 = ol.adam_step(w, g, np.zeros(100), np.zeros(100), 1, 1e-3, eps=0.0)
    np.testing.assert_allclose(new, w - 1e-3 * np.sign(g), rtol=0, atol=1e-15)
    same, _, _ = ol.adam_step(w, np.zeros(100), np.zeros(100), np.zeros(100), 1, 1e-3)
    np.testing.assert_array_equal(same, w)


def test_fit_pairs_with_every_pair_is_the_exhaustive_search():
    p = _small(m=12)
    ex = oracle.fit(p.X, p.y, 3, 15)
    got = ol.fit_pairs(p.X, p.y, ol.all_pairs(12), 15)
    np.testing.assert_array_equal(got["tuples"], ex["tuples"][0])
    np.testing.assert_allclose(got["score"], ex["score"][0], rtol=1e-14)


def test_fit_pairs_restricted_to_one_pair():
    p = _small(m=12)
    got = ol.fit_pairs(p.X, p.y, np.array([[2, 7]]), 10)
    assert all({2, 7} <= set(t) for t in got["tuples"].tolist())
    assert tuple(got["tuples"][0]) == (2, 7, 11)
    assert len(ol.reachable_triples(np.array([[2, 7], [2, 11]]), 12)) == 2 * 10 - 1
