"""Learned proposal scorer on the GPU against the oracle: pair features and
labels, the network's loss and gradient (BF16 tensor-core kernels), the
Adam step, the pair-restricted exact search, and the recall of the trained
network against the exhaustive search."""

import numpy as np
import pytest

import oracle
import paper_2502_20072_gb300 as l0
from oracle import learned as ol
from workloads import make_problem

from l0_testutil import RMSE_RTOL, TIE_GAP, score_fn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Tolerances.  Pair features and labels come from the FP32 split-BF16 Gram,
# whose entries are within ~5e-6 of the FP64 correlations.  rho and R2
# divide by 1 - r^2 or 1 - C^2, which amplifies that error by up to
# 1 / min(1 - r_i^2, 1 - r_j^2, 1 - C_ij^2) (a planted column has r ~ 0.9997).
FEAT_ATOL = 1e-3
FEAT_AMP = 1e-5
EPS_G = 5e-6      # split-BF16 Gram entry error against the FP64 correlation
# The network: FP32 sums in a different order than the oracle's exact sums
# can move a BF16-rounded activation by one BF16 ulp (2^-8 relative); summed
# over a batch such flips stay well under 2 % of a gradient's norm.
GRAD_REL = 2e-2


def _prob(seed, n=300, m=40, sigma=0.01, planted=None, beta=None, n_planted=3):
    kw = dict(n_samples=n, n_sis=m, seed=seed, sigma=sigma, distinct=True)
    if planted is None:
        kw["n_planted"] = n_planted
    else:
        kw["planted"] = planted
        kw["beta"] = beta
    return make_problem(**kw)


def _mixed():
    return l0.Handle(precision=l0.MIXED_BF16X3)


def test_pair_features_match_oracle():
    p = _prob(101)
    with _mixed() as h:
        feats, lab = h.pair_data(p.X, p.y)
    got = feats.cpu().numpy()
    ref = ol.pair_features(p.X, p.y)
    assert got.shape == (40 * 39 // 2, 8)
    ri, rj, c = ref[:, 0], ref[:, 1], ref[:, 2]
    res2 = np.exp(8.0 * ref[:, 5])          # 1 - R2 of the pair
    amp = 1.0 / np.minimum(np.minimum(np.minimum(1 - ri**2, 1 - rj**2), 1 - c**2), 8 * res2)
    tol = FEAT_ATOL + FEAT_AMP * amp
    assert np.all(np.abs(got[:, :6] - ref) <= tol[:, None]), np.max(np.abs(got[:, :6] - ref) - tol[:, None])
    assert np.median(np.abs(got[:, :6] - ref)) < 1e-4
    assert np.all(got[:, 6:] == 0)


def test_pair_labels_match_oracle():
    p = _prob(102, m=30)
    with _mixed() as h:
        _, lab = h.pair_data(p.X, p.y)
    got = lab.cpu().numpy().astype(np.float64)
    ref = ol.labels(p.X, p.y)
    rel = np.exp(ref)
    big = rel > 1e-3
    # log of an FP32 Schur complement with ~1e-5 absolute error
    np.testing.assert_allclose(got[big], ref[big], atol=0.02)
    assert np.all(got[~big] < np.log(2e-3))
    # The best completions (relative SSE <= 1e-3, the pairs the scorer must
    # rank first) in linear space.  rel = 1 - c^T C^-1 c over the standardized
    # columns moves by at most eps (1 + |beta|_1)^2 to first order when every
    # Gram entry moves by eps (beta = C^-1 c, the standardized coefficients),
    # and the minimum over k moves by at most the largest such move: with
    # eps = EPS_G, doubled for the second order, plus FP32 rounding of O(1)
    # terms.
    pairs = ol.all_pairs(30)
    Z = (p.X - p.X.mean(axis=1, keepdims=True))
    Z /= np.linalg.norm(Z, axis=1, keepdims=True)
    yz = p.y - p.y.mean()
    yz /= np.linalg.norm(yz)
    for q in np.flatnonzero(~big):
        i, j = pairs[q]
        best_k, best = -1, np.inf
        for kk in range(30):
            if kk in (i, j):
                continue
            A = Z[[i, j, kk]].T
            beta, *_ = np.linalg.lstsq(A, yz, rcond=None)
            r = yz - A @ beta
            if r @ r < best:
                best, best_k, bb = float(r @ r), kk, beta
        tol = 2.0 * EPS_G * (1.0 + np.abs(bb).sum()) ** 2 + 1e-6
        assert abs(np.exp(got[q]) - rel[q]) <= tol, (q, np.exp(got[q]), rel[q], tol)
    # the planted triple's pairs complete it best
    assert np.argmin(got) == np.argmin(ref) or abs(got.min() - ref.min()) < 1.0


def _net_case(seed, B):
    rng = np.random.default_rng(seed)
    feats = rng.uniform(-1, 1, size=(B, 6))
    flat = np.zeros(ol.N_PARAMS)
    p = ol.unpack(flat)
    p["W1"][:] = rng.uniform(-1, 1, size=(256, 6))
    p["b1"][:] = rng.uniform(-0.1, 0.1, size=256)
    p["W2"][:] = rng.uniform(-1, 1, size=(256, 256)) * np.sqrt(6.0 / 256)
    p["b2"][:] = rng.uniform(-0.1, 0.1, size=256)
    p["w3"][:] = rng.uniform(-1, 1, size=256) * np.sqrt(6.0 / 256)
    p["b3"][:] = -3.0
    flat = ol.pack(p).astype(np.float32).astype(np.float64)
    target = rng.normal(-4.0, 2.0, size=B)
    return feats, flat, target


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _feat_rows(feats):
    f = np.zeros((len(feats), 8), dtype=np.float32)
    f[:, :6] = feats
    return f


@pytest.mark.parametrize("B", [1, 128, 300, 1000])
def test_network_loss_and_gradient_match_oracle(B):
    feats, flat, target = _net_case(7 + B, B)
    ref_loss, ref_g = ol.loss_and_grad(flat, feats, target, round_bf16=True)
    with l0.Scorer(seed=1) as s:
        s.set_params(flat)
        loss, g = s.loss_grad(_dev(_feat_rows(feats)), _dev(target))
    assert loss == pytest.approx(ref_loss, rel=1e-3)
    pr, pg = ol.unpack(ref_g), ol.unpack(g.astype(np.float64))
    for name in ("W1", "b1", "W2", "b2", "w3", "b3"):
        err = np.linalg.norm(pg[name] - pr[name]) / max(np.linalg.norm(pr[name]), 1e-30)
        assert err < GRAD_REL, (name, err)
    cos = ref_g @ g / (np.linalg.norm(ref_g) * np.linalg.norm(g))
    assert cos > 0.9995


def test_network_predict_matches_oracle():
    feats, flat, _ = _net_case(21, 777)
    ref, _ = ol.forward(flat, feats, round_bf16=True)
    with l0.Scorer() as s:
        s.set_params(flat)
        out = s.predict(_dev(_feat_rows(feats))).cpu().numpy()
    np.testing.assert_allclose(out, ref, atol=2e-2 * (1 + np.abs(ref).max()), rtol=0)
    assert np.corrcoef(out, ref)[0, 1] > 0.9999


def test_first_adam_step_is_a_sign_step():
    feats, flat, target = _net_case(5, 512)
    with l0.Scorer() as s:
        s.set_params(flat)
        loss0, g = s.loss_grad(_dev(_feat_rows(feats)), _dev(target))
        losses = s.train(_dev(_feat_rows(feats)), _dev(target), batch_rows=512, steps=1, lr=1e-3)
        new = s.get_params().astype(np.float64)
    assert losses[0] == pytest.approx(loss0, rel=1e-6)
    g = g.astype(np.float64)
    step = new - flat.astype(np.float32).astype(np.float64)
    expect = -1e-3 * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(step, expect, atol=2e-6 * (1 + np.abs(flat)).max())


def test_training_reduces_the_loss():
    feats, flat, target = _net_case(9, 4096)
    with l0.Scorer(seed=3) as s:
        losses = s.train(_dev(_feat_rows(feats)), _dev(target), batch_rows=1024, steps=200, lr=3e-3)
    assert losses[-10:].mean() < 0.5 * losses[:4].mean()


def _check_pairs(p, pairs, k, precision):
    ref = ol.fit_pairs(p.X, p.y, pairs, k)
    with l0.Handle(precision=precision) as h:
        got_t, got_r = h.fit_pairs(p.X, p.y, pairs, k)
        st = h.stats()
    fin = np.isfinite(ref["score"])
    n = p.X.shape[1]

    def sf(tuples):
        if len(tuples) == 0:
            return []
        sse, _ = oracle.score(p.X, p.y, np.array(tuples, dtype=np.int32))
        return sse[:, 0]
    ok, msg = oracle.agreement(ref["tuples"][fin], ref["score"][fin], got_t[fin],
                               rel_gap=TIE_GAP, score_fn=sf)
    assert ok, msg
    np.testing.assert_allclose(got_r[fin], ref["rmse"][fin], rtol=RMSE_RTOL, atol=0)
    assert np.all(got_t[~fin] == -1)
    return st


@pytest.mark.parametrize("precision", [l0.FP64, l0.MIXED_BF16X3])
def test_fit_pairs_matches_oracle(precision):
    p = _prob(33, m=36, n=200)
    rng = np.random.default_rng(4)
    pairs = np.array([sorted(rng.choice(36, 2, replace=False)) for _ in range(25)])
    pairs = np.concatenate([pairs, pairs[:5, ::-1], pairs[:3]])    # reversed and repeated
    st = _check_pairs(p, pairs, 40, precision)
    n_tri = len(ol.reachable_triples(pairs, 36))
    assert st["tuple_fits"] == n_tri
    assert st["proposal_pairs"] == len(pairs)


def test_fit_pairs_with_every_pair_is_exhaustive():
    p = _prob(34, m=24, n=150)
    pairs = ol.all_pairs(24)
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        t1, r1 = h.fit_pairs(p.X, p.y, pairs, 30)
        t2, r2 = h.fit(p.X, p.y, 3, 30)
    np.testing.assert_array_equal(t1, t2[0])
    np.testing.assert_array_equal(r1, r2[0])


def test_fit_pairs_rejects_bad_pairs():
    p = _prob(35, m=20, n=100)
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        with pytest.raises(l0.L0Error) as e:
            h.fit_pairs(p.X, p.y, np.array([[3, 3]]), 5)
        assert e.value.code == l0.EINVAL
        with pytest.raises(l0.L0Error) as e:
            h.fit_pairs(p.X, p.y, np.array([[0, 20]]), 5)
        assert e.value.code == l0.EINVAL


def _recall(ref_t, got_t):
    ref = set(map(tuple, ref_t.tolist()))
    got = set(map(tuple, got_t.tolist()))
    return len(ref & got) / len(ref)


def _spearman(a, b):
    ra = np.argsort(np.argsort(a)).astype(np.float64)
    rb = np.argsort(np.argsort(b)).astype(np.float64)
    return float(np.corrcoef(ra, rb)[0, 1])


def test_trained_scorer_recall_and_gain():
    """Train on exhaustive labels of seeded instances (eight planted terms,
    noise sigma = 1, so that the best triples spread over many pairs), then
    compare the learned search with the exhaustive search on a held-out
    instance.  The network's gain over the method without it: it spares
    more than 90 % of the triple fits at recall >= 0.99, where the same
    network untrained finds well under that."""
    from paper_2502_20072_gb300 import learn
    m_tr, m_te, n = 120, 200, 400
    train = [_prob(seed, n=n, m=m_tr, n_planted=8, sigma=1.0) for seed in range(500, 516)]
    F, Y = learn.pair_training_set(train, seed=0)
    test = _prob(777, n=n, m=m_te, n_planted=8, sigma=1.0)
    k, frac = 100, 0.02
    with l0.Scorer(seed=11) as untrained:
        s, losses, secs = learn.train_scorer(F, Y, steps=3000, batch_rows=8192, lr=2e-3, seed=11)
        with s, _mixed() as h:
            assert losses[-50:].mean() < 0.85 * losses[:5].mean()
            tf, tl = h.pair_data(test.X, test.y, standardize=True)
            truth = tl.cpu().numpy()
            rho_tr = _spearman(s.predict(tf).cpu().numpy(), truth)
            rho_un = _spearman(untrained.predict(tf).cpu().numpy(), truth)
            ex_t, _ = h.fit(test.X, test.y, 3, k)
            ex_fits = h.stats()["tuple_fits"]
            le_t, _ = h.fit_learned(test.X, test.y, s, k, fraction=frac)
            st = h.stats()
            un_t, _ = h.fit_learned(test.X, test.y, untrained, k, fraction=frac)
    rt, ru = _recall(ex_t[0], le_t), _recall(ex_t[0], un_t)
    print("trained in %.2f s; rank correlation with the exhaustive labels %.3f (untrained %.3f);"
          " recall@%d trained %.3f untrained %.3f; %d pairs, %d of %d fits"
          % (secs, rho_tr, rho_un, k, rt, ru, st["proposal_pairs"], st["tuple_fits"], ex_fits))
    assert rt >= 0.99
    assert ru < rt - 0.2
    assert rho_tr > rho_un
    assert st["tuple_fits"] < 0.1 * ex_fits
    assert st["proposal_pairs"] >= frac * m_te * (m_te - 1) / 2
