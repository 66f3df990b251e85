"""Oracle pins for the sparse-graph steps (Sec. 2.2, "Training sparse models").

The decimation score is checked against the symmetric Kullback-Leibler
divergence computed by exact enumeration of a small model and of the model
without the element; the activation score against the data log-likelihood
gain of fitting one coupling, maximised numerically over exact enumeration;
the selections and the masked update against their defining invariants.
"""
import itertools

import numpy as np
import pytest

import oracle as orc

scipy_opt = pytest.importorskip("scipy.optimize")


def _symmetric_model(L, q, rng, scale=0.8):
    h = rng.normal(0, 0.7, (L, q))
    J = np.zeros((L, L, q, q))
    for i in range(L):
        for j in range(i + 1, L):
            B = rng.normal(0, scale, (q, q))
            J[i, j] = B
            J[j, i] = B.T
    return h, J


def _states(L, q):
    return np.array(list(itertools.product(range(q), repeat=L)), dtype=np.int64)


def _log_weights(h, J, S):
    """-E(s) for every state by definition (Eq. 1): sum_i h + sum_{i<j} J."""
    L = S.shape[1]
    e = np.zeros(len(S))
    for i in range(L):
        e += h[i, S[:, i]]
        for j in range(i + 1, L):
            e += J[i, j, S[:, i], S[:, j]]
    return e


def _probs(h, J, S):
    lw = _log_weights(h, J, S)
    w = np.exp(lw - lw.max())
    return w / w.sum()


def _pair_marginals(P, S, L, q):
    out = np.zeros((L, L, q, q))
    for i in range(L):
        for j in range(L):
            np.add.at(out[i, j], (S[:, i], S[:, j]), P)
    return out


def _elements(L, q):
    """(i, j, a, b) of every element, in the oracle's numbering."""
    return [(i, j, a, b) for i in range(L) for j in range(i + 1, L) for a in range(q) for b in range(q)]


@pytest.mark.parametrize("L,q,seed", [(3, 3, 1), (4, 2, 2), (3, 4, 3)])
def test_decimation_score_is_the_exact_symmetric_kl(L, q, seed):
    rng = np.random.default_rng(seed)
    h, J = _symmetric_model(L, q, rng)
    S = _states(L, q)
    P = _probs(h, J, S)
    pij = _pair_marginals(P, S, L, q)
    active = np.ones((L, L, q, q), dtype=np.uint8)
    score = orc.decimation_scores(J, pij, active)
    for e, (i, j, a, b) in enumerate(_elements(L, q)):
        J2 = J.copy()
        J2[i, j, a, b] = 0.0
        J2[j, i, b, a] = 0.0
        P2 = _probs(h, J2, S)
        d = np.sum(P * np.log(P / P2)) + np.sum(P2 * np.log(P2 / P))
        assert abs(score[e] - d) < 1e-12 * max(1.0, abs(d)), (e, score[e], d)


def test_decimation_score_of_a_zero_coupling_is_zero_and_inactive_is_infinite():
    rng = np.random.default_rng(4)
    L, q = 3, 3
    h, J = _symmetric_model(L, q, rng)
    J[0, 1, 2, 1] = J[1, 0, 1, 2] = 0.0
    active = np.ones((L, L, q, q), dtype=np.uint8)
    active[0, 2, 1, 1] = active[2, 0, 1, 1] = 0
    S = _states(L, q)
    pij = _pair_marginals(_probs(h, J, S), S, L, q)
    score = orc.decimation_scores(J, pij, active)
    els = _elements(L, q)
    assert score[els.index((0, 1, 2, 1))] == 0.0
    assert np.isinf(score[els.index((0, 2, 1, 1))])
    assert np.all(score[np.isfinite(score)] >= 0.0)


@pytest.mark.parametrize("L,q,seed", [(3, 2, 5), (3, 3, 6)])
def test_activation_score_is_the_single_coupling_likelihood_gain(L, q, seed):
    rng = np.random.default_rng(seed)
    h, J = _symmetric_model(L, q, rng, scale=0.5)
    S = _states(L, q)
    P = _probs(h, J, S)
    D = rng.dirichlet(np.ones(len(S)))  # a data distribution over all states, strictly positive
    fij = _pair_marginals(D, S, L, q)
    pij = _pair_marginals(P, S, L, q)
    score = orc.activation_scores(fij, pij)
    lw0 = _log_weights(h, J, S)
    for e, (i, j, a, b) in enumerate(_elements(L, q)):
        on = ((S[:, i] == a) & (S[:, j] == b)).astype(float)

        def neg_ll(d):  # data log-likelihood with J_ij(a,b) += d, by enumeration
            lw = lw0 + d * on
            return -(np.sum(D * lw) - (np.log(np.sum(np.exp(lw - lw.max()))) + lw.max()))

        best = scipy_opt.minimize_scalar(neg_ll, bounds=(-30, 30), method="bounded",
                                         options={"xatol": 1e-12})
        gain = neg_ll(0.0) - best.fun
        assert abs(score[e] - gain) < 1e-7, (e, score[e], gain)


def test_activation_score_closed_cases():
    # f = p: nothing to gain; p = 0 < f: infinite
    L, q = 2, 2
    fij = np.zeros((L, L, q, q))
    pij = np.zeros((L, L, q, q))
    fij[0, 1] = [[0.25, 0.25], [0.25, 0.25]]
    pij[0, 1] = [[0.25, 0.25], [0.5, 0.0]]
    s = orc.activation_scores(fij, pij)
    assert s[0] == 0.0 and s[1] == 0.0
    assert np.isinf(s[3])
    assert abs(s[2] - (0.25 * np.log(0.5) + 0.75 * np.log(0.75 / 0.5))) < 1e-15


def _random_graph(L, q, rng, density):
    act = np.zeros((L, L, q, q), dtype=np.uint8)
    for i in range(L):
        for j in range(i + 1, L):
            m = (rng.random((q, q)) < density).astype(np.uint8)
            act[i, j] = m
            act[j, i] = m.T
    return act


@pytest.mark.parametrize("n", [0, 1, 7, 40, 10 ** 6])
def test_graph_decimate_removes_the_smallest_scores(n):
    rng = np.random.default_rng(7)
    L, q = 6, 3
    _, J = _symmetric_model(L, q, rng)
    act = _random_graph(L, q, rng, 0.6)
    J = J * act
    els = _elements(L, q)
    score = np.round(rng.random(len(els)) * 8) / 8  # many exact ties
    score = np.where([act[e] for e in els], score, np.inf)
    J2, act2, removed = orc.graph_decimate(J, act, score, n)
    was = np.array([act[e] for e in els], dtype=bool)
    now = np.array([act2[e] for e in els], dtype=bool)
    gone = was & ~now
    assert removed == min(n, was.sum()) == gone.sum()
    assert not np.any(now & ~was)
    kept = was & now
    if gone.any() and kept.any():
        # smallest scores first; on the boundary score, lower element numbers first
        assert score[gone].max() <= score[kept].min()
        t = score[gone].max()
        tie_gone = np.flatnonzero(gone & (score == t))
        tie_kept = np.flatnonzero(kept & (score == t))
        if tie_kept.size:
            assert tie_gone.max() < tie_kept.min()
    assert np.array_equal(act2, act2.transpose(1, 0, 3, 2))
    for e in np.flatnonzero(gone):
        i, j, a, b = els[e]
        assert J2[i, j, a, b] == 0.0 and J2[j, i, b, a] == 0.0
    untouched = np.ones_like(J, dtype=bool)
    for e in np.flatnonzero(gone):
        i, j, a, b = els[e]
        untouched[i, j, a, b] = untouched[j, i, b, a] = False
    assert np.array_equal(J2[untouched], J[untouched])


@pytest.mark.parametrize("n", [0, 5, 30, 10 ** 6])
def test_graph_activate_takes_the_largest_scores(n):
    rng = np.random.default_rng(8)
    L, q = 5, 3
    act = _random_graph(L, q, rng, 0.3)
    els = _elements(L, q)
    score = np.round(rng.random(len(els)) * 6) / 6
    score[3] = np.inf
    act2, fresh = orc.graph_activate(act, score, n)
    was = np.array([act[e] for e in els], dtype=bool)
    now = np.array([act2[e] for e in els], dtype=bool)
    assert not np.any(was & ~now)
    order = sorted(range(len(els)), key=lambda e: (-score[e], e))
    chosen = np.zeros(len(els), dtype=bool)
    chosen[order[:min(n, len(els))]] = True
    assert np.array_equal(now, was | chosen)
    assert fresh == int((chosen & ~was).sum())
    assert np.array_equal(act2, act2.transpose(1, 0, 3, 2))


def test_masked_update_keeps_inactive_couplings_at_zero():
    rng = np.random.default_rng(9)
    L, q, M = 5, 3, 50
    h, J = _symmetric_model(L, q, rng)
    act = _random_graph(L, q, rng, 0.5)
    J = J * act
    fi = rng.dirichlet(np.ones(q), L)
    fij = rng.random((L, L, q, q)) / q ** 2
    fij = (fij + fij.transpose(1, 0, 3, 2)) / 2
    S = rng.integers(0, q, (M, L)).astype(np.uint8)
    C = orc.chain_stats(S, q)
    h1, J1 = orc.update_masked(h, J, fi, fij, C, M, 0.1, act)
    h2, J2 = orc.update(h, J, fi, fij, C, M, 0.1)
    assert np.array_equal(h1, h2)
    assert np.all(J1[act == 0] == 0.0)
    on = act == 1
    assert np.array_equal(J1[on], J2[on])
    assert np.array_equal(J1, J1.transpose(1, 0, 3, 2))
