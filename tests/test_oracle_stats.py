"""Pins of the oracle's statistics: chain counts, sequence weights (Eq. 7),
weighted frequencies with pseudocount (Eqs. 3, 8-9), the Pearson check and
the Boltzmann update (Eq. 5).

References: numpy one-hot einsum counts, an O(N^2 L) numpy identity matrix,
np.corrcoef, sum rules and closed-form special cases.
"""
import numpy as np
import pytest

from paper_2501_18456_gb300 import synth


def onehot(S, q):
    N, L = S.shape
    X = np.zeros((N, L, q))
    X[np.arange(N)[:, None], np.arange(L)[None, :], S] = 1.0
    return X


def full_counts_from_blocks(C, L, q, orc):
    F = np.zeros((L, L, q, q), dtype=np.int64)
    for i in range(L):
        for j in range(i, L):
            B = C[orc.block_index(L, i, j)]
            F[i, j] = B
            F[j, i] = B.T
    return F


def test_block_index_layout(orc):
    L = 7
    seen = []
    for i in range(L):
        for j in range(i, L):
            seen.append(orc.block_index(L, i, j))
    assert seen == list(range(orc.n_blocks(L)))


@pytest.mark.parametrize("M,L,q", [(1, 1, 1), (57, 9, 5), (300, 6, 21)])
def test_chain_stats_matches_einsum(orc, M, L, q):
    S = synth.random_states(M, L, q, 7)
    C = orc.chain_stats(S, q)
    X = onehot(S, q)
    ref = np.einsum("mia,mjb->ijab", X, X).astype(np.int64)
    assert np.array_equal(full_counts_from_blocks(C, L, q, orc), ref)


def test_chain_stats_sum_rules(orc):
    M, L, q = 123, 8, 6
    S = synth.random_states(M, L, q, 8)
    C = orc.chain_stats(S, q).astype(np.int64)
    F = full_counts_from_blocks(C, L, q, orc)
    for i in range(L):
        ci = np.diag(F[i, i])
        assert ci.sum() == M
        assert np.array_equal(F[i, i], np.diag(ci))  # off-diagonal of (i,i) is zero
        for j in range(L):
            assert np.array_equal(F[i, j].sum(axis=1), ci)


def identity_matrix(S):
    return (S[:, None, :] == S[None, :, :]).sum(axis=2)


@pytest.mark.parametrize("N,L,seqid", [(1, 5, 0.8), (200, 40, 0.8), (150, 120, 0.8), (90, 33, 0.5)])
def test_seq_weights_brute_force(orc, N, L, seqid):
    S = synth.clustered_msa(N, L, 21, 3, n_ancestors=max(1, N // 8))
    w, meff = orc.seq_weights(S, seqid)
    ident = identity_matrix(S)
    thr = orc.identity_threshold(seqid, L)
    assert thr == int(np.ceil(seqid * L - 1e-9))
    Nm = (ident >= thr).sum(axis=1)
    assert np.allclose(w, 1.0 / Nm, rtol=0, atol=0)
    assert meff == pytest.approx((1.0 / Nm).sum(), rel=1e-14)


def test_identity_threshold_reading(orc):
    # "identity >= 0.8 L": L = 256 -> 205 positions; L = 120 -> exactly 96
    assert orc.identity_threshold(0.8, 256) == 205
    assert orc.identity_threshold(0.8, 120) == 96
    assert orc.identity_threshold(0.8, 5) == 4


def test_seq_weights_special_cases(orc):
    L = 30
    same = np.tile(synth.random_states(1, L, 21, 1), (17, 1))
    w, meff = orc.seq_weights(same)
    assert np.allclose(w, 1 / 17) and meff == pytest.approx(1.0)
    far = np.array([[k % 21] * L for k in range(21)], dtype=np.uint8)  # pairwise identity 0
    w, meff = orc.seq_weights(far)
    assert np.all(w == 1.0) and meff == 21.0


def test_data_stats_matches_einsum(orc):
    N, L, q = 400, 7, 5
    S = synth.clustered_msa(N, L, q, 9, n_ancestors=40)
    w = np.random.default_rng(2).uniform(0.1, 1.0, size=N)
    alpha = 0.13
    fi, fij = orc.data_stats(S, w, q, alpha)
    X = onehot(S, q)
    meff = w.sum()
    f1 = np.einsum("m,mia->ia", w, X) / meff
    f2 = np.einsum("m,mia,mjb->ijab", w, X, X) / meff
    assert np.allclose(fi, (1 - alpha) * f1 + alpha / q, atol=1e-14)
    for i in range(L):
        for j in range(L):
            if i == j:
                assert np.allclose(fij[i, i], np.diag(fi[i]), atol=1e-14)
            else:
                assert np.allclose(fij[i, j], (1 - alpha) * f2[i, j] + alpha / q**2, atol=1e-14)


def test_data_stats_pseudocount_limits_and_sum_rules(orc):
    N, L, q = 100, 5, 4
    S = synth.clustered_msa(N, L, q, 10, n_ancestors=10)
    fi, fij = orc.data_stats(S, None, q, 1.0)
    assert np.allclose(fi, 1 / q) and np.allclose(fij[0, 1], 1 / q**2)
    fi, fij = orc.data_stats(S, None, q, 0.2)
    assert np.allclose(fi.sum(axis=1), 1.0)
    for i in range(L):
        for j in range(L):
            if i != j:
                assert np.allclose(fij[i, j].sum(axis=1), fi[i], atol=1e-14)
                assert np.allclose(fij[i, j], fij[j, i].T)
    # alpha = 0, uniform weights: plain frequencies
    fi0, _ = orc.data_stats(S, None, q, 0.0)
    assert np.allclose(fi0, onehot(S, q).mean(axis=0))


def connected(fi, fij):
    L, q = fi.shape
    xs = []
    for i in range(L):
        for j in range(i + 1, L):
            xs.append((fij[i, j] - np.outer(fi[i], fi[j])).ravel())
    return np.concatenate(xs)


def test_pearson_matches_corrcoef(orc):
    N, L, q, M = 300, 8, 5, 250
    data = synth.clustered_msa(N, L, q, 11, n_ancestors=30)
    fi, fij = orc.data_stats(data, None, q, 0.05)
    S = synth.random_states(M, L, q, 12)
    C = orc.chain_stats(S, q)
    rho = orc.pearson(fi, fij, C, M)
    X = onehot(S, q)
    p1 = X.mean(axis=0)
    p2 = np.einsum("mia,mjb->ijab", X, X) / M
    want = np.corrcoef(connected(fi, fij), connected(p1, p2))[0, 1]
    assert rho == pytest.approx(want, abs=1e-12)


def test_pearson_identical_statistics_is_one(orc):
    M, L, q = 500, 6, 4
    S = synth.clustered_msa(M, L, q, 13, n_ancestors=20)
    fi, fij = orc.data_stats(S, None, q, 0.0)  # exact chain frequencies
    rho = orc.pearson(fi, fij, orc.chain_stats(S, q), M)
    assert rho == pytest.approx(1.0, abs=1e-12)


def test_update_closed_form_and_symmetry(orc):
    N, L, q, M = 200, 6, 5, 150
    rng = np.random.default_rng(4)
    h = rng.normal(size=(L, q))
    J = np.zeros((L, L, q, q))
    for i in range(L):
        for j in range(i + 1, L):
            B = rng.normal(size=(q, q))
            J[i, j], J[j, i] = B, B.T
    fi, fij = orc.data_stats(synth.clustered_msa(N, L, q, 14, n_ancestors=20), None, q, 0.1)
    S = synth.random_states(M, L, q, 15)
    C = orc.chain_stats(S, q)
    lr = 0.05
    h2, J2 = orc.update(h, J, fi, fij, C, M, lr)
    X = onehot(S, q)
    p1 = X.mean(axis=0)
    p2 = np.einsum("mia,mjb->ijab", X, X) / M
    assert np.allclose(h2, h + lr * (fi - p1), atol=1e-14)
    for i in range(L):
        for j in range(L):
            if i == j:
                assert np.all(J2[i, i] == 0)
            else:
                assert np.allclose(J2[i, j], J[i, j] + lr * (fij[i, j] - p2[i, j]), atol=1e-14)
    assert np.array_equal(J2, J2.transpose(1, 0, 3, 2))


def test_update_fixed_point(orc):
    """f = p leaves the parameters unchanged (Eq. 5 at convergence)."""
    M, L, q = 64, 5, 3
    S = synth.random_states(M, L, q, 16)
    fi, fij = orc.data_stats(S, None, q, 0.0)
    h = np.random.default_rng(1).normal(size=(L, q))
    J = np.zeros((L, L, q, q))
    h2, J2 = orc.update(h, J, fi, fij, orc.chain_stats(S, q), M, 0.3)
    assert np.allclose(h2, h, atol=1e-15) and np.allclose(J2, 0, atol=1e-15)


def all_states(L, q):
    return np.array(np.meshgrid(*[np.arange(q)] * L, indexing="ij")).reshape(L, -1).T.astype(np.uint8)


def exact_log_likelihood(orc, h, J, msa, S_all):
    """Mean of -E over the data minus log Z, Z by enumeration of all q^L states."""
    e_all = -orc.energy(h, J, S_all)
    top = e_all.max()
    return float(-orc.energy(h, J, msa).mean() - (top + np.log(np.exp(e_all - top).sum())))


@pytest.mark.parametrize("point", ["uniform", "integer_weights"])
def test_update_is_log_likelihood_gradient(orc, point):
    """Eq. 5 is gradient ascent on the data log-likelihood.  When the chain
    ensemble holds the model's marginals exactly, (theta' - theta) / lr must
    equal the central finite difference of the log-likelihood computed by
    enumeration from energies alone.  A coupling J_ij(a, b) is tied to
    J_ji(b, a), so both move together.  This pins the sign of the step, the
    pair indexing and the transposed half of J without restating Eq. 5.
    Exact model marginals: at theta = 0 the chain ensemble is every state
    once; at a model whose Boltzmann weights exp(-E) are integers it is every
    state repeated by its weight."""
    L, q = 3, 3
    S_all = all_states(L, q)
    rng = np.random.default_rng(5)
    h = np.zeros((L, q))
    J = np.zeros((L, L, q, q))
    if point == "uniform":
        chains = S_all
    else:
        h = np.log(rng.integers(1, 4, size=(L, q)).astype(np.float64))
        for i in range(L):
            for j in range(i + 1, L):
                B = np.log(rng.integers(1, 3, size=(q, q)).astype(np.float64))
                J[i, j], J[j, i] = B, B.T
        w = np.exp(-orc.energy(h, J, S_all))
        mult = np.rint(w).astype(np.int64)
        assert np.allclose(w, mult, rtol=1e-12, atol=0) and mult.min() >= 1
        chains = np.repeat(S_all, mult, axis=0)
    M = chains.shape[0]
    msa = synth.random_states(40, L, q, 6)
    fi, fij = orc.data_stats(msa, None, q, 0.0)
    lr = 0.1
    h2, J2 = orc.update(h, J, fi, fij, orc.chain_stats(chains, q), M, lr)
    eps = 1e-5

    def grad(hp, Jp, hm, Jm):
        return (exact_log_likelihood(orc, hp, Jp, msa, S_all)
                - exact_log_likelihood(orc, hm, Jm, msa, S_all)) / (2 * eps)

    for i in range(L):
        for a in range(q):
            hp, hm = h.copy(), h.copy()
            hp[i, a] += eps
            hm[i, a] -= eps
            assert abs((h2[i, a] - h[i, a]) / lr - grad(hp, J, hm, J)) < 1e-7
    for i in range(L):
        for j in range(i + 1, L):
            for a in range(q):
                for b in range(q):
                    Jp, Jm = J.copy(), J.copy()
                    Jp[i, j, a, b] += eps
                    Jp[j, i, b, a] += eps
                    Jm[i, j, a, b] -= eps
                    Jm[j, i, b, a] -= eps
                    g = grad(h, Jp, h, Jm)
                    assert abs((J2[i, j, a, b] - J[i, j, a, b]) / lr - g) < 1e-7
                    assert abs((J2[j, i, b, a] - J[j, i, b, a]) / lr - g) < 1e-7
    # the step is not vacuous: the data differ from the model
    assert np.abs(h2 - h).max() > 1e-3 and np.abs(J2 - J).max() > 1e-3


def test_update_iterates_to_generating_model(orc):
    """Iterating Eq. 5 on exact statistics recovers the model that generated
    them: the data side is the exact enumeration of a planted model (L=3,
    q=3, no pseudocount), the model side at every step the exact enumeration
    of the current parameters (as integer counts scaled by K = 2^24, exact to
    6e-8). From h = J = 0 the iteration must reach the planted model up to
    gauge: equal energy differences E(s) - E(s0) over all 27 states."""
    L, q, K = 3, 3, 1 << 24
    S_all = all_states(L, q)
    h0, J0 = synth.planted_local_model(L, q, 21, sigma_h=0.8, sigma_J=0.8)
    h0, J0 = h0.astype(np.float64), J0.astype(np.float64)

    def probs(h, J):
        e = -orc.energy(h, J, S_all)
        w = np.exp(e - e.max())
        return w / w.sum()

    fi, fij = orc.data_stats(S_all, probs(h0, J0), q, 0.0)
    X = np.zeros((S_all.shape[0], L, q))
    X[np.arange(S_all.shape[0])[:, None], np.arange(L)[None, :], S_all] = 1.0
    h, J = np.zeros((L, q)), np.zeros((L, L, q, q))
    for _ in range(3000):
        pij = np.einsum("s,sia,sjb->ijab", probs(h, J), X, X)
        C = np.zeros((orc.n_blocks(L), q, q), dtype=np.int64)
        for i in range(L):
            for j in range(i, L):
                C[orc.block_index(L, i, j)] = np.rint(K * pij[i, j])
        h, J = orc.update(h, J, fi, fij, C.astype(np.int32), K, 1.0)
    dE = orc.energy(h, J, S_all) - orc.energy(h, J, S_all[:1])
    dE0 = orc.energy(h0, J0, S_all) - orc.energy(h0, J0, S_all[:1])
    assert np.abs(dE - dE0).max() < 1e-3, np.abs(dE - dE0).max()
    assert np.abs(dE0).max() > 1.0  # the planted model is far from uniform
