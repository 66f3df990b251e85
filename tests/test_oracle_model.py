"""Pins of the oracle's energy, conditionals, mutant scan and Gibbs sampler.

Independent references: the one-hot quadratic form of Eq. 1 written with
numpy, exact enumeration of all q^L states on tiny models, gauge
transformations that leave energy differences invariant, and the exact
stationary distribution for the sampler.
"""
import itertools

import numpy as np
import pytest

from paper_2501_18456_gb300 import synth


def random_model(L, q, seed, sh=0.7, sJ=0.4):
    rng = np.random.default_rng(seed)
    h = rng.normal(0, sh, size=(L, q))
    J = np.zeros((L, L, q, q))
    for i in range(L):
        for j in range(i + 1, L):
            B = rng.normal(0, sJ, size=(q, q))
            J[i, j] = B
            J[j, i] = B.T
    return h, J


def quad_energy(h, J, s):
    """E(s) = -x.h - 1/2 x^T Jf x with x the one-hot vector and Jf the
    (Lq x Lq) coupling matrix whose diagonal blocks are zero."""
    L, q = h.shape
    x = np.zeros(L * q)
    x[np.arange(L) * q + np.asarray(s)] = 1.0
    Jf = J.transpose(0, 2, 1, 3).reshape(L * q, L * q)
    return -x @ h.ravel() - 0.5 * x @ Jf @ x


def all_states(L, q):
    return np.array(list(itertools.product(range(q), repeat=L)), dtype=np.uint8)


def test_energy_matches_quadratic_form(orc):
    h, J = random_model(6, 4, 1)
    S = synth.random_states(50, 6, 4, 2)
    E = orc.energy(h, J, S)
    for k in range(len(S)):
        assert E[k] == pytest.approx(quad_energy(h, J, S[k]), abs=1e-12)


def test_energy_sign_convention(orc):
    """Single site, no couplings: E = -h(s), so a larger field means a lower energy."""
    h = np.array([[0.0, 2.0, -1.0]])
    J = np.zeros((1, 1, 3, 3))
    assert list(orc.energy(h, J, np.array([[0], [1], [2]], dtype=np.uint8))) == [0.0, -2.0, 1.0]


def test_energy_gauge_invariance(orc):
    """J_ij(a,b) += g(a), J_ji(b,a) += g(a), h_i(a) -= g(a) leaves E unchanged;
    a per-site constant added to h shifts every energy by the same amount."""
    L, q = 5, 4
    h, J = random_model(L, q, 3)
    S = synth.random_states(40, L, q, 4)
    E0 = orc.energy(h, J, S)
    rng = np.random.default_rng(5)
    h2, J2 = h.copy(), J.copy()
    for (i, j) in [(0, 2), (3, 1), (4, 0)]:
        g = rng.normal(size=q)
        J2[i, j] += g[:, None]
        J2[j, i] += g[None, :]
        h2[i] -= g
    assert np.allclose(orc.energy(h2, J2, S), E0, atol=1e-12)
    h3 = h.copy()
    h3[2] += 0.75
    E3 = orc.energy(h3, J, S)
    assert np.allclose(E3 - E0, -0.75, atol=1e-12)


@pytest.mark.parametrize("L,q", [(3, 3), (4, 3), (3, 5), (2, 21)])
def test_conditional_matches_enumeration(orc, L, q):
    h, J = random_model(L, q, 10 + L * q)
    S = all_states(L, q)
    E = orc.energy(h, J, S)
    p = np.exp(-(E - E.min()))
    p /= p.sum()
    ptab = p.reshape((q,) * L)
    rng = np.random.default_rng(0)
    for s in S[rng.choice(len(S), size=min(20, len(S)), replace=False)]:
        for i in range(L):
            idx = list(s)
            sl = []
            for a in range(q):
                idx[i] = a
                sl.append(ptab[tuple(idx)])
            want = np.array(sl) / np.sum(sl)
            got = orc.conditional(h, J, s, i)
            assert np.allclose(got, want, atol=1e-12, rtol=1e-12)


def test_conditional_beta_matches_enumeration(orc):
    L, q, beta = 3, 4, 1.3
    h, J = random_model(L, q, 21)
    S = all_states(L, q)
    E = orc.energy(h, J, S)
    w = np.exp(-beta * (E - E.min())).reshape((q,) * L)
    s = np.array([1, 3, 0], dtype=np.uint8)
    want = w[1, :, 0] / w[1, :, 0].sum()
    assert np.allclose(orc.conditional(h, J, s, 1, beta), want, atol=1e-12)


def test_three_site_protein_alphabet_enumeration(orc):
    """L = 3, q = 21 (9261 states): fields from enumeration."""
    L, q = 3, 21
    h, J = random_model(L, q, 77, sh=1.0, sJ=0.3)
    S = all_states(L, q)
    E = orc.energy(h, J, S).reshape((q,) * L)
    s = np.array([4, 0, 17], dtype=np.uint8)
    # H_i(a) - H_i(b) = -(E(..a..) - E(..b..))
    H = orc.fields(h, J, s, 2)
    dE = E[4, 0, :] - E[4, 0, 0]
    assert np.allclose(H - H[0], -dE, atol=1e-12)


def test_fields_by_definition(orc):
    L, q = 7, 5
    h, J = random_model(L, q, 8)
    s = synth.random_states(1, L, q, 9)[0]
    for i in range(L):
        want = h[i] + sum(J[i, j, :, s[j]] for j in range(L) if j != i)
        assert np.allclose(orc.fields(h, J, s, i), want, atol=1e-13)


def test_mutant_scan_matches_energy_and_conditional(orc):
    L, q = 6, 5
    h, J = random_model(L, q, 31)
    wt = synth.random_states(1, L, q, 32)[0]
    dE = orc.mutant_scan(h, J, wt)
    E0 = orc.energy(h, J, wt[None])[0]
    for i in range(L):
        assert dE[i, wt[i]] == 0.0
        P = orc.conditional(h, J, wt, i)
        for a in range(q):
            m = wt.copy()
            m[i] = a
            assert dE[i, a] == pytest.approx(orc.energy(h, J, m[None])[0] - E0, abs=1e-12)
            # log P(a)/P(wt_i) = -dE(i,a): ties the sampler's conditional to the scan
            assert np.log(P[a] / P[wt[i]]) == pytest.approx(-dE[i, a], abs=1e-10)


def test_gibbs_stationary_distribution(orc):
    """Long runs of many chains reproduce the exact distribution of a tiny model."""
    L, q = 3, 3
    h, J = random_model(L, q, 41, sh=0.8, sJ=0.6)
    S = all_states(L, q)
    E = orc.energy(h, J, S)
    p = np.exp(-(E - E.min()))
    p /= p.sum()
    M = 20000
    s0 = orc.chains_init(M, L, q, 3)
    s = orc.gibbs(h, J, s0, seed=3, sweep0=0, nsweeps=40)
    idx = (s.astype(np.int64) * (q ** np.arange(L - 1, -1, -1))).sum(axis=1)
    emp = np.bincount(idx, minlength=q ** L) / M
    sd = np.sqrt(p * (1 - p) / M)
    assert np.all(np.abs(emp - p) < 5 * sd + 1e-4)


def test_gibbs_beta_zero_is_uniform(orc):
    L, q = 4, 5
    h, J = random_model(L, q, 43, sh=3.0, sJ=2.0)
    s = orc.gibbs(h, J, orc.chains_init(5000, L, q, 1), seed=9, sweep0=0, nsweeps=2, beta=0.0)
    counts = np.bincount(s.ravel(), minlength=q)
    expect = s.size / q
    assert ((counts - expect) ** 2 / expect).sum() < 30


def test_gibbs_is_sequential_and_keyed(orc):
    """One sweep equals site-by-site redraws with the keyed uniforms; a sweep
    split over two calls (sweep counter continued) equals one call."""
    L, q = 5, 4
    h, J = random_model(L, q, 51)
    s0 = orc.chains_init(7, L, q, 2)
    one = orc.gibbs(h, J, s0, seed=2, sweep0=0, nsweeps=3)
    two = orc.gibbs(h, J, orc.gibbs(h, J, s0, seed=2, sweep0=0, nsweeps=1), seed=2, sweep0=1, nsweeps=2)
    assert np.array_equal(one, two)
    manual = s0.copy()
    for m in range(7):
        for i in range(L):
            H = orc.fields(h, J, manual[m], i)
            u = orc.u24(2, m, 0, i, 0) / 2**24
            manual[m, i] = orc.draw(H, 1.0, u)[0]
    assert np.array_equal(manual, orc.gibbs(h, J, s0, seed=2, sweep0=0, nsweeps=1))


def test_gibbs_verify_accepts_oracle_and_rejects_planted_error(orc):
    L, q = 8, 6
    h, J = random_model(L, q, 61)
    s0 = orc.chains_init(40, L, q, 4)
    s1 = orc.gibbs(h, J, s0, seed=4, sweep0=5, nsweeps=1)
    bad, mx, mn = orc.gibbs_verify(h, J, s0, s1, seed=4, sweep=5)
    assert bad == 0 and mn > 0
    wrong = s1.copy()
    wrong[3, 2] = (wrong[3, 2] + 1) % q
    assert orc.gibbs_verify(h, J, s0, wrong, seed=4, sweep=5)[0] >= 1
    # a different sweep word gives different uniforms
    assert orc.gibbs_verify(h, J, s0, s1, seed=4, sweep=6)[0] > 0


def test_gibbs_flips_records_the_planted_disagreement(orc):
    """The flip record names the chain (global index), the site, the symbol
    found and the oracle's own draw of the first disagreement."""
    L, q = 8, 6
    h, J = random_model(L, q, 61)
    s0 = orc.chains_init(40, L, q, 4, chain0=100)
    s1 = orc.gibbs(h, J, s0, seed=4, sweep0=5, nsweeps=1, chain0=100)
    bad, mn, flips = orc.gibbs_flips(h, J, s0, s1, seed=4, sweep=5, chain0=100)
    assert bad == 0 and flips == [] and mn > 0
    wrong = s1.copy()
    wrong[3, 2] = (s1[3, 2] + 1) % q
    bad, _, flips = orc.gibbs_flips(h, J, s0, wrong, seed=4, sweep=5, chain0=100)
    assert bad >= 1
    first = flips[0]
    assert (first["chain"], first["site"]) == (103, 2)
    assert first["got"] == wrong[3, 2] and first["want"] == s1[3, 2]
    assert bad == orc.gibbs_verify(h, J, s0, wrong, seed=4, sweep=5, chain0=100)[0]
