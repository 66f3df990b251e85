"""Pins of the oracle's Metropolis-Hastings sampler (Sec. 2.1, the --sampler
option; proposal uniform over the other q-1 symbols, acceptance
min(1, exp(beta dH))).

Independent references: the exact stationary distribution P(s) ~ exp(-E(s))
by enumeration of all q^L states (with E from the one-hot quadratic form in
numpy), the closed-form single-site transition probabilities
P(a -> b) = min(1, exp(beta (H_b - H_a))) / (q - 1) with H from enumeration
of conditionals, the beta = 0 limit (every proposal accepted: a uniform
random walk over the other symbols), and a planted error in the
teacher-forced verifier.
"""
import itertools

import numpy as np
import pytest

from test_oracle_model import quad_energy, random_model


def exact_distribution(h, J, beta=1.0):
    L, q = h.shape
    states = np.array(list(itertools.product(range(q), repeat=L)), dtype=np.uint8)
    E = np.array([quad_energy(h, J, s) for s in states])
    w = np.exp(-beta * (E - E.min()))
    return states, w / w.sum()


@pytest.mark.parametrize("beta", [1.0, 0.7])
def test_metropolis_stationary_distribution_matches_enumeration(orc, beta):
    L, q, M = 3, 3, 30000
    h, J = random_model(L, q, 41, sh=0.8, sJ=0.6)
    states, P = exact_distribution(h, J, beta)
    s0 = orc.chains_init(M, L, q, 5)
    S = orc.metropolis(h, J, s0, 5, 0, 40, beta)
    idx = (S.astype(np.int64) * (q ** np.arange(L - 1, -1, -1))).sum(axis=1)
    counts = np.bincount(idx, minlength=q ** L)
    expect = P * M
    z = (counts - expect) / np.sqrt(expect * (1 - P))
    assert np.abs(z).max() < 4.5, np.abs(z).max()
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 26 + 5 * np.sqrt(2 * 26)  # 26 degrees of freedom


def test_metropolis_single_site_transition_closed_form(orc):
    """From one fixed state, the first site's update over many independent
    chains follows P(a -> b) = min(1, exp(dH)) / (q-1), b != a."""
    L, q, M = 3, 4, 200000
    h, J = random_model(L, q, 7, sh=1.0, sJ=0.5)
    start = np.array([2, 1, 3], dtype=np.uint8)
    s0 = np.tile(start, (M, 1))
    S = orc.metropolis(h, J, s0, 11, 0, 1, 1.0)
    # site 0 is updated first and not again in the sweep
    H = orc.fields(h, J, start, 0)
    a = start[0]
    p = np.array([0.0 if b == a else min(1.0, np.exp(H[b] - H[a])) / (q - 1) for b in range(q)])
    p[a] = 1.0 - p.sum()
    counts = np.bincount(S[:, 0], minlength=q)
    z = (counts - M * p) / np.sqrt(M * p * (1 - p))
    assert np.abs(z).max() < 4.5, (counts, M * p)


def test_metropolis_beta_zero_accepts_every_proposal(orc):
    """beta = 0: every proposal is accepted, so each site moves to another
    symbol at every update, and the long-run states are uniform."""
    L, q, M = 4, 5, 4000
    h, J = random_model(L, q, 3)
    s0 = orc.chains_init(M, L, q, 2)
    s1 = orc.metropolis(h, J, s0, 2, 0, 1, 0.0)
    assert np.all(s1 != s0)
    S = orc.metropolis(h, J, s0, 2, 0, 30, 0.0)
    counts = np.bincount(S.ravel(), minlength=q)
    assert np.abs(counts / S.size - 1 / q).max() < 0.02


def test_metropolis_single_symbol_alphabet_is_a_no_op(orc):
    h = np.zeros((3, 1))
    J = np.zeros((3, 3, 1, 1))
    s0 = np.zeros((5, 3), dtype=np.uint8)
    assert np.array_equal(orc.metropolis(h, J, s0, 1, 0, 3, 1.0), s0)


def test_metropolis_verify_accepts_oracle_and_records_planted_error(orc):
    L, q = 6, 5
    h, J = random_model(L, q, 19)
    s0 = orc.chains_init(50, L, q, 8, chain0=7)
    s1 = orc.metropolis(h, J, s0, 8, 3, 1, 1.0, chain0=7)
    bad, mn, flips = orc.metropolis_flips(h, J, s0, s1, 8, 3, 1.0, chain0=7)
    assert bad == 0 and flips == [] and mn > 0
    wrong = s1.copy()
    wrong[4, 1] = (s1[4, 1] + 1) % q
    bad, _, flips = orc.metropolis_flips(h, J, s0, wrong, 8, 3, 1.0, chain0=7)
    assert bad >= 1 and (flips[0]["chain"], flips[0]["site"]) == (11, 1)
    assert flips[0]["want"] == s1[4, 1]
    # the Gibbs sweep of the same chains is not a Metropolis sweep
    g = orc.gibbs(h, J, s0, 8, 3, 1, 1.0, chain0=7)
    assert orc.metropolis_flips(h, J, s0, g, 8, 3, 1.0, chain0=7)[0] > 0
