"""Seeded synthetic inputs for the bmDCA hot path.

Shared by the tests, the benchmark and the oracle checks.  This module only
draws random inputs (numpy PCG64 streams keyed by the seed); it contains none
of the method's arithmetic (no energies, no sampling, no statistics).

Inputs mimic protein / RNA families (alphabets of Table 1: q = 21 for
proteins, q = 5 for RNA/DNA, gap = symbol 0):

  planted_local_model    h ~ N(0, sh^2), symmetric J_ij(a,b) ~ N(0, sJ^2) for
                         1 <= |i-j| <= width, else 0
  planted_contact_model  h ~ N(0, sh^2); couplings on a sparse contact map:
                         every pair with |i-j| <= short plus random long-range
                         pairs up to a fraction `frac` of all pairs,
                         J ~ N(0, sJ^2) on those pairs
  random_states          uniform symbols
  clustered_msa          family-like alignment: ancestors with a site-specific
                         profile and ~gap_frac gaps, descendants obtained by
                         resampling a per-descendant fraction of sites, so
                         close relatives exceed 80% identity and sequence
                         reweighting matters
  cluster_mix            the same clustering over given sequences: each of N
                         descendants copies ancestor k mod n_anc and takes a
                         per-descendant U[lo, hi] fraction of its sites from
                         its own donor sequence (a random selection only)
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed, stream]))


def _symmetrize_pairs(J: np.ndarray, pairs, blocks: np.ndarray) -> None:
    """Write block k to (i,j) and its transpose to (j,i) for pairs[k] = (i, j)."""
    for k, (i, j) in enumerate(pairs):
        J[i, j] = blocks[k]
        J[j, i] = blocks[k].T


def planted_local_model(L: int, q: int, seed: int, sigma_h: float = 0.5, sigma_J: float = 0.05,
                        width: int = 3):
    rng = _rng(seed, 1)
    h = rng.normal(0.0, sigma_h, size=(L, q)).astype(np.float32)
    J = np.zeros((L, L, q, q), dtype=np.float32)
    pairs = [(i, j) for i in range(L) for j in range(i + 1, min(L, i + width + 1))]
    blocks = rng.normal(0.0, sigma_J, size=(len(pairs), q, q)).astype(np.float32)
    _symmetrize_pairs(J, pairs, blocks)
    return h, J


def contact_pairs(L: int, seed: int, frac: float = 0.03, short: int = 2):
    """Sparse contact map: all pairs with 1 <= j-i <= short plus random
    long-range pairs until round(frac * L(L-1)/2) pairs are in."""
    rng = _rng(seed, 2)
    pairs = [(i, j) for i in range(L) for j in range(i + 1, min(L, i + short + 1))]
    total = int(round(frac * L * (L - 1) / 2))
    chosen = set(pairs)
    far = [(i, j) for i in range(L) for j in range(i + short + 1, L)]
    need = max(0, total - len(pairs))
    if need and far:
        idx = rng.choice(len(far), size=min(need, len(far)), replace=False)
        for k in sorted(idx.tolist()):
            chosen.add(far[k])
    return sorted(chosen)


def planted_contact_model(L: int, q: int, seed: int, frac: float = 0.03, sigma_h: float = 1.0,
                          sigma_J: float = 0.2, short: int = 2):
    rng = _rng(seed, 3)
    h = rng.normal(0.0, sigma_h, size=(L, q)).astype(np.float32)
    J = np.zeros((L, L, q, q), dtype=np.float32)
    pairs = contact_pairs(L, seed, frac, short)
    blocks = rng.normal(0.0, sigma_J, size=(len(pairs), q, q)).astype(np.float32)
    _symmetrize_pairs(J, pairs, blocks)
    return h, J


def random_states(M: int, L: int, q: int, seed: int) -> np.ndarray:
    return _rng(seed, 4).integers(0, q, size=(M, L), dtype=np.uint8)


def clustered_msa(N: int, L: int, q: int, seed: int, n_ancestors: int | None = None,
                  gap_frac: float = 0.2, resample_lo: float = 0.02, resample_hi: float = 0.3,
                  conc: float = 0.5) -> np.ndarray:
    """N sequences in clusters of ~N/n_ancestors around random ancestors."""
    rng = _rng(seed, 5)
    if n_ancestors is None:
        n_ancestors = max(1, N // 10)
    # Site profiles over the q-1 non-gap symbols (Dirichlet: conserved sites).
    prof = rng.dirichlet(np.full(max(q - 1, 1), conc), size=L)

    def sample_sites(n: int) -> np.ndarray:
        out = np.zeros((n, L), dtype=np.uint8)
        if q == 1:
            return out
        gap = rng.random((n, L)) < gap_frac
        for i in range(L):
            out[:, i] = 1 + rng.choice(q - 1, size=n, p=prof[i])
        out[gap] = 0
        return out

    anc = sample_sites(n_ancestors)
    owner = np.arange(N) % n_ancestors
    X = anc[owner].copy()
    rate = rng.uniform(resample_lo, resample_hi, size=(N, 1))
    mask = rng.random((N, L)) < rate
    fresh = sample_sites(N)
    X[mask] = fresh[mask]
    return X[rng.permutation(N)]


def cluster_mix(ancestors: np.ndarray, donors: np.ndarray, seed: int, resample_lo: float = 0.02,
                resample_hi: float = 0.3) -> np.ndarray:
    """Descendant m = ancestors[m % n_anc] with a U[lo, hi] fraction of its
    sites (chosen at random) replaced by donors[m]; rows shuffled."""
    rng = _rng(seed, 6)
    anc = np.ascontiguousarray(ancestors, dtype=np.uint8)
    don = np.ascontiguousarray(donors, dtype=np.uint8)
    N, L = don.shape
    X = anc[np.arange(N) % anc.shape[0]].copy()
    rate = rng.uniform(resample_lo, resample_hi, size=(N, 1))
    mask = rng.random((N, L)) < rate
    X[mask] = don[mask]
    return X[rng.permutation(N)]
