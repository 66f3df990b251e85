"""FP64 CPU oracle for the bmDCA hot path (adabmDCA 2.0, arXiv 2501.18456).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports, links or executes anything here.

The arithmetic lives in ``bmdca_oracle.c`` (plain C, FP64, loops in the
paper's order).  This module compiles it with gcc into ``oracle/_build`` and
wraps each function with numpy marshalling only.  Citations per function are
in the C file; in short:

  philox4x64 / u24 ........ Philox4x64-10 (Salmon et al. SC'11), the shared
                            random-number definition both sides implement
  chains_init ............. Sec. 2.1 (uniform random chains)
  energy .................. Eq. 1
  fields / conditional .... Eq. 1 with all but one site fixed
  gibbs / gibbs_verify .... Sec. 2.1 (PCD Gibbs sweeps), Sec. 3.3 (sweep)
  metropolis / _flips ..... Sec. 2.1 (Metropolis-Hastings sweeps, the
                            --sampler option)
  chain_stats ............. Sec. 2.1 (p_i, p_ij from the chains)
  seq_weights ............. Eq. 7 (80% identity weights), M_eff Sec. 3.3
  data_stats .............. Eq. 3 + pseudocount Eqs. 8-9
  pearson ................. Sec. 2.1 "Convergence criterium"
  update .................. Eq. 5 (Boltzmann learning step)
  mutant_scan ............. Sec. 4.4 (single-mutant dE)

Parity status of every function is "pinned" (see the CPU tests).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "bmdca_oracle.c"
_OUT = _HERE / "_build" / "liboracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (plain -O2, no fast-math)."""
    _OUT.parent.mkdir(parents=True, exist_ok=True)
    if force or not _OUT.exists() or _OUT.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _OUT.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", str(_SRC),
                               "-o", str(tmp), "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(str(build()))
    P = ctypes.c_void_p
    I, U64, D = ctypes.c_int, ctypes.c_uint64, ctypes.c_double
    sig = {
        "orc_philox4x64_10": (None, [P, P, P]),
        "orc_u24": (ctypes.c_uint32, [U64, U64, U64, U64, U64]),
        "orc_chains_init": (None, [I, I, I, U64, U64, P]),
        "orc_energy": (D, [P, P, I, I, P]),
        "orc_energy_batch": (None, [P, P, I, I, P, I, P]),
        "orc_fields": (None, [P, P, I, I, P, I, P]),
        "orc_draw": (I, [P, I, D, D, P]),
        "orc_conditional": (None, [P, P, I, I, P, I, D, P]),
        "orc_gibbs": (None, [P, P, I, I, I, P, U64, U64, U64, I, D]),
        "orc_gibbs_verify": (ctypes.c_long, [P, P, I, I, I, P, P, U64, U64, U64, D, P, P]),
        "orc_gibbs_verify_rec": (ctypes.c_long, [P, P, I, I, I, P, P, U64, U64, U64, D, P, P,
                                                 ctypes.c_long, P, P, P, P, P]),
        "orc_metropolis": (None, [P, P, I, I, I, P, U64, U64, U64, I, D]),
        "orc_metropolis_verify_rec": (ctypes.c_long, [P, P, I, I, I, P, P, U64, U64, U64, D, P, P,
                                                      ctypes.c_long, P, P, P, P, P]),
        "orc_chain_stats": (None, [P, I, I, I, P]),
        "orc_seq_weights": (None, [P, I, I, I, P, P]),
        "orc_data_stats": (None, [P, P, I, I, I, D, P, P]),
        "orc_pearson": (D, [P, P, P, I, I, I]),
        "orc_update": (None, [P, P, P, P, P, I, D, I, I]),
        "orc_mutant_scan": (None, [P, P, I, I, P, P]),
        "orc_decimation_scores": (None, [P, P, P, I, I, P]),
        "orc_activation_scores": (None, [P, P, I, I, P]),
        "orc_graph_decimate": (ctypes.c_long, [P, P, P, I, I, ctypes.c_long]),
        "orc_graph_activate": (ctypes.c_long, [P, P, I, I, ctypes.c_long]),
        "orc_update_masked": (None, [P, P, P, P, P, I, D, I, I, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def _shape_hJ(h, J):
    h = _f64(h)
    J = _f64(J)
    L, q = h.shape
    assert J.shape == (L, L, q, q)
    return h, J, L, q


# --- random numbers -------------------------------------------------------

def philox4x64(counter, key) -> np.ndarray:
    """One Philox4x64-10 block for a 4-word counter and a 2-word key."""
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def u24(seed: int, chain: int, sweep: int, site: int, tag: int) -> int:
    """Top 24 bits of word 0 of Philox(counter=(chain,sweep,site,tag), key=(seed,0))."""
    return int(_load().orc_u24(seed, chain, sweep, site, tag))


# --- model ---------------------------------------------------------------

def chains_init(M: int, L: int, q: int, seed: int, chain0: int = 0) -> np.ndarray:
    s = np.zeros((M, L), dtype=np.uint8)
    _load().orc_chains_init(M, L, q, seed, chain0, _p(s))
    return s


def energy(h, J, seqs) -> np.ndarray:
    h, J, L, q = _shape_hJ(h, J)
    S = _u8(seqs).reshape(-1, L)
    E = np.zeros(S.shape[0], dtype=np.float64)
    _load().orc_energy_batch(_p(h), _p(J), L, q, _p(S), S.shape[0], _p(E))
    return E


def fields(h, J, s, i: int) -> np.ndarray:
    h, J, L, q = _shape_hJ(h, J)
    s = _u8(s)
    H = np.zeros(q, dtype=np.float64)
    _load().orc_fields(_p(h), _p(J), L, q, _p(s), i, _p(H))
    return H


def draw(H, beta: float, u: float):
    """Inverse-CDF categorical draw; returns (symbol, margin)."""
    H = _f64(H)
    mg = np.zeros(1, dtype=np.float64)
    a = _load().orc_draw(_p(H), H.shape[0], beta, u, _p(mg))
    return int(a), float(mg[0])


def conditional(h, J, s, i: int, beta: float = 1.0) -> np.ndarray:
    h, J, L, q = _shape_hJ(h, J)
    s = _u8(s)
    P = np.zeros(q, dtype=np.float64)
    _load().orc_conditional(_p(h), _p(J), L, q, _p(s), i, beta, _p(P))
    return P


def gibbs(h, J, states, seed: int, sweep0: int, nsweeps: int, beta: float = 1.0,
          chain0: int = 0) -> np.ndarray:
    """Run nsweeps sequential Gibbs sweeps on a copy of states; returns it."""
    h, J, L, q = _shape_hJ(h, J)
    S = np.array(states, dtype=np.uint8, copy=True, order="C")
    M = S.shape[0]
    _load().orc_gibbs(_p(h), _p(J), L, q, M, _p(S), seed, chain0, sweep0, nsweeps, beta)
    return S


def gibbs_verify(h, J, before, after, seed: int, sweep: int, beta: float = 1.0, chain0: int = 0):
    """Teacher-forced check of one sweep; returns (n_bad, max_bad_margin, min_margin)."""
    h, J, L, q = _shape_hJ(h, J)
    b = _u8(before)
    a = _u8(after)
    M = b.shape[0]
    mx = np.zeros(1)
    mn = np.zeros(1)
    bad = _load().orc_gibbs_verify(_p(h), _p(J), L, q, M, _p(b), _p(a), seed, chain0, sweep, beta,
                                   _p(mx), _p(mn))
    return int(bad), float(mx[0]), float(mn[0])


def gibbs_flips(h, J, before, after, seed: int, sweep: int, beta: float = 1.0, chain0: int = 0,
                cap: int = 4096):
    """gibbs_verify with a record of every disagreement: returns
    (n_bad, min_margin, flips), flips = list of dicts with the chain (global
    index), site, oracle margin, symbol found and symbol the oracle draws
    (the first `cap` disagreements)."""
    h, J, L, q = _shape_hJ(h, J)
    b = _u8(before)
    a = _u8(after)
    M = b.shape[0]
    mx = np.zeros(1)
    mn = np.zeros(1)
    rc = np.zeros(cap, dtype=np.int64)
    rs = np.zeros(cap, dtype=np.int32)
    rm = np.zeros(cap, dtype=np.float64)
    rg = np.zeros(cap, dtype=np.int32)
    rw = np.zeros(cap, dtype=np.int32)
    bad = _load().orc_gibbs_verify_rec(_p(h), _p(J), L, q, M, _p(b), _p(a), seed, chain0, sweep, beta,
                                       _p(mx), _p(mn), cap, _p(rc), _p(rs), _p(rm), _p(rg), _p(rw))
    flips = [{"chain": int(rc[k]) + chain0, "site": int(rs[k]), "margin": float(rm[k]),
              "got": int(rg[k]), "want": int(rw[k])} for k in range(min(int(bad), cap))]
    return int(bad), float(mn[0]), flips


def metropolis(h, J, states, seed: int, sweep0: int, nsweeps: int, beta: float = 1.0,
               chain0: int = 0) -> np.ndarray:
    """Run nsweeps sequential Metropolis-Hastings sweeps on a copy of states."""
    h, J, L, q = _shape_hJ(h, J)
    S = np.array(states, dtype=np.uint8, copy=True, order="C")
    _load().orc_metropolis(_p(h), _p(J), L, q, S.shape[0], _p(S), seed, chain0, sweep0, nsweeps, beta)
    return S


def metropolis_flips(h, J, before, after, seed: int, sweep: int, beta: float = 1.0, chain0: int = 0,
                     cap: int = 4096):
    """Teacher-forced check of one Metropolis sweep: (n_bad, min_margin, flips)
    with the flips recorded as in gibbs_flips."""
    h, J, L, q = _shape_hJ(h, J)
    b = _u8(before)
    a = _u8(after)
    M = b.shape[0]
    mx = np.zeros(1)
    mn = np.zeros(1)
    rc = np.zeros(cap, dtype=np.int64)
    rs = np.zeros(cap, dtype=np.int32)
    rm = np.zeros(cap, dtype=np.float64)
    rg = np.zeros(cap, dtype=np.int32)
    rw = np.zeros(cap, dtype=np.int32)
    bad = _load().orc_metropolis_verify_rec(_p(h), _p(J), L, q, M, _p(b), _p(a), seed, chain0, sweep, beta,
                                            _p(mx), _p(mn), cap, _p(rc), _p(rs), _p(rm), _p(rg), _p(rw))
    flips = [{"chain": int(rc[k]) + chain0, "site": int(rs[k]), "margin": float(rm[k]),
              "got": int(rg[k]), "want": int(rw[k])} for k in range(min(int(bad), cap))]
    return int(bad), float(mn[0]), flips


# --- statistics ------------------------------------------------------------

def n_blocks(L: int) -> int:
    return L * (L + 1) // 2


def block_index(L: int, i: int, j: int) -> int:
    """Index of block (i, j), i <= j, in the upper-block-triangle count layout."""
    return i * L - i * (i - 1) // 2 + (j - i)


def chain_stats(states, q: int) -> np.ndarray:
    S = _u8(states)
    M, L = S.shape
    C = np.zeros((n_blocks(L), q, q), dtype=np.int32)
    _load().orc_chain_stats(_p(S), M, L, q, _p(C))
    return C


def identity_threshold(seqid: float, L: int) -> int:
    """Smallest integer identity count that is >= seqid * L (Eq. 7 reading)."""
    return int(math.ceil(seqid * L - 1e-9))


def seq_weights(msa, seqid: float = 0.8):
    X = _u8(msa)
    N, L = X.shape
    w = np.zeros(N, dtype=np.float64)
    meff = np.zeros(1, dtype=np.float64)
    _load().orc_seq_weights(_p(X), N, L, identity_threshold(seqid, L), _p(w), _p(meff))
    return w, float(meff[0])


def data_stats(msa, weights, q: int, pseudocount: float):
    X = _u8(msa)
    N, L = X.shape
    w = None if weights is None else _f64(weights)
    fi = np.zeros((L, q), dtype=np.float64)
    fij = np.zeros((L, L, q, q), dtype=np.float64)
    _load().orc_data_stats(_p(X), None if w is None else _p(w), N, L, q, pseudocount, _p(fi), _p(fij))
    return fi, fij


def pearson(fi, fij, counts, M: int) -> float:
    fi = _f64(fi)
    fij = _f64(fij)
    C = np.ascontiguousarray(counts, dtype=np.int32)
    L, q = fi.shape
    return float(_load().orc_pearson(_p(fi), _p(fij), _p(C), M, L, q))


def update(h, J, fi, fij, counts, M: int, lr: float):
    """Returns updated copies (h', J')."""
    h = np.array(h, dtype=np.float64, copy=True, order="C")
    J = np.array(J, dtype=np.float64, copy=True, order="C")
    fi = _f64(fi)
    fij = _f64(fij)
    C = np.ascontiguousarray(counts, dtype=np.int32)
    L, q = h.shape
    _load().orc_update(_p(h), _p(J), _p(fi), _p(fij), _p(C), M, lr, L, q)
    return h, J


def mutant_scan(h, J, wt) -> np.ndarray:
    h, J, L, q = _shape_hJ(h, J)
    wt = _u8(wt)
    dE = np.zeros((L, q), dtype=np.float64)
    _load().orc_mutant_scan(_p(h), _p(J), L, q, _p(wt), _p(dE))
    return dE


# ---------------------------------------------------------------- sparse graphs (Sec. 2.2)

def n_elements(L: int, q: int) -> int:
    """Coupling elements (i < j, a, b), numbered pair by pair in row order."""
    return L * (L - 1) // 2 * q * q


def pair_freqs(counts, M: int, L: int, q: int) -> np.ndarray:
    """Model pair frequencies p_ij(a,b) = count / M in the natural layout
    [i][j][a][b] (both halves), from the upper block-triangle counts."""
    C = np.asarray(counts, dtype=np.int64).reshape(-1, q, q)
    P = np.zeros((L, L, q, q))
    for i in range(L):
        for j in range(i, L):
            blk = C[i * L - i * (i - 1) // 2 + (j - i)] / M
            P[i, j] = blk
            P[j, i] = blk.T
    return P


def decimation_scores(J, pij, active) -> np.ndarray:
    """Symmetric KL of removing each element (+inf where inactive)."""
    J = _f64(J)
    pij = _f64(pij)
    active = _u8(active)
    L, _, q, _ = J.shape
    out = np.zeros(n_elements(L, q))
    _load().orc_decimation_scores(_p(J), _p(pij), _p(active), L, q, _p(out))
    return out


def activation_scores(fij, pij) -> np.ndarray:
    """Bernoulli KL between data and model pair frequencies of each element."""
    fij = _f64(fij)
    pij = _f64(pij)
    L, _, q, _ = fij.shape
    out = np.zeros(n_elements(L, q))
    _load().orc_activation_scores(_p(fij), _p(pij), L, q, _p(out))
    return out


def graph_decimate(J, active, score, n: int):
    """Returns copies (J', active', removed)."""
    J = np.array(J, dtype=np.float64, copy=True, order="C")
    active = np.array(active, dtype=np.uint8, copy=True, order="C")
    score = _f64(score)
    L, _, q, _ = J.shape
    removed = _load().orc_graph_decimate(_p(J), _p(active), _p(score), L, q, int(n))
    return J, active, int(removed)


def graph_activate(active, score, n: int):
    """Returns copies (active', newly_activated)."""
    active = np.array(active, dtype=np.uint8, copy=True, order="C")
    score = _f64(score)
    L, _, q, _ = active.shape
    fresh = _load().orc_graph_activate(_p(active), _p(score), L, q, int(n))
    return active, int(fresh)


def update_masked(h, J, fi, fij, counts, M: int, lr: float, active):
    """Eq. 5 on a sparse graph; returns updated copies (h', J')."""
    h = np.array(h, dtype=np.float64, copy=True, order="C")
    J = np.array(J, dtype=np.float64, copy=True, order="C")
    fi = _f64(fi)
    fij = _f64(fij)
    C = np.ascontiguousarray(counts, dtype=np.int32)
    active = _u8(active)
    L, q = h.shape
    _load().orc_update_masked(_p(h), _p(J), _p(fi), _p(fij), _p(C), M, lr, L, q, _p(active))
    return h, J
