"""Boundary-flip log of the GPU parity tests.

A GPU draw may differ from the oracle's only when the oracle's uniform lies
within FLIP_MARGIN of a CDF boundary (FP32 against FP64 fields).  Every such
flip found by a teacher-forced check is recorded here with its test, chain,
site and margin; conftest prints the whole record at the end of the run, so
a passing run still shows each flip and how close to the boundary it was.
"""
import numpy as np

FLIP_MARGIN = 1e-5
FLIPS = []      # dicts: where, chain, site, sweep, margin, got, want
CHECKED = [0]   # site-updates verified


def verify(orc, h, J, before, after, seed, sweep, beta=1.0, chain0=0, where="", metropolis=False):
    """Teacher-forced check of one sweep (Gibbs, or Metropolis-Hastings);
    records each disagreement and returns (n_bad, worst_margin)."""
    check = orc.metropolis_flips if metropolis else orc.gibbs_flips
    bad, _, flips = check(np.asarray(h, np.float64), np.asarray(J, np.float64), before, after,
                          seed, sweep, beta, chain0)
    CHECKED[0] += int(np.asarray(before).size)
    worst = 0.0
    for f in flips:
        f = dict(f, where=where, sweep=sweep)
        FLIPS.append(f)
        worst = max(worst, f["margin"])
    return bad, worst


def summary_lines():
    out = [f"teacher-forced site-updates checked: {CHECKED[0]}; boundary flips: {len(FLIPS)}"]
    for f in FLIPS:
        out.append(f"  flip {f['where']}: chain {f['chain']} site {f['site']} sweep {f['sweep']} "
                   f"margin {f['margin']:.3e} gpu {f['got']} oracle {f['want']}")
    if FLIPS:
        out.append(f"  worst flip margin {max(f['margin'] for f in FLIPS):.3e} (bound {FLIP_MARGIN:g})")
    return out
