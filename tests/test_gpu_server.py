"""GPU tests of the continuous-batching server (bm_server_*): every result is
identical alone, in a mixed burst and through the direct entry points, and
agrees with the FP64 oracle (Sec. 4.1 sampling, Sec. 4.3 scoring, Sec. 4.4
single-mutant scans); work overlaps on the device; admission respects the
scratch budget."""
import numpy as np
import pytest
import torch

import fliplog
from paper_2501_18456_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def pinned(shape, dtype):
    return torch.empty(shape, dtype=dtype).pin_memory()


PARAMS = {}  # model handle id -> (h, J) as loaded


@pytest.fixture
def models(bm):
    out = []
    for k, (L, q) in enumerate([(40, 21), (30, 5), (64, 21)]):
        h, J = synth.planted_local_model(L, q, 30 + k, sigma_h=1.0, sigma_J=0.3)
        m = bm.bm_potts_load(to_dev(h), to_dev(J))
        PARAMS[id(m)] = (h, J)
        out.append(m)
    return out


def oracle_checks(orc, models, outs, seqs, wt):
    """Served results against the oracle:
    * the one-sweep sample: its chains start from the oracle's chains_init
      for the request's seed, and every site-update of the sweep equals the
      oracle's teacher-forced draw (boundary flips logged, margin < 1e-5);
    * the scores: oracle energies, with the tolerance of the energy parity test;
    * the scan: oracle single-mutant dE, with the mutant-scan parity tolerance."""
    mA, mB, mC = models
    out_1 = outs[3].numpy()
    hA, JA = PARAMS[id(mA)]
    s0 = orc.chains_init(out_1.shape[0], mA.L, mA.q, 6)
    bad, worst = fliplog.verify(orc, hA, JA, s0, out_1, 6, 0, 0.8, 0, "served sample")
    assert bad == 0 or worst < fliplog.FLIP_MARGIN, (bad, worst)
    assert bad <= max(2, s0.size // 10000)
    hB, JB = PARAMS[id(mB)]
    E_o = orc.energy(hB.astype(np.float64), JB.astype(np.float64), seqs)
    scale = np.abs(hB).max() * mB.L + np.abs(JB).max() * mB.L * mB.L / 2
    assert np.abs(outs[1].numpy() - E_o).max() < 2e-5 * scale + 1e-6
    hC, JC = PARAMS[id(mC)]
    want = orc.mutant_scan(hC.astype(np.float64), JC.astype(np.float64), wt)
    got = outs[2].numpy()
    assert np.all(got[np.arange(mC.L), wt] == 0.0)
    assert np.abs(got - want).max() < 1e-5 * (1 + np.abs(want).max())


def direct_sample(bm, m, n, nsweeps, beta, seed):
    c = bm.bm_chains_init(m, n, seed)
    bm.bm_gibbs_sweep(m, c, nsweeps, beta)
    out = torch.empty((n, m.L), dtype=torch.uint8, device=DEV)
    bm.bm_chains_get(c, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def direct_score(bm, m, seqs):
    E = torch.empty(seqs.shape[0], dtype=torch.float32, device=DEV)
    bm.bm_energy_score(m, to_dev(seqs), E)
    torch.cuda.synchronize()
    return E.cpu().numpy()


def direct_scan(bm, m, wt):
    dE = torch.empty((m.L, m.q), dtype=torch.float32, device=DEV)
    bm.bm_mutant_scan(m, torch.from_numpy(wt), dE)
    torch.cuda.synchronize()
    return dE.cpu().numpy()


def submit_probe_requests(bm, srv, ids, models, seqs, wt):
    """The four requests whose results are checked; returns their output tensors."""
    mA, mB, mC = models
    out_s = pinned((300, mA.L), torch.uint8)
    out_e = pinned((seqs.shape[0],), torch.float32)
    out_d = pinned((mC.L, mC.q), torch.float32)
    out_1 = pinned((500, mA.L), torch.uint8)
    in_e = torch.from_numpy(seqs).pin_memory()
    in_d = torch.from_numpy(wt).pin_memory()
    r = [srv.submit(bm.BM_REQ_SAMPLE, ids[0], out_s, n=300, nsweeps=7, beta=1.2, seed=5),
         srv.submit(bm.BM_REQ_SCORE, ids[1], out_e, inp=in_e, n=seqs.shape[0]),
         srv.submit(bm.BM_REQ_SCAN, ids[2], out_d, inp=in_d),
         srv.submit(bm.BM_REQ_SAMPLE, ids[0], out_1, n=500, nsweeps=1, beta=0.8, seed=6)]
    return r, (out_s, out_e, out_d, out_1)


def test_results_alone_in_mix_and_direct_agree(bm, orc, models):
    mA, mB, mC = models
    seqs = synth.random_states(2000, mB.L, mB.q, 7)
    wt = synth.random_states(1, mC.L, mC.q, 8)[0]
    ref = (direct_sample(bm, mA, 300, 7, 1.2, 5), direct_score(bm, mB, seqs), direct_scan(bm, mC, wt),
           direct_sample(bm, mA, 500, 1, 0.8, 6))

    srv = bm.Server(budget_bytes=1 << 30, slots=16)
    ids = [srv.add_model(m) for m in models]
    # alone
    rids, outs = submit_probe_requests(bm, srv, ids, models, seqs, wt)
    for rid in rids:
        assert srv.wait(rid)[0] == bm.BM_OK
    alone = [o.numpy().copy() for o in outs]
    oracle_checks(orc, models, outs, seqs, wt)
    # in a burst of other requests of every kind
    rng = np.random.default_rng(3)
    extra = []
    for k in range(40):
        mi = int(rng.integers(3))
        m = models[mi]
        kind = int(rng.integers(1, 4))
        if kind == bm.BM_REQ_SAMPLE:
            n = int(rng.integers(50, 800))
            o = pinned((n, m.L), torch.uint8)
            extra.append(srv.submit(kind, ids[mi], o, n=n, nsweeps=int(rng.integers(1, 12)),
                                    beta=float(rng.choice([0.8, 1.0, 1.2])), seed=1000 + k))
        elif kind == bm.BM_REQ_SCORE:
            n = int(rng.integers(100, 5000))
            i = torch.from_numpy(synth.random_states(n, m.L, m.q, 100 + k)).pin_memory()
            extra.append(srv.submit(kind, ids[mi], pinned((n,), torch.float32), inp=i, n=n))
        else:
            i = torch.from_numpy(synth.random_states(1, m.L, m.q, 200 + k)[0]).pin_memory()
            extra.append(srv.submit(kind, ids[mi], pinned((m.L, m.q), torch.float32), inp=i))
        if k == 20:
            rids, outs = submit_probe_requests(bm, srv, ids, models, seqs, wt)
    for rid in extra + rids:
        assert srv.wait(rid)[0] == bm.BM_OK
    mixed = [o.numpy() for o in outs]
    oracle_checks(orc, models, outs, seqs, wt)
    for a, b, r in zip(alone, mixed, ref):
        assert np.array_equal(a, r)
        assert np.array_equal(b, r)
    st = srv.stats()
    assert st["completed"] == 48 and st["failed"] == 0
    assert st["max_running"] > 1, "requests never overlapped on the device"
    assert st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_admission_respects_budget(bm, models):
    mA = models[0]
    n = 1000
    need = ((n * mA.L + 255) // 256) * 256
    srv = bm.Server(budget_bytes=need + need // 2, slots=8)  # room for one request at a time
    i = srv.add_model(mA)
    outs = [pinned((n, mA.L), torch.uint8) for _ in range(6)]
    rids = [srv.submit(bm.BM_REQ_SAMPLE, i, o, n=n, nsweeps=3, seed=k) for k, o in enumerate(outs)]
    for rid in rids:
        assert srv.wait(rid)[0] == bm.BM_OK
    st = srv.stats()
    assert st["completed"] == 6 and st["max_running"] == 1
    for k, o in enumerate(outs):
        assert np.array_equal(o.numpy(), direct_sample(bm, mA, n, 3, 1.0, k))
    srv.close()


def test_rejects_bad_requests(bm, models):
    srv = bm.Server(budget_bytes=4096, slots=2)
    i = srv.add_model(models[0])
    with pytest.raises(bm.BmError) as e:  # scratch above the budget
        srv.submit(bm.BM_REQ_SAMPLE, i, pinned((1000, models[0].L), torch.uint8), n=1000, nsweeps=1)
    assert e.value.code == bm.BM_ENOMEM
    with pytest.raises(bm.BmError) as e:  # unknown model
        srv.submit(bm.BM_REQ_SAMPLE, 5, pinned((1, 40), torch.uint8), n=1, nsweeps=1)
    assert e.value.code == bm.BM_EINVAL
    with pytest.raises(bm.BmError) as e:  # unknown request id
        srv.wait(12345)
    assert e.value.code == bm.BM_EINVAL
    srv.close()
