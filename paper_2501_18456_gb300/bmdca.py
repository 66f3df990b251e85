"""Thin ctypes binding of libbmdca.so (include/bmdca.h).

Argument marshalling only: every function forwards to the C entry point of
the same name; torch tensors supply memory (host or device) and the current
CUDA stream.  Every computation happens in the library's CUDA kernels; there
is no Python or CPU fallback.  If the library is missing the first call
raises RuntimeError.
"""
from __future__ import annotations

import ctypes
import math
from pathlib import Path

import torch

_LIB_PATH = Path(__file__).resolve().parent / "_build" / "libbmdca.so"
_lib = None

BM_OK, BM_EINVAL, BM_ENOMEM, BM_ECUDA, BM_ENUMERIC, BM_ETIMEOUT, BM_EDEVICE, BM_EBUSY = (
    0, -1, -2, -3, -4, -5, -6, -7)
BM_HOST, BM_DEVICE = 0, 1
BM_ENGINE_SIMT, BM_ENGINE_AUTO, BM_ENGINE_MMA, BM_ENGINE_MMA_PAIR, BM_ENGINE_MMA_PAIR2 = 0, 1, 2, 3, 4
BM_SAMPLER_GIBBS, BM_SAMPLER_METROPOLIS = 0, 1
BM_STATS_AUTO, BM_STATS_SIMT, BM_STATS_MMA_BF16, BM_STATS_MMA_FP8 = 0, 1, 2, 3
BM_FIELDS_FP32, BM_FIELDS_FP16X2, BM_FIELDS_BF16X2 = 0, 1, 2
BM_REQ_SAMPLE, BM_REQ_SCORE, BM_REQ_SCAN = 1, 2, 3


class Request(ctypes.Structure):
    """bm_request (include/bmdca.h)."""
    _fields_ = [("type", ctypes.c_int), ("model", ctypes.c_int), ("n", ctypes.c_int), ("nsweeps", ctypes.c_int),
                ("beta", ctypes.c_float), ("seed", ctypes.c_uint64), ("in_", ctypes.c_void_p),
                ("out", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    """bm_server_stats (include/bmdca.h)."""
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("sequences", ctypes.c_double), ("span_s", ctypes.c_double), ("max_running", ctypes.c_int)]

# name -> (restype, argtypes); kept in the order of include/bmdca.h
_P, _I, _U64, _F, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_float, ctypes.c_double
SIGNATURES = {
    "bm_version": (ctypes.c_char_p, []),
    "bm_last_error": (ctypes.c_char_p, []),
    "bm_potts_load": (_I, [_P, _P, _I, _I, _I, _P, _P]),
    "bm_potts_free": (_I, [_P]),
    "bm_potts_get": (_I, [_P, _P, _P, _I, _P]),
    "bm_potts_set": (_I, [_P, _P, _P, _I, _P]),
    "bm_device_status": (_I, [_P, _P]),
    "bm_potts_shape": (_I, [_P, _P, _P]),
    "bm_chains_init": (_I, [_P, _I, _U64, _P, _I, _P, _P]),
    "bm_chains_init_shard": (_I, [_P, _I, _U64, _U64, _P, _P]),
    "bm_chains_free": (_I, [_P]),
    "bm_chains_get": (_I, [_P, _P, _I, _P]),
    "bm_chains_set": (_I, [_P, _P, _I, _P]),
    "bm_chains_sweep_counter": (_I, [_P, _P]),
    "bm_chains_set_sweep_counter": (_I, [_P, _U64]),
    "bm_chains_shape": (_I, [_P, _P, _P]),
    "bm_gibbs_sweep": (_I, [_P, _P, _I, _F, _P]),
    "bm_model_set_engine": (_I, [_P, _I]),
    "bm_model_set_sampler": (_I, [_P, _I]),
    "bm_model_sweep_engine": (_I, [_P, _I, _P]),
    "bm_chains_set_stats_engine": (_I, [_P, _I]),
    "bm_chains_device_status": (_I, [_P, _P]),
    "bm_chain_stats": (_I, [_P, _P, _P]),
    "bm_seq_weights": (_I, [_P, _I, _I, _D, _P, _P, _P]),
    "bm_seq_weights_static": (_I, [_P, _I, _I, _D, _P, _P, _P]),
    "bm_data_stats": (_I, [_P, _P, _I, _I, _I, _D, _P, _P, _P]),
    "bm_update": (_I, [_P, _P, _P, _P, _I, _F, _D, _P, _P, _P]),
    "bm_graph_enable": (_I, [_P, _I, _P]),
    "bm_graph_disable": (_I, [_P]),
    "bm_graph_count": (_I, [_P, _P, _P]),
    "bm_graph_get": (_I, [_P, _P, _I, _P]),
    "bm_graph_decimate": (_I, [_P, _P, _I, ctypes.c_longlong, _P, _P]),
    "bm_graph_activate": (_I, [_P, _P, _P, _I, ctypes.c_longlong, _P, _P]),
    "bm_energy_score": (_I, [_P, _P, _I, _P, _P]),
    "bm_mutant_scan": (_I, [_P, _P, _I, _P, _P]),
    "bm_fields": (_I, [_P, _P, _I, _P, _I, _P]),
    "bm_batch_create": (_I, [_P, _P, _I, _P]),
    "bm_batch_free": (_I, [_P]),
    "bm_batch_autotune": (_I, [_P, _P]),
    "bm_batch_sweep": (_I, [_P, _I, _F, _P]),
    "bm_batch_shape": (_I, [_P, _P, _P, _P]),
    "bm_server_create": (_I, [ctypes.c_size_t, _I, _P]),
    "bm_server_destroy": (_I, [_P]),
    "bm_server_add_model": (_I, [_P, _P, _P]),
    "bm_server_submit": (_I, [_P, _P, _P]),
    "bm_server_wait": (_I, [_P, _U64, _D, _P, _P]),
    "bm_server_stats_get": (_I, [_P, _P, _I]),
}


class BmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def library_path() -> Path:
    return _LIB_PATH


def lib():
    """Load libbmdca.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise RuntimeError(f"libbmdca.so not found at {_LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(str(_LIB_PATH))
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, name: str):
    if rc != BM_OK:
        raise BmError(rc, f"{name}: {lib().bm_last_error().decode()}")


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t: torch.Tensor | None, dtype: torch.dtype | None = None, numel: int | None = None,
         name: str = "tensor"):
    """(pointer, where) for a contiguous tensor; validates dtype and size."""
    if t is None:
        return None, BM_HOST
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr()), (BM_DEVICE if t.is_cuda else BM_HOST)


def _dev(t: torch.Tensor, dtype, numel, name):
    p, where = _ptr(t, dtype, numel, name)
    if where != BM_DEVICE:
        raise ValueError(f"{name}: must be a CUDA tensor")
    return p


def n_blocks(L: int) -> int:
    return L * (L + 1) // 2


def bm_version() -> str:
    return lib().bm_version().decode()


class Model:
    """Owning wrapper of a bm_model handle."""

    def __init__(self, handle: ctypes.c_void_p, L: int, q: int):
        self.handle, self.L, self.q = handle, L, q

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bm_potts_free(self.handle)
        self.handle = None


class Chains:
    """Owning wrapper of a bm_chains handle."""

    def __init__(self, handle: ctypes.c_void_p, M: int, L: int, q: int):
        self.handle, self.M, self.L, self.q = handle, M, L, q

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bm_chains_free(self.handle)
        self.handle = None


def bm_potts_load(h: torch.Tensor, J: torch.Tensor, stream=None) -> Model:
    L, q = h.shape
    ph, wh = _ptr(h, torch.float32, L * q, "h")
    pJ, wJ = _ptr(J, torch.float32, L * L * q * q, "J")
    if wh != wJ:
        raise ValueError("h and J must both be host or both be device tensors")
    out = ctypes.c_void_p()
    _check(lib().bm_potts_load(ph, pJ, L, q, wh, _stream(stream), ctypes.byref(out)), "bm_potts_load")
    return Model(out, L, q)


def bm_potts_free(m: Model):
    m.free()


def bm_potts_get(m: Model, h: torch.Tensor | None = None, J: torch.Tensor | None = None,
                 stream=None):
    ph, wh = _ptr(h, torch.float32, m.L * m.q, "h")
    pJ, wJ = _ptr(J, torch.float32, m.L * m.L * m.q * m.q, "J")
    if h is not None and J is not None and wh != wJ:
        raise ValueError("h and J must both be host or both be device tensors")
    where = wh if h is not None else wJ
    _check(lib().bm_potts_get(m.handle, ph, pJ, where, _stream(stream)), "bm_potts_get")


def bm_potts_set(m: Model, h: torch.Tensor | None = None, J: torch.Tensor | None = None,
                 stream=None):
    ph, wh = _ptr(h, torch.float32, m.L * m.q, "h")
    pJ, wJ = _ptr(J, torch.float32, m.L * m.L * m.q * m.q, "J")
    if h is not None and J is not None and wh != wJ:
        raise ValueError("h and J must both be host or both be device tensors")
    where = wh if h is not None else wJ
    _check(lib().bm_potts_set(m.handle, ph, pJ, where, _stream(stream)), "bm_potts_set")


def bm_device_status(m: Model, stream=None):
    _check(lib().bm_device_status(m.handle, _stream(stream)), "bm_device_status")


def bm_model_set_engine(m: Model, engine: int):
    _check(lib().bm_model_set_engine(m.handle, engine), "bm_model_set_engine")


def bm_model_set_sampler(m: Model, sampler: int):
    _check(lib().bm_model_set_sampler(m.handle, sampler), "bm_model_set_sampler")


def bm_model_sweep_engine(m: Model, M: int) -> int:
    """The kernel form bm_gibbs_sweep runs for M chains (AUTO resolved)."""
    out = ctypes.c_int(0)
    _check(lib().bm_model_sweep_engine(m.handle, M, ctypes.byref(out)), "bm_model_sweep_engine")
    return out.value


def bm_chains_init(m: Model, M: int, seed: int, init: torch.Tensor | None = None,
                   stream=None) -> Chains:
    p, where = _ptr(init, torch.uint8, M * m.L, "init")
    out = ctypes.c_void_p()
    _check(lib().bm_chains_init(m.handle, M, seed, p, where, _stream(stream), ctypes.byref(out)),
           "bm_chains_init")
    return Chains(out, M, m.L, m.q)


def bm_chains_init_shard(m: Model, M: int, seed: int, chain0: int, stream=None) -> Chains:
    out = ctypes.c_void_p()
    _check(lib().bm_chains_init_shard(m.handle, M, seed, chain0, _stream(stream), ctypes.byref(out)),
           "bm_chains_init_shard")
    return Chains(out, M, m.L, m.q)


def bm_chains_free(c: Chains):
    c.free()


def bm_chains_get(c: Chains, dst: torch.Tensor, stream=None):
    p, where = _ptr(dst, torch.uint8, c.M * c.L, "dst")
    _check(lib().bm_chains_get(c.handle, p, where, _stream(stream)), "bm_chains_get")


def bm_chains_set(c: Chains, src: torch.Tensor, stream=None):
    p, where = _ptr(src, torch.uint8, c.M * c.L, "src")
    _check(lib().bm_chains_set(c.handle, p, where, _stream(stream)), "bm_chains_set")


def bm_chains_sweep_counter(c: Chains) -> int:
    v = ctypes.c_uint64()
    _check(lib().bm_chains_sweep_counter(c.handle, ctypes.byref(v)), "bm_chains_sweep_counter")
    return int(v.value)


def bm_chains_set_sweep_counter(c: Chains, sweep: int):
    _check(lib().bm_chains_set_sweep_counter(c.handle, sweep), "bm_chains_set_sweep_counter")


def bm_gibbs_sweep(m: Model, c: Chains, nsweeps: int, beta: float = 1.0, stream=None):
    _check(lib().bm_gibbs_sweep(m.handle, c.handle, nsweeps, beta, _stream(stream)), "bm_gibbs_sweep")


def bm_chains_set_stats_engine(c: Chains, engine: int):
    _check(lib().bm_chains_set_stats_engine(c.handle, engine), "bm_chains_set_stats_engine")


def bm_chains_device_status(c: Chains, stream=None):
    _check(lib().bm_chains_device_status(c.handle, _stream(stream)), "bm_chains_device_status")


def bm_chain_stats(c: Chains, counts: torch.Tensor, stream=None):
    p = _dev(counts, torch.int32, n_blocks(c.L) * c.q * c.q, "counts")
    _check(lib().bm_chain_stats(c.handle, p, _stream(stream)), "bm_chain_stats")


def bm_seq_weights(msa: torch.Tensor, w: torch.Tensor, seqid: float = 0.8, want_meff: bool = True,
                   stream=None):
    N, L = msa.shape
    pm = _dev(msa, torch.uint8, N * L, "msa")
    pw = _dev(w, torch.float32, N, "w")
    meff = ctypes.c_double()
    _check(lib().bm_seq_weights(pm, N, L, seqid, pw, ctypes.byref(meff) if want_meff else None,
                                _stream(stream)), "bm_seq_weights")
    return float(meff.value) if want_meff else None


def bm_seq_weights_static(msa: torch.Tensor, w: torch.Tensor, seqid: float = 0.8,
                          want_meff: bool = True, stream=None):
    """bm_seq_weights without device allocation (fixed static scratch; see bmdca.h)."""
    N, L = msa.shape
    pm = _dev(msa, torch.uint8, N * L, "msa")
    pw = _dev(w, torch.float32, N, "w")
    meff = ctypes.c_double()
    _check(lib().bm_seq_weights_static(pm, N, L, seqid, pw,
                                       ctypes.byref(meff) if want_meff else None, _stream(stream)),
           "bm_seq_weights_static")
    return float(meff.value) if want_meff else None


def bm_data_stats(msa: torch.Tensor, w: torch.Tensor | None, q: int, pseudocount: float,
                  fi: torch.Tensor, fij: torch.Tensor, stream=None):
    N, L = msa.shape
    pm = _dev(msa, torch.uint8, N * L, "msa")
    pw = None if w is None else _dev(w, torch.float32, N, "w")
    pfi = _dev(fi, torch.float32, L * q, "fi")
    pfij = _dev(fij, torch.float32, L * L * q * q, "fij")
    _check(lib().bm_data_stats(pm, pw, N, L, q, pseudocount, pfi, pfij, _stream(stream)),
           "bm_data_stats")


def bm_update(m: Model, fi: torch.Tensor, fij: torch.Tensor, counts: torch.Tensor, M: int,
              lr: float, target: float = math.inf, want_pearson: bool = True, stream=None):
    """Returns (pearson or None, applied)."""
    pfi = _dev(fi, torch.float32, m.L * m.q, "fi")
    pfij = _dev(fij, torch.float32, m.L * m.L * m.q * m.q, "fij")
    pc = _dev(counts, torch.int32, n_blocks(m.L) * m.q * m.q, "counts")
    rho = ctypes.c_double()
    applied = ctypes.c_int()
    _check(lib().bm_update(m.handle, pfi, pfij, pc, M, lr, target,
                           ctypes.byref(rho) if want_pearson else None, ctypes.byref(applied),
                           _stream(stream)), "bm_update")
    return (float(rho.value) if want_pearson else None), bool(applied.value)


# ---------------------------------------------------------------- sparse graphs (Sec. 2.2)

def bm_graph_enable(m: Model, dense: bool = True, stream=None):
    """Create the model's coupling graph: all elements active (dense) or none."""
    _check(lib().bm_graph_enable(m.handle, 1 if dense else 0, _stream(stream)), "bm_graph_enable")


def bm_graph_disable(m: Model):
    _check(lib().bm_graph_disable(m.handle), "bm_graph_disable")


def bm_graph_count(m: Model) -> tuple[int, int]:
    """(active elements, all elements i < j, a, b)."""
    na, ne = ctypes.c_longlong(0), ctypes.c_longlong(0)
    _check(lib().bm_graph_count(m.handle, ctypes.byref(na), ctypes.byref(ne)), "bm_graph_count")
    return na.value, ne.value


def bm_graph_get(m: Model, active: torch.Tensor, stream=None):
    """Copy the activity bytes [L][L][q][q] into a uint8 tensor."""
    p, where = _ptr(active, torch.uint8, m.L * m.L * m.q * m.q, "active")
    _check(lib().bm_graph_get(m.handle, p, where, _stream(stream)), "bm_graph_get")


def bm_graph_decimate(m: Model, counts: torch.Tensor, M: int, n: int, stream=None) -> int:
    """edDCA step: remove the n active elements of smallest symmetric KL; returns the count removed."""
    pc = _dev(counts, torch.int32, n_blocks(m.L) * m.q * m.q, "counts")
    out = ctypes.c_longlong(0)
    _check(lib().bm_graph_decimate(m.handle, pc, M, int(n), ctypes.byref(out), _stream(stream)), "bm_graph_decimate")
    return out.value


def bm_graph_activate(m: Model, fij: torch.Tensor, counts: torch.Tensor, M: int, n: int, stream=None) -> int:
    """eaDCA step: make the n elements of largest data/model divergence active; returns the count newly active."""
    pf = _dev(fij, torch.float32, m.L * m.L * m.q * m.q, "fij")
    pc = _dev(counts, torch.int32, n_blocks(m.L) * m.q * m.q, "counts")
    out = ctypes.c_longlong(0)
    _check(lib().bm_graph_activate(m.handle, pf, pc, M, int(n), ctypes.byref(out), _stream(stream)), "bm_graph_activate")
    return out.value


def bm_energy_score(m: Model, seqs: torch.Tensor, E: torch.Tensor, stream=None):
    n = seqs.shape[0] if seqs.dim() == 2 else 0
    ps = _dev(seqs, torch.uint8, n * m.L, "seqs")
    pe = _dev(E, torch.float32, n, "E")
    _check(lib().bm_energy_score(m.handle, ps, n, pe, _stream(stream)), "bm_energy_score")


def bm_mutant_scan(m: Model, wt: torch.Tensor, dE: torch.Tensor, stream=None):
    pw, where = _ptr(wt, torch.uint8, m.L, "wt")
    pd = _dev(dE, torch.float32, m.L * m.q, "dE")
    _check(lib().bm_mutant_scan(m.handle, pw, where, pd, _stream(stream)), "bm_mutant_scan")


def bm_fields(m: Model, seqs: torch.Tensor, H: torch.Tensor, form: int = BM_FIELDS_FP32, stream=None):
    n = seqs.shape[0] if seqs.dim() == 2 else 0
    ps = _dev(seqs, torch.uint8, n * m.L, "seqs")
    ph = _dev(H, torch.float32, n * m.L * m.q, "H")
    _check(lib().bm_fields(m.handle, ps, n, ph, form, _stream(stream)), "bm_fields")


class Server:
    """Owner of a bm_server handle (continuous-batching request server).

    Keeps the models it serves (and the tensors of queued requests) alive
    until the server is closed or the request is waited for."""

    def __init__(self, budget_bytes: int, slots: int = 16):
        h = ctypes.c_void_p()
        _check(lib().bm_server_create(int(budget_bytes), int(slots), ctypes.byref(h)), "bm_server_create")
        self.handle = h.value
        self._models = []
        self._pending = {}

    def close(self):
        if self.handle:
            lib().bm_server_destroy(self.handle)
            self.handle = None
            self._pending.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_model(self, m: Model) -> int:
        i = ctypes.c_int()
        _check(lib().bm_server_add_model(self.handle, m.handle, ctypes.byref(i)), "bm_server_add_model")
        self._models.append(m)
        return i.value

    def submit(self, req_type: int, model: int, out: torch.Tensor, inp: torch.Tensor | None = None, n: int = 0,
               nsweeps: int = 0, beta: float = 1.0, seed: int = 0) -> int:
        """Queue a request; `out` (and `inp`) are contiguous host (pinned for overlap) or device tensors."""
        for t in (out, inp):
            if t is not None and not t.is_contiguous():
                raise ValueError("request tensors must be contiguous")
        r = Request(int(req_type), int(model), int(n), int(nsweeps), float(beta), int(seed),
                    inp.data_ptr() if inp is not None else None, out.data_ptr())
        rid = ctypes.c_uint64()
        _check(lib().bm_server_submit(self.handle, ctypes.byref(r), ctypes.byref(rid)), "bm_server_submit")
        self._pending[rid.value] = (out, inp)
        return rid.value

    def wait(self, rid: int, timeout_ms: float = -1.0):
        """Block until request rid completes; returns (status, latency_ms)."""
        st = ctypes.c_int()
        lat = ctypes.c_double()
        _check(lib().bm_server_wait(self.handle, int(rid), float(timeout_ms), ctypes.byref(st), ctypes.byref(lat)),
               "bm_server_wait")
        self._pending.pop(rid, None)
        return st.value, lat.value

    def stats(self, reset: bool = False) -> dict:
        out = ServerStats()
        _check(lib().bm_server_stats_get(self.handle, ctypes.byref(out), 1 if reset else 0), "bm_server_stats_get")
        return {k: getattr(out, k) for k, _ in ServerStats._fields_}


class Batch:
    """Owner of a bm_batch handle: CUDA-core sweeps of many (model, chains)
    pairs with the same q in one graph launch.  Keeps the handles alive."""

    def __init__(self, models, chains):
        if len(models) != len(chains):
            raise ValueError("one chains handle per model")
        arr_m = (ctypes.c_void_p * len(models))(*[m.handle for m in models])
        arr_c = (ctypes.c_void_p * len(chains))(*[c.handle for c in chains])
        h = ctypes.c_void_p()
        _check(lib().bm_batch_create(arr_m, arr_c, len(models), ctypes.byref(h)), "bm_batch_create")
        self.handle = h.value
        self._keep = (list(models), list(chains))

    def close(self):
        if self.handle:
            lib().bm_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, stream=None):
        _check(lib().bm_batch_autotune(self.handle, _stream(stream)), "bm_batch_autotune")

    def sweep(self, nsweeps: int, beta: float = 1.0, stream=None):
        _check(lib().bm_batch_sweep(self.handle, int(nsweeps), float(beta), _stream(stream)), "bm_batch_sweep")

    def shape(self) -> dict:
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().bm_batch_shape(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "bm_batch_shape")
        return {"chains_per_cta": a.value, "stages": b.value, "ctas": c.value}
