"""Thin PyTorch adapter over the C ABI: device memory and streams come from
torch, every step of the descent runs in the CUDA library.

    import paper_2202_00517_gb300 as knnd
    g = knnd.Handle(n, m, K, dtype="f32", precision="mixed")
    out = g.build(points_cuda, seed=1)        # dict: idx, key, rounds, updates, fcc_hits, ...
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import check

_PREC = {"fp64": _lib.KNND_PREC_FP64, "mixed": _lib.KNND_PREC_MIXED_FP32,
         "mixed_fp32": _lib.KNND_PREC_MIXED_FP32, "bf16x3": _lib.KNND_PREC_MIXED_BF16X3,
         "auto": _lib.KNND_PREC_AUTO}
_CMP = {"kl": _lib.KNND_CMP_KL, "kl_reverse": _lib.KNND_CMP_KL_REVERSE, "sqeuclidean": _lib.KNND_CMP_SQEUCLIDEAN,
        "inner": _lib.KNND_CMP_INNER}
_LOOP = {"auto": _lib.KNND_LOOP_AUTO, "host": _lib.KNND_LOOP_HOST, "graph": _lib.KNND_LOOP_GRAPH}
_JOIN = {"auto": 0, "tma": _lib.KNND_JOIN_TMA, "plain": _lib.KNND_JOIN_PLAIN}
_JOIN_NAMES = {_lib.KNND_JOIN_TMA: "tma", _lib.KNND_JOIN_PLAIN: "plain", _lib.KNND_JOIN_FP64: "fp64",
               _lib.KNND_JOIN_TC: "tc"}
_DTYPE = {"f32": _lib.KNND_F32, "f64": _lib.KNND_F64, torch.float32: _lib.KNND_F32,
          torch.float64: _lib.KNND_F64}


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _require(ok: bool, msg: str):
    """Argument checks that hold under python -O too (unlike assert)."""
    if not ok:
        raise ValueError(msg)


def _info_dict(info: _lib.knnd_build_info) -> dict:
    r = info.rounds
    return {"rounds": r, "stop_reason": info.stop_reason,
            "updates": [info.updates[i] for i in range(r)],
            "fcc_hits": [info.fcc_hits[i] for i in range(r + 1)],
            "proposals": info.proposals, "init_pairs": info.init_pairs,
            "rescored": info.rescored, "bound_violations": info.bound_violations,
            "merge_fallbacks": info.merge_fallbacks, "join_survivors": info.join_survivors,
            "bound_audited": info.bound_audited, "join_kernel": _JOIN_NAMES.get(info.join_kernel, "none")}


class Handle:
    """One problem shape (n points, m coordinates, K friends) on one device."""

    def __init__(self, n: int, m: int, K: int, dtype="f32", precision="mixed", fcc_samples: int = 10000,
                 max_rounds: int = 64, stop_on_zero_updates: bool = True, debug: bool = False,
                 timing: bool = False, incremental: bool = False, stop_delta: float = 0.0, comparator: str = "kl",
                 loop: str = "auto", stream=None, split_den: int = 0, merge_keep: int = 0, join_blocks: int = 0,
                 join_form: str = "auto"):
        lib = _lib.load()
        self.n, self.m, self.K = n, m, K
        self.dtype = _DTYPE[dtype]
        self.torch_dtype = torch.float32 if self.dtype == _lib.KNND_F32 else torch.float64
        prm = _lib.knnd_params(fcc_samples, max_rounds, int(stop_on_zero_updates), int(debug), int(timing),
                               int(incremental), float(stop_delta), _CMP[comparator], _LOOP[loop], int(split_den),
                               int(merge_keep), int(join_blocks), _JOIN[join_form])
        h = ctypes.c_void_p()
        check(lib.knnd_create(ctypes.byref(h), n, m, K, self.dtype, _PREC[precision], ctypes.byref(prm),
                              _stream_ptr(stream)), "knnd_create")
        self._h = h
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.knnd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        check(self._lib.knnd_set_stream(self._h, _stream_ptr(stream)), "knnd_set_stream")

    def _check_points(self, points):
        _require(points.is_cuda, "points must be a CUDA tensor")
        _require(points.dtype == self.torch_dtype, f"points must be {self.torch_dtype}")
        _require(points.dim() == 2 and points.shape[0] == self.n and points.shape[1] >= self.m,
                 f"points must be ({self.n}, >= {self.m})")
        _require(points.stride(1) == 1, "each point's coordinates must be contiguous")
        return points.stride(0)

    def new_graph(self, device=None):
        device = device or torch.device("cuda", torch.cuda.current_device())
        idx = torch.empty((self.n, self.K), dtype=torch.int32, device=device)
        key = torch.empty((self.n, self.K), dtype=torch.float64, device=device)
        flag = torch.empty((self.n, self.K), dtype=torch.uint8, device=device)
        return idx, key, flag

    def prepare(self, points):
        ld = self._check_points(points)
        check(self._lib.knnd_prepare(self._h, _ptr(points), ld), "knnd_prepare")

    def init_graph(self, points, seed: int, idx=None, key=None, flag=None):
        ld = self._check_points(points) if points is not None else self.m
        if idx is None:
            idx, key, flag = self.new_graph()
        check(self._lib.knnd_init_graph(self._h, _ptr(points), ld, seed, _ptr(idx), _ptr(key), _ptr(flag)),
              "knnd_init_graph")
        return idx, key, flag

    def round(self, points, seed: int, r: int, idx, key, flag=None, updates=None, fcc_hits=None):
        """In place: (idx, key) G_{r-1} -> G_r.  updates / fcc_hits: int64 device scalars or None."""
        ld = self._check_points(points) if points is not None else self.m
        check(self._lib.knnd_round(self._h, _ptr(points), ld, seed, r, _ptr(idx), _ptr(key), _ptr(flag),
                                   _ptr(updates), _ptr(fcc_hits)), "knnd_round")

    def fcc(self, idx, seed: int, r: int, hits):
        check(self._lib.knnd_fcc(self._h, _ptr(idx), seed, r, _ptr(hits)), "knnd_fcc")

    def sync(self):
        check(self._lib.knnd_sync(self._h), "knnd_sync")

    def build(self, points, seed: int, idx=None, key=None, flag=None) -> dict:
        ld = self._check_points(points)
        if idx is None:
            idx, key, flag = self.new_graph(points.device)
        info = _lib.knnd_build_info()
        check(self._lib.knnd_build(self._h, _ptr(points), ld, seed, _ptr(idx), _ptr(key), _ptr(flag),
                                   ctypes.byref(info)), "knnd_build")
        out = _info_dict(info)
        out.update(idx=idx, key=key, flag=flag)
        return out

    def build_host(self, points_host, seed: int, idx_host=None, key_host=None) -> dict:
        """Build from host memory (pinned for full bandwidth); returns host idx/key."""
        _require(not points_host.is_cuda, "points_host must be a host tensor")
        _require(points_host.dtype == self.torch_dtype, f"points_host must be {self.torch_dtype}")
        _require(points_host.dim() == 2 and points_host.shape[0] == self.n and points_host.shape[1] >= self.m,
                 f"points_host must be ({self.n}, >= {self.m})")
        _require(points_host.stride(1) == 1, "each point's coordinates must be contiguous")
        ld = points_host.stride(0)
        if idx_host is None:
            idx_host = torch.empty((self.n, self.K), dtype=torch.int32, pin_memory=True)
            key_host = torch.empty((self.n, self.K), dtype=torch.float64, pin_memory=True)
        info = _lib.knnd_build_info()
        check(self._lib.knnd_build_host(self._h, _ptr(points_host), ld, seed, _ptr(idx_host), _ptr(key_host),
                                        ctypes.byref(info)), "knnd_build_host")
        out = _info_dict(info)
        out.update(idx=idx_host, key=key_host)
        return out

    def stats(self) -> dict:
        st = _lib.knnd_stats()
        check(self._lib.knnd_get_stats(self._h, ctypes.byref(st)), "knnd_get_stats")
        return {"kernel_launches": st.kernel_launches, "rounds": st.rounds,
                "workspace_bytes": st.workspace_bytes,
                "phase_count": {p: st.phase_count[i] for i, p in enumerate(_lib.PHASES)},
                "phase_ms": {p: st.phase_ms[i] for i, p in enumerate(_lib.PHASES)}}

    def reset_stats(self):
        check(self._lib.knnd_reset_stats(self._h), "knnd_reset_stats")


def build(points, K: int, seed: int = 0, precision: str = "mixed", **kw) -> dict:
    """One-call build on a CUDA (device) or CPU (host) points tensor."""
    n, m = points.shape
    dtype = "f32" if points.dtype == torch.float32 else "f64"
    h = Handle(n, m, K, dtype=dtype, precision=precision, **kw)
    try:
        if points.is_cuda:
            return h.build(points, seed)
        return h.build_host(points.contiguous(), seed)
    finally:
        h.close()


def build_batched(points_list, Ks, seeds, precision: str = "mixed", fcc_samples: int = 10000,
                  max_rounds: int = 64, stop_on_zero_updates: bool = True, workspace_limit: int = 0,
                  incremental: bool = False, stop_delta: float = 0.0, comparator: str = "kl", stream=None,
                  outputs=None, split_den: int = 0, merge_keep: int = 0, join_blocks: int = 0,
                  join_form: str = "auto"):
    """Batched form: build many independent instances together.

    points_list: CUDA tensors (n_i x m_i, one dtype for all); Ks, seeds: per instance.
    Returns a list of dicts (idx, key, rounds, updates, fcc_hits, ...), one per instance.
    """
    lib = _lib.load()
    count = len(points_list)
    _require(count > 0, "need at least one instance")
    _require(len(Ks) == count and len(seeds) == count, "one K and one seed per instance")
    _require(outputs is None or len(outputs) == count, "one (idx, key) pair per instance")
    dt = points_list[0].dtype
    dtype = _DTYPE[dt]
    arr = (_lib.knnd_instance * count)()
    outs = []
    for i, (p, K, sd) in enumerate(zip(points_list, Ks, seeds)):
        _require(p.is_cuda and p.dim() == 2 and p.stride(1) == 1,
                 f"instance {i}: points must be a 2-D CUDA tensor with contiguous rows")
        _require(p.dtype == dt, f"instance {i}: every instance must have the dtype of the first")
        n, m = p.shape
        if outputs is not None:
            idx, key = outputs[i]
        else:
            idx = torch.empty((n, K), dtype=torch.int32, device=p.device)
            key = torch.empty((n, K), dtype=torch.float64, device=p.device)
        outs.append((idx, key))
        arr[i] = _lib.knnd_instance(p.data_ptr(), p.stride(0), n, m, K, sd, idx.data_ptr(), key.data_ptr())
    prm = _lib.knnd_params(fcc_samples, max_rounds, int(stop_on_zero_updates), 0, 0, int(incremental),
                           float(stop_delta), _CMP[comparator], _lib.KNND_LOOP_AUTO, int(split_den), int(merge_keep),
                           int(join_blocks), _JOIN[join_form])
    infos = (_lib.knnd_build_info * count)()
    check(lib.knnd_build_batched(count, ctypes.cast(arr, ctypes.c_void_p), dtype, _PREC[precision],
                                 ctypes.byref(prm), workspace_limit, ctypes.cast(infos, ctypes.c_void_p),
                                 _stream_ptr(stream)), "knnd_build_batched")
    res = []
    for i in range(count):
        d = _info_dict(infos[i])
        d.update(idx=outs[i][0], key=outs[i][1])
        res.append(d)
    return res
