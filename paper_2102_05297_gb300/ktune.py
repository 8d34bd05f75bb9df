"""Thin ctypes binding of libktune (include/ktune.h).

Every function here only marshals arguments: each ``ktune_*`` name is the C
entry point of the same name, called with plain pointers and sizes.  The
library must be built (``python -m paper_2102_05297_gb300.build``); importing
this module without it raises ImportError, so there is no silent fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import struct
from typing import List, Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libktune.so")
if not os.path.exists(LIB_PATH):
    raise ImportError("libktune.so is not built; run `python -m paper_2102_05297_gb300.build`")
lib = C.CDLL(LIB_PATH)

KTUNE_OK, KTUNE_EINVAL, KTUNE_ENOMEM, KTUNE_EMODEL = 0, -1, -2, -3
KTUNE_EXHAUSTED, KTUNE_ETIMEOUT, KTUNE_ECUDA, KTUNE_ESTATE = -4, -5, -6, -7
KTUNE_MATERIALISE, KTUNE_ON_THE_FLY = 0, 1
KTUNE_SELECT_SAMPLE, KTUNE_SELECT_TOPK = 0, 1
MODEL_MAGIC = 0x314D544B


class ktune_space_desc(C.Structure):
    _fields_ = [("n_params", C.c_int), ("n_values", C.POINTER(C.c_int)),
                ("values", C.POINTER(C.c_int64)), ("bytecode", C.POINTER(C.c_int32)),
                ("n_bytecode", C.c_int)]


class ktune_search_opts(C.Structure):
    _fields_ = [("k", C.c_int), ("inst_reaction", C.c_double), ("gamma", C.c_float),
                ("cores", C.c_double), ("seed", C.c_uint64), ("search_id", C.c_uint32),
                ("select", C.c_int)]


class ktune_step_stats(C.Structure):
    _fields_ = [("n_scored", C.c_int64), ("n_active", C.c_int), ("depth", C.c_int),
                ("s_min", C.c_float), ("s_max", C.c_float), ("n_kernels", C.c_int),
                ("kernel_ms", C.c_float * 8)]


_vp, _i64p, _f32p, _i32p = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_float), C.POINTER(C.c_int)
_SIGS = {
    "ktune_abi_version": ([], C.c_int),
    "ktune_last_error": ([], C.c_char_p),
    "ktune_space_create": ([C.POINTER(ktune_space_desc), C.c_int, _vp, C.POINTER(_vp)], C.c_int),
    "ktune_space_destroy": ([_vp], C.c_int),
    "ktune_space_count": ([_vp, _i64p, _i64p], C.c_int),
    "ktune_space_decode": ([_vp, C.c_int64, _i64p], C.c_int),
    "ktune_space_valid_raw": ([_vp, C.c_int64, C.c_int64, _i64p], C.c_int),
    "ktune_space_valid_digits": ([_vp, C.c_int64, C.c_int64, _vp], C.c_int),
    "ktune_space_packed_device": ([_vp], _vp),
    "ktune_model_load": ([_vp, _vp, C.c_size_t, C.POINTER(_vp)], C.c_int),
    "ktune_model_destroy": ([_vp], C.c_int),
    "ktune_model_info": ([_vp, _i32p, _i32p], C.c_int),
    "ktune_model_predict_device": ([_vp, C.c_int64, C.c_int64, _vp, _vp], C.c_int),
    "ktune_search_create": ([_vp, _vp, C.POINTER(ktune_search_opts), _vp, C.POINTER(_vp)], C.c_int),
    "ktune_search_destroy": ([_vp], C.c_int),
    "ktune_search_current": ([_vp, _i64p], C.c_int),
    "ktune_search_set_profile": ([_vp, C.c_int64], C.c_int),
    "ktune_step": ([_vp, _f32p, C.c_int, _i64p, _f32p, _i32p], C.c_int),
    "ktune_step_device": ([_vp, _f32p, C.c_int, _vp, _vp, _vp, _vp], C.c_int),
    "ktune_report": ([_vp, C.POINTER(C.c_double), C.c_int], C.c_int),
    "ktune_search_evaluated": ([_vp, _i64p], C.c_int),
    "ktune_search_stats": ([_vp, C.POINTER(ktune_step_stats)], C.c_int),
    "ktune_search_set_timing": ([_vp, C.c_int], C.c_int),
    "ktune_search_set_cached": ([_vp, C.c_int], C.c_int),
    "ktune_search_set_neighbourhood": ([_vp, C.c_int], C.c_int),
    "ktune_search_scores_device": ([_vp, C.c_int64, C.c_int64, _vp, _vp, _vp], C.c_int),
    "ktune_search_set_fused": ([_vp, C.c_int], C.c_int),
    "ktune_search_save": ([_vp, _vp, C.POINTER(C.c_size_t)], C.c_int),
    "ktune_search_load": ([_vp, _vp, _vp, C.c_size_t, _vp, C.POINTER(_vp)], C.c_int),
    "ktune_batch_create": ([C.POINTER(_vp), C.c_int, _vp, C.POINTER(_vp)], C.c_int),
    "ktune_batch_destroy": ([_vp], C.c_int),
    "ktune_batch_step": ([_vp, C.POINTER(_f32p), C.c_int, _i64p, _f32p, _i32p], C.c_int),
    "ktune_batch_autotune": ([_vp, C.POINTER(_f32p), C.c_int, _i32p, _f32p, C.c_int], C.c_int),
    "ktune_batch_variant": ([C.c_int, _i32p, _i32p, _i32p], C.c_int),
    "ktune_score_noalloc": ([_vp, C.c_int64, _vp, _vp, _vp, C.c_int, C.c_int, _i32p, _vp,
                             C.c_uint64, C.c_double, C.c_double, _vp, _vp, _vp], C.c_int),
    "ktune_mlp_create": ([_vp, C.c_int, _i32p, _f32p, C.c_int, _vp, C.POINTER(_vp)], C.c_int),
    "ktune_mlp_destroy": ([_vp], C.c_int),
    "ktune_mlp_info": ([_vp, _i32p, _i64p], C.c_int),
    "ktune_mlp_set_params": ([_vp, _f32p], C.c_int),
    "ktune_mlp_get_params": ([_vp, _f32p], C.c_int),
    "ktune_mlp_set_data": ([_vp, _i64p, _f32p, C.c_int64], C.c_int),
    "ktune_mlp_grads": ([_vp, _i32p, C.c_int, C.POINTER(C.c_double), _f32p], C.c_int),
    "ktune_mlp_train": ([_vp, _i32p, C.c_int, C.c_int, C.c_float, C.POINTER(C.c_double)], C.c_int),
    "ktune_mlp_predict": ([_vp, _i64p, C.c_int64, _f32p], C.c_int),
    "ktune_mlp_predict_device": ([_vp, C.c_int64, C.c_int64, _vp, _vp], C.c_int),
    "ktune_model_from_mlp": ([_vp, C.POINTER(_vp)], C.c_int),
    "ktune_mlp_set_wait": ([_vp, C.c_uint64, C.c_int], C.c_int),
    "ktune_gemm_bf16": ([_vp, C.c_int, _vp, C.c_int, _vp, C.c_int, C.c_int, C.c_int, C.c_int,
                         _vp], C.c_int),
}
EXPORTED = list(_SIGS)
for _n, (_a, _r) in _SIGS.items():
    _f = getattr(lib, _n)
    _f.argtypes = _a
    _f.restype = _r
    globals()[_n] = _f


class KtuneError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s failed (%d): %s" % (where, code, lib.ktune_last_error().decode()))


def check(rc: int, where: str) -> int:
    if rc != KTUNE_OK:
        raise KtuneError(rc, where)
    return rc


def _arr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.POINTER(np.ctypeslib.as_ctypes_type(dtype)))


# ---------------------------------------------------------------------------
def model_blob(model: dict) -> bytes:
    """Serialise a tree ensemble ({"roles", "trees"}), a least-squares model
    ({"kind": "lsq", "roles", "coef" [n_sub][K][T]}) or a measured counter table
    ({"kind": "table", "roles", "table" [N][K] in TS order}); layouts in
    include/ktune.h."""
    roles = model["roles"]
    if model.get("kind") == "table":
        table = np.ascontiguousarray(model["table"], "<f4")
        assert table.ndim == 2 and table.shape[1] == len(roles)
        return b"".join([struct.pack("<4I", MODEL_MAGIC, 1, 2, len(roles)),
                         np.asarray(roles, "<i4").tobytes(),
                         struct.pack("<Q", table.shape[0]), table.tobytes()])
    if model.get("kind") == "lsq":
        coef = np.ascontiguousarray(model["coef"], "<f4")
        assert coef.ndim == 3 and coef.shape[1] == len(roles)
        return b"".join([struct.pack("<4I", MODEL_MAGIC, 1, 3, len(roles)),
                         np.asarray(roles, "<i4").tobytes(),
                         struct.pack("<2I", coef.shape[0], coef.shape[2]), coef.tobytes()])
    out = [struct.pack("<4I", MODEL_MAGIC, 1, 1, len(roles)),
           np.asarray(roles, "<i4").tobytes()]
    for t in model["trees"]:
        n = len(t["feature"])
        out.append(struct.pack("<I", n))
        for key, dt in (("feature", "<i4"), ("threshold", "<i4"), ("left", "<i4"),
                        ("right", "<i4"), ("value", "<f4")):
            out.append(np.asarray(t[key], dt).tobytes())
    return b"".join(out)


def _stream_ptr(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Space:
    """Owns a ktune_space handle."""

    def __init__(self, values: Sequence[Sequence[int]], bytecode: Sequence[int] = (),
                 flags: int = KTUNE_MATERIALISE, stream=None):
        self.radices = [len(v) for v in values]
        nv, self._nv = _arr(self.radices, np.int32)
        vals, self._vals = _arr([x for v in values for x in v], np.int64)
        bc, self._bc = _arr(list(bytecode) or [0], np.int32)
        self._keep = (nv, vals, bc)
        d = ktune_space_desc(len(values), self._nv, self._vals, self._bc, len(bytecode))
        h = C.c_void_p()
        check(lib.ktune_space_create(C.byref(d), flags, _stream_ptr(stream), C.byref(h)),
              "ktune_space_create")
        self.h = h
        self.flags = flags

    @classmethod
    def from_desc(cls, desc, flags=KTUNE_MATERIALISE, stream=None):
        return cls(desc.values, desc.bytecode, flags, stream)

    def count(self):
        nv, nr = C.c_int64(), C.c_int64()
        check(lib.ktune_space_count(self.h, C.byref(nv), C.byref(nr)), "ktune_space_count")
        return nv.value, nr.value

    def decode(self, raw: int) -> List[int]:
        out = (C.c_int64 * len(self.radices))()
        check(lib.ktune_space_decode(self.h, raw, out), "ktune_space_decode")
        return list(out)

    def valid_raw(self, first: int = 0, count: Optional[int] = None) -> np.ndarray:
        if count is None:
            count = self.count()[0] - first
        out = np.empty(count, np.int64)
        check(lib.ktune_space_valid_raw(self.h, first, count,
                                        out.ctypes.data_as(C.POINTER(C.c_int64))),
              "ktune_space_valid_raw")
        return out

    def valid_digits(self, first: int = 0, count: Optional[int] = None) -> np.ndarray:
        if count is None:
            count = self.count()[0] - first
        out = np.empty((count, len(self.radices)), np.uint8)
        check(lib.ktune_space_valid_digits(self.h, first, count, out.ctypes.data),
              "ktune_space_valid_digits")
        return out

    def packed_device(self) -> int:
        return lib.ktune_space_packed_device(self.h) or 0

    def close(self):
        if getattr(self, "h", None):
            lib.ktune_space_destroy(self.h)
            self.h = None

    __del__ = close


class Model:
    """Owns a ktune_model handle: a tree ensemble or a least-squares model
    (dict, see model_blob) or, through ``Model.from_mlp``, a view of an Mlp."""

    @classmethod
    def from_mlp(cls, mlp: "Mlp") -> "Model":
        self = cls.__new__(cls)
        h = C.c_void_p()
        check(lib.ktune_model_from_mlp(mlp.h, C.byref(h)), "ktune_model_from_mlp")
        self.h = h
        self.space = mlp.space
        self.mlp = mlp            # keeps the MLP alive as long as the model
        self.K, self.depth = mlp.K, 0
        return self

    def __init__(self, space: Space, model: dict):
        blob = model_blob(model)
        self._blob = C.create_string_buffer(blob, len(blob))
        h = C.c_void_p()
        check(lib.ktune_model_load(space.h, self._blob, len(blob), C.byref(h)), "ktune_model_load")
        self.h = h
        self.space = space
        k, d = C.c_int(), C.c_int()
        check(lib.ktune_model_info(h, C.byref(k), C.byref(d)), "ktune_model_info")
        self.K, self.depth = k.value, d.value

    def predict_device(self, first: int, count: int, out_ptr: int, stream=None):
        check(lib.ktune_model_predict_device(self.h, first, count, out_ptr, _stream_ptr(stream)),
              "ktune_model_predict_device")

    def close(self):
        if getattr(self, "h", None):
            lib.ktune_model_destroy(self.h)
            self.h = None

    __del__ = close


class Search:
    def __init__(self, space: Space, model: Model, k: int = 5, inst_reaction: float = 0.7,
                 gamma: float = -0.25, cores: float = 1000.0, seed: int = 0, search_id: int = 0,
                 select: int = KTUNE_SELECT_SAMPLE, stream=None):
        o = ktune_search_opts(k, inst_reaction, gamma, cores, seed, search_id, select)
        h = C.c_void_p()
        check(lib.ktune_search_create(space.h, model.h, C.byref(o), _stream_ptr(stream),
                                      C.byref(h)), "ktune_search_create")
        self.h = h
        self.k = k
        self.K = model.K
        self.space, self.model = space, model
        self._buffers()

    def _buffers(self):
        """step()'s argument buffers, with their ctypes pointers made once."""
        self._raw = np.empty(64, np.int64)
        self._score = np.empty(64, np.float32)
        self._cnt = np.empty(64, np.float32)
        self._cnt_p = self._cnt.ctypes.data_as(_f32p)
        self._raw_p = self._raw.ctypes.data_as(_i64p)
        self._score_p = self._score.ctypes.data_as(_f32p)
        self._n = C.c_int()
        self._n_ref = C.byref(self._n)

    def current(self) -> int:
        r = C.c_int64()
        check(lib.ktune_search_current(self.h, C.byref(r)), "ktune_search_current")
        return r.value

    def set_profile(self, raw: int):
        check(lib.ktune_search_set_profile(self.h, raw), "ktune_search_set_profile")

    def step(self, counters, k: Optional[int] = None):
        """Returns (raw indices, scores); raises KtuneError except on
        KTUNE_EXHAUSTED, where the partial batch is returned."""
        k = self.k if k is None else k
        c = np.asarray(counters, np.float32).reshape(-1)
        if c.shape[0] < self.K:
            raise ValueError("expected %d counters, got %d" % (self.K, c.shape[0]))
        self._cnt[:self.K] = c[:self.K]
        rc = lib.ktune_step(self.h, self._cnt_p, k, self._raw_p, self._score_p, self._n_ref)
        if rc not in (KTUNE_OK, KTUNE_EXHAUSTED):
            check(rc, "ktune_step")
        n = self._n.value
        return self._raw[:n].copy(), self._score[:n].copy()

    def step_device(self, counters, k: int, out_raw_ptr: int, out_score_ptr: int,
                    n_out_ptr: int = 0, stream=None):
        """Enqueue a step; counters on the host, outputs in device memory."""
        c, cp = _arr(counters, np.float32)
        check(lib.ktune_step_device(self.h, cp, k, out_raw_ptr, out_score_ptr,
                                    n_out_ptr or None, _stream_ptr(stream)), "ktune_step_device")

    def report(self, runtimes):
        r, rp = _arr(runtimes, np.float64)
        check(lib.ktune_report(self.h, rp, len(r)), "ktune_report")

    def evaluated(self) -> int:
        n = C.c_int64()
        check(lib.ktune_search_evaluated(self.h, C.byref(n)), "ktune_search_evaluated")
        return n.value

    def stats(self) -> ktune_step_stats:
        st = ktune_step_stats()
        check(lib.ktune_search_stats(self.h, C.byref(st)), "ktune_search_stats")
        return st

    def set_timing(self, enable: bool = True):
        check(lib.ktune_search_set_timing(self.h, int(enable)), "ktune_search_set_timing")

    def set_cached(self, enable: bool = True):
        """Predict all of TS once and score later steps from the cache."""
        check(lib.ktune_search_set_cached(self.h, int(enable)), "ktune_search_set_cached")

    def set_neighbourhood(self, radius: int):
        """Restrict later steps to c_profile's Hamming neighbourhood (0: off)."""
        check(lib.ktune_search_set_neighbourhood(self.h, int(radius)),
              "ktune_search_set_neighbourhood")

    def set_fused(self, shape: int = 1):
        """0: four kernels per step; 1..3: the whole step as one persistent
        kernel of that shape (ktune_search_set_fused)."""
        check(lib.ktune_search_set_fused(self.h, int(shape)), "ktune_search_set_fused")

    def scores_device(self, first: int, count: int, scores_ptr: int = 0, weights_ptr: int = 0,
                      stream=None):
        """Copy the last step's scores / integer weights of TS[first, first+count)
        into device buffers (ktune_search_scores_device; 0 skips one)."""
        check(lib.ktune_search_scores_device(self.h, first, count, scores_ptr or None,
                                             weights_ptr or None, _stream_ptr(stream)),
              "ktune_search_scores_device")

    def save(self) -> bytes:
        """The search's checkpoint (ktune_search_save)."""
        n = C.c_size_t(0)
        check(lib.ktune_search_save(self.h, None, C.byref(n)), "ktune_search_save")
        buf = C.create_string_buffer(n.value)
        check(lib.ktune_search_save(self.h, buf, C.byref(n)), "ktune_search_save")
        return buf.raw[:n.value]

    @classmethod
    def load(cls, space: Space, model: Model, blob: bytes, stream=None) -> "Search":
        """A search restored from a checkpoint (ktune_search_load)."""
        self = cls.__new__(cls)
        h = C.c_void_p()
        buf = C.create_string_buffer(blob, len(blob))
        check(lib.ktune_search_load(space.h, model.h, buf, len(blob), _stream_ptr(stream),
                                    C.byref(h)), "ktune_search_load")
        self.h = h
        hdr_k = int.from_bytes(blob[40:44], "little")   # opts.k
        self.k = hdr_k
        self.K = model.K
        self.space, self.model = space, model
        self._buffers()
        return self

    def close(self):
        if getattr(self, "h", None):
            lib.ktune_search_destroy(self.h)
            self.h = None

    __del__ = close


class Batch:
    """Owns a ktune_batch over Search objects (which must outlive it)."""

    def __init__(self, searches, stream=None):
        self.searches = list(searches)
        arr = (C.c_void_p * len(self.searches))(*[x.h.value for x in self.searches])
        h = C.c_void_p()
        check(lib.ktune_batch_create(arr, len(arr), _stream_ptr(stream), C.byref(h)),
              "ktune_batch_create")
        self.h = h

    def _counters(self, counters):
        keep = [np.ascontiguousarray(c, dtype=np.float32) for c in counters]
        ptrs = (C.POINTER(C.c_float) * len(keep))(
            *[c.ctypes.data_as(C.POINTER(C.c_float)) for c in keep])
        return keep, ptrs

    def step(self, counters, k: int):
        """One step of every search; returns per search (raw indices, scores)."""
        n = len(self.searches)
        keep, ptrs = self._counters(counters)
        raw = np.zeros(n * k, np.int64)
        sc = np.zeros(n * k, np.float32)
        no = np.zeros(n, np.int32)
        rc = lib.ktune_batch_step(self.h, ptrs, k, raw.ctypes.data_as(C.POINTER(C.c_int64)),
                                  sc.ctypes.data_as(C.POINTER(C.c_float)),
                                  no.ctypes.data_as(C.POINTER(C.c_int)))
        if rc not in (KTUNE_OK, KTUNE_EXHAUSTED):
            check(rc, "ktune_batch_step")
        return [(raw[i * k:i * k + no[i]].copy(), sc[i * k:i * k + no[i]].copy()) for i in range(n)]

    def autotune(self, counters, reps: int = 5):
        keep, ptrs = self._counters(counters)
        nv = lib.ktune_batch_variant(0, None, None, None)
        ms = np.zeros(nv, np.float32)
        ch = C.c_int()
        check(lib.ktune_batch_autotune(self.h, ptrs, reps, C.byref(ch),
                                       ms.ctypes.data_as(C.POINTER(C.c_float)), nv),
              "ktune_batch_autotune")
        return ch.value, ms

    @staticmethod
    def variant(v: int):
        t, c, i = C.c_int(), C.c_int(), C.c_int()
        lib.ktune_batch_variant(v, C.byref(t), C.byref(c), C.byref(i))
        return t.value, c.value, i.value

    def close(self):
        if getattr(self, "h", None):
            lib.ktune_batch_destroy(self.h)
            self.h = None

    __del__ = close


# ---------------------------------------------------------------------------
MLP_HIDDEN = 256


class Mlp:
    """Owns a ktune_mlp handle (the MLP counter model, trained on the GPU).

    Parameters travel as a dict of float32 arrays W1 [256, F], b1 [256], W2,
    b2, W3, b3, W4 [K, 256], b4 [K], flattened in that order for the C call."""

    NAMES = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")

    def __init__(self, space: Space, roles, ranges, max_batch: int = 4096, stream=None):
        roles_a, roles_p = _arr(roles, np.int32)
        rng_a, rng_p = _arr(ranges, np.float32)
        h = C.c_void_p()
        check(lib.ktune_mlp_create(space.h, len(roles_a), roles_p, rng_p, max_batch,
                                   _stream_ptr(stream), C.byref(h)), "ktune_mlp_create")
        self.h = h
        self.space = space
        self.K = len(roles_a)
        f, n = C.c_int(), C.c_int64()
        check(lib.ktune_mlp_info(h, C.byref(f), C.byref(n)), "ktune_mlp_info")
        self.F, self.n_params = f.value, n.value

    def shapes(self):
        H, F, K = MLP_HIDDEN, self.F, self.K
        return {"W1": (H, F), "b1": (H,), "W2": (H, H), "b2": (H,), "W3": (H, H), "b3": (H,),
                "W4": (K, H), "b4": (K,)}

    def _flat(self, params) -> np.ndarray:
        sh = self.shapes()
        parts = []
        for k in self.NAMES:
            a = np.asarray(params[k], dtype=np.float32)
            if a.shape != sh[k]:
                raise ValueError("%s has shape %s, expected %s" % (k, a.shape, sh[k]))
            parts.append(a.ravel())
        return np.ascontiguousarray(np.concatenate(parts), dtype=np.float32)

    def _unflat(self, flat) -> dict:
        out, o = {}, 0
        for k in self.NAMES:
            shp = self.shapes()[k]
            n = int(np.prod(shp))
            out[k] = flat[o:o + n].reshape(shp).copy()
            o += n
        return out

    def set_params(self, params: dict):
        flat = self._flat(params)
        check(lib.ktune_mlp_set_params(self.h, flat.ctypes.data_as(_f32p)), "ktune_mlp_set_params")

    def get_params(self) -> dict:
        flat = np.empty(self.n_params, dtype=np.float32)
        check(lib.ktune_mlp_get_params(self.h, flat.ctypes.data_as(_f32p)), "ktune_mlp_get_params")
        return self._unflat(flat)

    def set_data(self, raw, counters):
        raw_a, raw_p = _arr(raw, np.int64)
        c_a, c_p = _arr(np.asarray(counters, dtype=np.float32).reshape(len(raw_a), self.K),
                        np.float32)
        check(lib.ktune_mlp_set_data(self.h, raw_p, c_p, len(raw_a)), "ktune_mlp_set_data")

    def grads(self, idx):
        idx_a, idx_p = _arr(idx, np.int32)
        loss = C.c_double()
        flat = np.empty(self.n_params, dtype=np.float32)
        check(lib.ktune_mlp_grads(self.h, idx_p, len(idx_a), C.byref(loss),
                                  flat.ctypes.data_as(_f32p)), "ktune_mlp_grads")
        return loss.value, self._unflat(flat)

    def train(self, idx, batch: int, lr: float = 1e-3, return_losses: bool = True):
        idx_a, idx_p = _arr(idx, np.int32)
        steps = len(idx_a) // batch
        losses = np.zeros(max(steps, 1), dtype=np.float64)
        check(lib.ktune_mlp_train(self.h, idx_p, batch, steps, lr,
                                  losses.ctypes.data_as(C.POINTER(C.c_double))
                                  if return_losses else None), "ktune_mlp_train")
        return losses[:steps]

    def predict(self, raw) -> np.ndarray:
        raw_a, raw_p = _arr(raw, np.int64)
        out = np.empty((len(raw_a), self.K), dtype=np.float32)
        check(lib.ktune_mlp_predict(self.h, raw_p, len(raw_a), out.ctypes.data_as(_f32p)),
              "ktune_mlp_predict")
        return out

    def set_wait(self, limit_ns: int = 1000000000, stall: bool = False):
        """Limit of each bounded wait of the forward kernel; stall=True makes
        later launches wait on a barrier nothing arrives at (ktune_mlp_set_wait)."""
        check(lib.ktune_mlp_set_wait(self.h, int(limit_ns), int(stall)), "ktune_mlp_set_wait")

    def predict_device(self, first: int, count: int, out_ptr: int, stream=None):
        check(lib.ktune_mlp_predict_device(self.h, first, count, out_ptr, _stream_ptr(stream)),
              "ktune_mlp_predict_device")

    def close(self):
        if getattr(self, "h", None):
            lib.ktune_mlp_destroy(self.h)
            self.h = None

    __del__ = close


def gemm_bf16(a_ptr: int, lda: int, b_ptr: int, ldb: int, c_ptr: int, ldc: int, M: int, N: int,
              Kd: int, stream=None):
    """C = A B^T on the tensor cores (device pointers; see ktune_gemm_bf16)."""
    check(lib.ktune_gemm_bf16(a_ptr, lda, b_ptr, ldb, c_ptr, ldc, M, N, Kd, _stream_ptr(stream)),
          "ktune_gemm_bf16")
