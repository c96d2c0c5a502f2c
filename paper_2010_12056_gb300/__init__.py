"""GB300 CP-ALS engine: Python binding of libcpals.so (argument marshalling only).

Every step of the decomposition runs in the library's CUDA kernels behind the C
ABI declared in include/cpals.h; this module converts arguments, keeps the
borrowed tensor alive and turns status codes into exceptions.  There is no CPU
fallback: if libcpals.so is missing or fails to load, every call raises.

PyTorch supplies device memory (the input tensor, output buffers) and the CUDA
stream the library enqueues on (the current torch stream at construction).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcpals.so")
_lib = None

PREC = {"fp32": 0, "tf32": 1, "bf16x3": 2, "bf16": 3, "tf32x3": 4, "f16x3": 5}
STATUS = {0: "CP_OK", 1: "CP_EINVAL", 2: "CP_ENOMEM", 3: "CP_ECUDA", 4: "CP_ENOTSPD",
          5: "CP_ENUMERIC", 6: "CP_ETIMEOUT", 7: "CP_ESTATE"}
KINDS = {0: "dt", 1: "msdt", 2: "pp", 3: "pp-regular"}
N_POLICY_PARAMS = 4801


class CPError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"{STATUS.get(code, code)}: {msg}")


class Config(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("pp_eps", ctypes.c_double), ("delta", ctypes.c_double),
                ("max_sweeps", ctypes.c_int), ("judge_every", ctypes.c_int),
                ("policy_gate", ctypes.c_int), ("seed", ctypes.c_uint64)]


class TraceRec(ctypes.Structure):
    _fields_ = [("sweep", ctypes.c_int32), ("kind", ctypes.c_int32), ("pp_init", ctypes.c_int32),
                ("rolled_back", ctypes.c_int32), ("resid", ctypes.c_double),
                ("max_rel_step", ctypes.c_double), ("max_rel_dAp", ctypes.c_double),
                ("v_share", ctypes.c_double), ("ms", ctypes.c_double),
                ("p_cur", ctypes.c_float), ("p_new", ctypes.c_float),
                ("decided_by", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ProbeRec(ctypes.Structure):
    _fields_ = [("feat_cur", ctypes.c_float * 8), ("feat_new", ctypes.c_float * 8),
                ("r0", ctypes.c_double), ("r_exact", ctypes.c_double), ("r_cur", ctypes.c_double),
                ("r_new", ctypes.c_double), ("ms_exact", ctypes.c_double), ("ms_cur", ctypes.c_double),
                ("ms_new", ctypes.c_double), ("has_ops", ctypes.c_int32), ("label_cur", ctypes.c_int32),
                ("label_new", ctypes.c_int32), ("followed", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("ttm", ctypes.c_int64), ("mttv", ctypes.c_int64), ("pp_init", ctypes.c_int64),
                ("sweeps_exact", ctypes.c_int64), ("sweeps_pp", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("ttm_flops", ctypes.c_double),
                ("mttv_flops", ctypes.c_double), ("pp_flops", ctypes.c_double),
                ("ttm_bytes", ctypes.c_double), ("mttv_bytes", ctypes.c_double),
                ("ttm_tensor_core", ctypes.c_int64), ("ttm_fused", ctypes.c_int64),
                ("solves_fp64", ctypes.c_int64), ("rollbacks", ctypes.c_int64),
                ("lookahead", ctypes.c_int64), ("ttm_child", ctypes.c_int64),
                ("ttm_stored_parts", ctypes.c_int64)]


OPTIONS = {"fuse_dt": 1, "lookahead": 2, "fuse_child": 3, "wait_limit": 4, "msdt_levels": 5, "solve_fp64": 6,
           "ttm_presplit": 7}

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "cp_config_default": (None, [ctypes.POINTER(Config)]),
    "cp_init": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(ctypes.c_int64), _I, _P, _I,
                     ctypes.POINTER(_D), ctypes.POINTER(Config), _P]),
    "cp_load_tensor": (_I, [_P, _P, _I]),
    "cp_mttkrp": (_I, [_P, _I, _P]),
    "cp_ttm": (_I, [_P, _I, _P]),
    "cp_sweep_dt": (_I, [_P, _I]),
    "cp_sweep_msdt": (_I, [_P, _I]),
    "cp_sweep_pp": (_I, [_P, _I, _D, _P]),
    "cp_pp_init": (_I, [_P]),
    "cp_run": (_I, [_P, _I, _P, ctypes.POINTER(_I)]),
    "cp_pp_probe": (_I, [_P, _I, ctypes.POINTER(ProbeRec)]),
    "cp_policy_features": (_I, [_P, ctypes.POINTER(ctypes.c_float)]),
    "cp_pp_mttkrp": (_I, [_P, _I, _P]),
    "cp_fit": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "cp_get_factor": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "cp_set_factor": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "cp_get_trace": (_I, [_P, ctypes.POINTER(TraceRec), ctypes.POINTER(ctypes.c_size_t)]),
    "cp_get_stats": (_I, [_P, ctypes.POINTER(Stats)]),
    "cp_set_option": (_I, [_P, _I, _I]),
    "cp_last_error": (ctypes.c_char_p, [_P]),
    "cp_free": (None, [_P]),
    "cp_policy_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_float), _P]),
    "cp_policy_get": (_I, [_P, ctypes.POINTER(ctypes.c_float)]),
    "cp_policy_forward": (_I, [_P, _P, _I, _P]),
    "cp_policy_grad": (_I, [_P, _P, _P, _I, _P, _P]),
    "cp_policy_train": (_I, [_P, _P, _P, _I, _I, ctypes.c_float]),
    "cp_policy_free": (None, [_P]),
    "cp_resid_noalloc": (_I, [_I, ctypes.POINTER(ctypes.c_int64), _I, _P, ctypes.POINTER(_P), _P, _P]),
}


def lib():
    """Load libcpals.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


class CPContext:
    """One decomposition of a dense tensor: a float32 CUDA tensor is borrowed, a
    float64 CUDA tensor converted once, a float32 CPU tensor (pinned for full
    bandwidth) copied once to the device by the library."""

    def __init__(self, T, R, A0=None, prec="f16x3", seed=20101205, pp_eps=0.1, judge_every=5,
                 policy_gate=True, delta=0.0, max_sweeps=0, stream=None):
        import torch
        if not (isinstance(T, torch.Tensor) and T.is_contiguous()):
            raise ValueError("T must be a contiguous tensor")
        if T.is_cuda:
            if T.dtype not in (torch.float32, torch.float64):
                raise ValueError("T must be float32 or float64")
            dtype = 1 if T.dtype == torch.float64 else 0
        else:
            if T.dtype != torch.float32:
                raise ValueError("a host tensor must be float32")
            dtype = 2
        self._L = lib()
        self.T = T
        self.dims = [int(d) for d in T.shape]
        self.N = len(self.dims)
        self.R = int(R)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        cfg = Config()
        self._L.cp_config_default(ctypes.byref(cfg))
        cfg.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        cfg.seed = int(seed)
        cfg.pp_eps = float(pp_eps)
        cfg.judge_every = int(judge_every)
        cfg.policy_gate = 1 if policy_gate else 0
        cfg.delta = float(delta)
        cfg.max_sweeps = int(max_sweeps)
        dims = (ctypes.c_int64 * self.N)(*self.dims)
        a0p = None
        if A0 is not None:
            flat = np.ascontiguousarray(np.concatenate([np.asarray(a, np.float64).ravel() for a in A0]))
            expect = sum(d * self.R for d in self.dims)
            if flat.size != expect:
                raise ValueError("A0 sizes do not match dims x R")
            self._a0 = flat
            a0p = flat.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        st = self._L.cp_init(ctypes.byref(h), self.N, dims, self.R, _dptr(T), dtype, a0p, ctypes.byref(cfg),
                             _stream_ptr(self._stream))
        if dtype == 2:
            self.T = None   # the library holds its own device copy
        self._dev = torch.device("cuda", torch.cuda.current_device()) if dtype == 2 else T.device
        if st != 0:
            raise CPError(st, "cp_init failed")
        self._h = h

    # -- helpers
    def _ck(self, st):
        if st != 0:
            msg = self._L.cp_last_error(self._h)
            raise CPError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            self._L.cp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls
    def mttkrp(self, mode, out=None):
        import torch
        if out is None:
            out = torch.empty(self.dims[mode], self.R, dtype=torch.float32, device=self._dev)
        self._ck(self._L.cp_mttkrp(self._h, int(mode), _dptr(out)))
        return out

    def ttm(self, mode, out=None):
        import torch
        if out is None:
            shape = [d for k, d in enumerate(self.dims) if k != mode] + [self.R]
            out = torch.empty(shape, dtype=torch.float32, device=self._dev)
        self._ck(self._L.cp_ttm(self._h, int(mode), _dptr(out)))
        return out

    def load_tensor(self, T=None):
        """cp_load_tensor: a new tensor of the same sizes (float32, host or CUDA), copied
        into the library's own buffer; None: the borrowed tensor changed in place."""
        import torch
        if T is None:
            self._ck(self._L.cp_load_tensor(self._h, None, 0))
            return
        if not (T.is_contiguous() and T.dtype == torch.float32 and list(T.shape) == self.dims):
            raise ValueError("T must be a contiguous float32 tensor of the context's sizes")
        self._ck(self._L.cp_load_tensor(self._h, _dptr(T), 0 if T.is_cuda else 1))

    def sweep_dt(self, n=1):
        self._ck(self._L.cp_sweep_dt(self._h, int(n)))

    def sweep_msdt(self, n=1):
        self._ck(self._L.cp_sweep_msdt(self._h, int(n)))

    def sweep_pp(self, n=1, eps=0.1, policy=None):
        self._ck(self._L.cp_sweep_pp(self._h, int(n), float(eps), policy._h if policy else None))

    def pp_init(self):
        self._ck(self._L.cp_pp_init(self._h))

    def run(self, route="msdt", policy=None):
        """cp_run: sweeps until |r - r_old| <= delta or max_sweeps (given at construction)."""
        n = ctypes.c_int(0)
        rt = {"dt": 0, "msdt": 1, "pp": 2}[route]
        self._ck(self._L.cp_run(self._h, rt, policy._h if policy else None, ctypes.byref(n)))
        return n.value

    def pp_mttkrp(self, mode, out=None):
        import torch
        if out is None:
            out = torch.empty(self.dims[mode], self.R, dtype=torch.float32, device=self._dev)
        self._ck(self._L.cp_pp_mttkrp(self._h, int(mode), _dptr(out)))
        return out

    def fit(self, exact=False):
        f, r = ctypes.c_double(), ctypes.c_double()
        self._ck(self._L.cp_fit(self._h, 1 if exact else 0, ctypes.byref(f), ctypes.byref(r)))
        return f.value, r.value

    def get_factor(self, mode):
        out = np.empty((self.dims[mode], self.R), dtype=np.float64)
        self._ck(self._L.cp_get_factor(self._h, int(mode), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def factors(self):
        return [self.get_factor(n) for n in range(self.N)]

    def set_factor(self, mode, A):
        A = np.ascontiguousarray(A, dtype=np.float64)
        if A.shape != (self.dims[mode], self.R):
            raise ValueError("bad factor shape")
        self._ck(self._L.cp_set_factor(self._h, int(mode), A.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def trace(self):
        n = ctypes.c_size_t(0)
        self._ck(self._L.cp_get_trace(self._h, None, ctypes.byref(n)))
        buf = (TraceRec * max(1, n.value))()
        self._ck(self._L.cp_get_trace(self._h, buf, ctypes.byref(n)))
        out = []
        for i in range(n.value):
            r = buf[i]
            out.append({"sweep": r.sweep, "kind": KINDS.get(r.kind, r.kind), "pp_init": r.pp_init,
                        "rolled_back": r.rolled_back, "resid": r.resid,
                        "max_rel_step": r.max_rel_step, "max_rel_dAp": r.max_rel_dAp,
                        "v_share": r.v_share, "ms": r.ms, "p_cur": r.p_cur, "p_new": r.p_new,
                        "decided_by": r.decided_by})
        return out

    def policy_features(self):
        """cp_policy_features: (current-operator features, rebuilt-operator features), 8 each."""
        f = (ctypes.c_float * 16)()
        self._ck(self._L.cp_policy_features(self._h, f))
        a = np.array(f[:], dtype=np.float32)
        return a[:8], a[8:]

    def probe(self, follow=-1):
        """cp_pp_probe: run the three PP choices from this state, keep `follow` (-1 cheapest safe)."""
        r = ProbeRec()
        self._ck(self._L.cp_pp_probe(self._h, int(follow), ctypes.byref(r)))
        return {"feat_cur": np.array(r.feat_cur[:], np.float32), "feat_new": np.array(r.feat_new[:], np.float32),
                "r0": r.r0, "r_exact": r.r_exact, "r_cur": r.r_cur, "r_new": r.r_new,
                "ms_exact": r.ms_exact, "ms_cur": r.ms_cur, "ms_new": r.ms_new, "has_ops": r.has_ops,
                "label_cur": r.label_cur, "label_new": r.label_new, "followed": r.followed}

    def set_option(self, option, value):
        """cp_set_option: option a key of OPTIONS; value a bool, or for 'lookahead' the
        blocks per SM of the look-ahead contraction (1..8), for 'wait_limit' cycles, for
        'msdt_levels' the combined upper levels."""
        v = int(value) if not isinstance(value, bool) else (1 if value else 0)
        if option == "lookahead" and value is True:
            v = 3
        self._ck(self._L.cp_set_option(self._h, OPTIONS[option], v))

    def stats(self):
        s = Stats()
        self._ck(self._L.cp_get_stats(self._h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in Stats._fields_}


def resid_noalloc(T, factors, out, stream=None):
    """cp_resid_noalloc: out[0] = ||T - [[A]]||^2, out[1] = ||T||^2 (no device allocation).

    T: contiguous float32 CUDA tensor; factors: float32 CUDA tensors (s_n x R);
    out: float64 CUDA tensor with 2 elements.  Enqueued on `stream` (default: the
    current torch stream); does not synchronise.
    """
    L = lib()
    N = T.dim()
    R = int(factors[0].shape[1])
    dims = (ctypes.c_int64 * N)(*[int(d) for d in T.shape])
    ptrs = (ctypes.c_void_p * N)(*[f.data_ptr() for f in factors])
    st = L.cp_resid_noalloc(N, dims, R, _dptr(T), ptrs, _dptr(out), _stream_ptr(stream))
    if st != 0:
        raise CPError(st, "cp_resid_noalloc failed")


class Policy:
    """The learned PP-regime scorer (FP32 MLP 8 -> 64 -> 64 -> 1) on the device."""

    def __init__(self, theta, stream=None):
        import torch
        self._L = lib()
        th = np.ascontiguousarray(theta, dtype=np.float32)
        if th.size != N_POLICY_PARAMS:
            raise ValueError("theta must hold 4801 parameters")
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = self._L.cp_policy_create(ctypes.byref(h), th.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                      _stream_ptr(self._stream))
        if st != 0:
            raise CPError(st, "cp_policy_create failed")
        self._h = h

    def _ck(self, st):
        if st != 0:
            raise CPError(st, "policy call failed")

    def get(self):
        out = np.empty(N_POLICY_PARAMS, dtype=np.float32)
        self._ck(self._L.cp_policy_get(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def forward(self, X):
        import torch
        X = X.contiguous()
        out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        self._ck(self._L.cp_policy_forward(self._h, _dptr(X), int(X.shape[0]), _dptr(out)))
        return out

    def grad(self, X, y):
        import torch
        X, y = X.contiguous(), y.contiguous()
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        g = torch.empty(N_POLICY_PARAMS, dtype=torch.float32, device=X.device)
        self._ck(self._L.cp_policy_grad(self._h, _dptr(X), _dptr(y), int(X.shape[0]), _dptr(loss), _dptr(g)))
        return loss, g

    def train(self, X, y, steps, lr=1e-3):
        X, y = X.contiguous(), y.contiguous()
        self._ck(self._L.cp_policy_train(self._h, _dptr(X), _dptr(y), int(X.shape[0]), int(steps), float(lr)))

    def close(self):
        if getattr(self, "_h", None):
            self._L.cp_policy_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
