"""ctypes binding of libgw_fgc.so (argument marshalling only).

The functions here carry the C entry points' names and arguments; every step
of the computation runs inside the CUDA library.  Loading fails loudly when
the library has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB_PATH = os.path.join(PKG, "libgw_fgc.so")
HEADER = os.path.join(ROOT, "include", "gw.h")

# gw_status
GW_OK = 0
GW_NOT_READY = 1
GW_ERR_INVALID = -1
GW_ERR_OOM = -2
GW_ERR_CUDA = -3
GW_ERR_TIMEOUT = -4
GW_ERR_NONFINITE = -5
GW_ERR_SHUTDOWN = -6
STATUS_NAMES = {0: "GW_OK", 1: "GW_NOT_READY", -1: "GW_ERR_INVALID", -2: "GW_ERR_OOM", -3: "GW_ERR_CUDA",
                -4: "GW_ERR_TIMEOUT", -5: "GW_ERR_NONFINITE", -6: "GW_ERR_SHUTDOWN"}
# gw_dtype
GW_F32 = 0
GW_F64 = 1
# gw_cost
GW_COST_POW = 0
GW_COST_SQEUCLID = 1
# gw_dense_precision
GW_DENSE_FP32 = 0
GW_DENSE_TF32 = 1
GW_DENSE_BF16 = 2
GW_DENSE_FP64 = 3
GW_DENSE_TC_TF32 = 4
GW_DENSE_TC_BF16 = 5
# gw_marginals
GW_MARG_TARGET = 0
GW_MARG_EXACT = 1


class gw_problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("hx", ctypes.c_double),
        ("hy", ctypes.c_double),
        ("k", ctypes.c_int),
        ("cost", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("n_outer", ctypes.c_int),
        ("n_inner", ctypes.c_int),
        ("theta", ctypes.c_double),
        ("feat_dim", ctypes.c_int),
        ("dtype", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("warm_start", ctypes.c_int),
        ("rho", ctypes.c_double),
        ("ky", ctypes.c_int),
    ]


class gw_barycenter_problem(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int),
        ("N", ctypes.c_int),
        ("k", ctypes.c_int),
        ("dtype", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("n_iter", ctypes.c_int),
        ("n_outer", ctypes.c_int),
        ("n_inner", ctypes.c_int),
    ]


class GWError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load() -> ctypes.CDLL:
    """Loads libgw_fgc.so (build it with paper_2404_08970_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -m paper_2404_08970_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    S = ctypes.c_int  # gw_status
    prob = ctypes.POINTER(gw_problem)
    sigs = {
        "gw_ctx_create": (S, [ctypes.POINTER(P), I]),
        "gw_ctx_destroy": (None, [P]),
        "gw_last_error": (ctypes.c_char_p, [P]),
        "gw_ctx_check": (S, [P, P]),
        "gw_ctx_profile": (S, [P, I]),
        "gw_ctx_profile_report": (S, [P, ctypes.c_char_p, ctypes.c_size_t, I]),
        "gw_grad": (S, [P, prob, P, P, P, P, I, P]),
        "gw_solve": (S, [P, prob, P, P, P, P, P, P, P, P, P]),
        "gw_grad_dense": (S, [P, prob, P, P, P, P, I, I, P]),
        "gw_grad_noalloc": (S, [prob, P, P, P, P, I, P]),
        "gw_grad_host": (S, [P, prob, P, P, P, P, I, P]),
        "gw_solve_batch": (S, [P, I, prob, P, P, P, P, P, P, P]),
        "gw_barycenter": (S, [P, ctypes.POINTER(gw_barycenter_problem), P, P, P, P, P, P, P, P]),
        "gw_server_create": (S, [ctypes.POINTER(P), I, ctypes.c_size_t, I]),
        "gw_server_destroy": (None, [P]),
        "gw_submit": (S, [P, prob, P, P, P, P, P, ctypes.POINTER(ctypes.c_uint64)]),
        "gw_poll": (S, [P, ctypes.c_uint64, P, ctypes.POINTER(ctypes.c_double)]),
        "gw_server_info": (S, [P, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long),
                               ctypes.POINTER(ctypes.c_size_t)]),
        "gw_server_last_error": (ctypes.c_char_p, [P]),
        "gw_tune_set": (S, [I, I, I, I, I]),
        "gw_tune_clear": (S, []),
        "gw_tune_load": (S, [ctypes.c_char_p]),
        "gw_tune_config": (I, [I, I, I]),
        "gw_tune_candidates": (I, [I, I, I, ctypes.POINTER(I), I]),
        "gw_tune_shape": (S, [I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


# gw_tune_kernel
GW_TUNE_SINKHORN = 0


def _tune_check(st: int, what: str) -> None:
    if st != GW_OK:
        raise GWError(st, what)


def gw_tune_set(kernel: int, dtype: int, m_lo: int, m_hi: int, config: int) -> None:
    """Table entry: rows of m_lo..m_hi columns of `dtype` use `config`."""
    _tune_check(load().gw_tune_set(kernel, dtype, m_lo, m_hi, config),
                f"gw_tune_set({kernel}, {dtype}, {m_lo}, {m_hi}, {config})")


def gw_tune_clear() -> None:
    _tune_check(load().gw_tune_clear(), "gw_tune_clear")


def gw_tune_load(path: str) -> None:
    _tune_check(load().gw_tune_load(os.fsencode(path)), f"gw_tune_load({path})")


def gw_tune_config(kernel: int, dtype: int, m: int) -> int:
    """Configuration in effect for rows of m columns (-1: invalid arguments)."""
    return load().gw_tune_config(kernel, dtype, m)


def gw_tune_candidates(kernel: int, dtype: int, m: int) -> list[int]:
    """Candidate configurations for rows of m columns, built-in choice first."""
    lib = load()
    count = lib.gw_tune_candidates(kernel, dtype, m, None, 0)
    if count < 0:
        raise GWError(GW_ERR_INVALID, f"gw_tune_candidates({kernel}, {dtype}, {m})")
    buf = (ctypes.c_int * max(1, count))()
    lib.gw_tune_candidates(kernel, dtype, m, buf, count)
    return list(buf[:count])


def gw_tune_shape(kernel: int, config: int) -> tuple[int, int, int]:
    """(warps per row group, values per thread, row groups per block)."""
    nw, vpt, ng = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _tune_check(load().gw_tune_shape(kernel, config, ctypes.byref(nw), ctypes.byref(vpt), ctypes.byref(ng)),
                f"gw_tune_shape({kernel}, {config})")
    return nw.value, vpt.value, ng.value


def declared_functions() -> list[str]:
    """Names of the functions include/gw.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gw_[a-z0-9_]+)\s*\(", text)))


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def gw_grad_noalloc(prob: gw_problem, u, v, T, G, marginals=GW_MARG_TARGET, stream=None) -> int:
    """gw_grad without device allocation (fixed static scratch; see include/gw.h)."""
    lib = load()
    st = lib.gw_grad_noalloc(ctypes.byref(prob), _ptr(u), _ptr(v), _ptr(T), _ptr(G), marginals, _stream(stream))
    if st < 0:
        raise GWError(st, "gw_grad_noalloc")
    return st


def problem(dim=1, nx=1, ny=1, hx=1.0, hy=1.0, k=1, cost=GW_COST_POW, eps=1e-2, n_outer=1, n_inner=1,
            theta=1.0, feat_dim=0, dtype=GW_F32, tau=0.0, warm_start=0, rho=0.0, ky=0) -> gw_problem:
    return gw_problem(dim, nx, ny, hx, hy, k, cost, eps, n_outer, n_inner, theta, feat_dim, dtype, tau,
                      warm_start, rho, ky)


class Context:
    """Owns a gw_ctx*.  Methods mirror the C entry points."""

    def __init__(self, device: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        st = lib.gw_ctx_create(ctypes.byref(h), device)
        if st != GW_OK:
            raise GWError(st, f"gw_ctx_create(device={device}) failed")
        self.h = h
        self.lib = lib

    def close(self):
        if getattr(self, "h", None):
            self.lib.gw_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self.lib.gw_last_error(self.h).decode()

    def _check(self, st: int, what: str) -> int:
        if st < 0:
            raise GWError(st, f"{what}: {self.last_error()}")
        return st

    def gw_ctx_check(self, stream=None) -> int:
        return self._check(self.lib.gw_ctx_check(self.h, _stream(stream)), "gw_ctx_check")

    def gw_ctx_profile(self, enable: bool) -> int:
        return self._check(self.lib.gw_ctx_profile(self.h, int(enable)), "gw_ctx_profile")

    def gw_ctx_profile_report(self, reset: bool = True) -> dict:
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(self.lib.gw_ctx_profile_report(self.h, buf, len(buf), int(reset)), "gw_ctx_profile_report")
        return json.loads(buf.value.decode())

    def gw_grad(self, prob: gw_problem, u, v, T, G, marginals=GW_MARG_TARGET, stream=None) -> int:
        st = self.lib.gw_grad(self.h, ctypes.byref(prob), _ptr(u), _ptr(v), _ptr(T), _ptr(G), marginals,
                              _stream(stream))
        return self._check(st, "gw_grad")

    def gw_grad_host(self, prob: gw_problem, u, v, T, G, marginals=GW_MARG_TARGET, stream=None) -> int:
        """u, v, T, G: host arrays (numpy, or CPU tensors, preferably pinned);
        G is ready once `stream` is synchronised."""
        st = self.lib.gw_grad_host(self.h, ctypes.byref(prob), _host_ptr(u), _host_ptr(v), _host_ptr(T),
                                   _host_ptr(G), marginals, _stream(stream))
        return self._check(st, "gw_grad_host")

    def gw_solve(self, prob: gw_problem, u, v, T, f=None, g=None, stats=None, phi=None, psi=None,
                 stream=None) -> int:
        st = self.lib.gw_solve(self.h, ctypes.byref(prob), _ptr(u), _ptr(v), _ptr(phi), _ptr(psi), _ptr(T),
                               _ptr(f), _ptr(g), _ptr(stats), _stream(stream))
        return self._check(st, "gw_solve")

    def gw_solve_batch(self, probs, u, v, T, stats=None, phi=None, psi=None, stream=None) -> int:
        """probs: list of gw_problem; u, v, T (and optionally stats, phi,
        psi): lists of device tensors (entries may be None where allowed)."""
        cnt = len(probs)
        arr = (gw_problem * cnt)(*probs)

        def ptrs(xs):
            if xs is None:
                return None
            return (ctypes.c_void_p * cnt)(*[_ptr(x) for x in xs])

        keep = [ptrs(u), ptrs(v), ptrs(phi), ptrs(psi), ptrs(T), ptrs(stats)]
        st = self.lib.gw_solve_batch(self.h, cnt, arr, *[ctypes.cast(k, ctypes.c_void_p) if k is not None else None
                                                         for k in keep], _stream(stream))
        return self._check(st, "gw_solve_batch")

    def gw_barycenter(self, prob: gw_barycenter_problem, n, h, lambdas, ps, p, C, stats=None, stream=None) -> int:
        """n, h, lambdas: sequences of prob.count host values; ps: device
        tensors (the inputs' marginals); p: device tensor (N); C: device
        N x N tensor (in: initial distances, out: the barycenter's)."""
        cnt = len(n)
        n_arr = (ctypes.c_int * cnt)(*[int(x) for x in n])
        h_arr = (ctypes.c_double * cnt)(*[float(x) for x in h])
        l_arr = (ctypes.c_double * cnt)(*[float(x) for x in lambdas])
        p_arr = (ctypes.c_void_p * cnt)(*[_ptr(x) for x in ps])
        st = self.lib.gw_barycenter(self.h, ctypes.byref(prob), ctypes.cast(n_arr, ctypes.c_void_p),
                                    ctypes.cast(h_arr, ctypes.c_void_p), ctypes.cast(l_arr, ctypes.c_void_p),
                                    ctypes.cast(p_arr, ctypes.c_void_p), _ptr(p), _ptr(C), _ptr(stats),
                                    _stream(stream))
        return self._check(st, "gw_barycenter")

    def gw_grad_dense(self, prob: gw_problem, u, v, T, G, marginals=GW_MARG_TARGET, precision=GW_DENSE_BF16,
                      stream=None) -> int:
        st = self.lib.gw_grad_dense(self.h, ctypes.byref(prob), _ptr(u), _ptr(v), _ptr(T), _ptr(G), marginals,
                                    precision, _stream(stream))
        return self._check(st, "gw_grad_dense")


def _host_ptr(a):
    """Address of a C-contiguous numpy array or CPU tensor (or None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("host tensors must be contiguous CPU tensors")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host arrays must be C-contiguous")
    return a.ctypes.data


class Server:
    """Owns a gw_server*: submit/poll of independent solves (host arrays)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 40 << 30, max_slots: int = 8):
        lib = load()
        h = ctypes.c_void_p()
        st = lib.gw_server_create(ctypes.byref(h), device, hbm_budget_bytes, max_slots)
        if st != GW_OK:
            raise GWError(st, "gw_server_create failed")
        self.h = h
        self.lib = lib
        self._keep = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.gw_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, prob: gw_problem, u, v, phi=None, psi=None, T_out=None) -> int:
        """u, v (and phi, psi) float64 numpy arrays; T_out an optional numpy
        array of n*m reals of the problem's dtype that receives the plan."""
        t = ctypes.c_uint64()
        st = self.lib.gw_submit(self.h, ctypes.byref(prob), _host_ptr(u), _host_ptr(v), _host_ptr(phi),
                                _host_ptr(psi), _host_ptr(T_out), ctypes.byref(t))
        if st != GW_OK:
            raise GWError(st, "gw_submit")
        if T_out is not None:
            self._keep[t.value] = T_out
        return t.value

    def poll(self, ticket: int):
        """None while not finished; else (status, stats (8 floats), latency_s)."""
        stats = (ctypes.c_double * 8)()
        lat = ctypes.c_double()
        st = self.lib.gw_poll(self.h, ticket, ctypes.cast(stats, ctypes.c_void_p), ctypes.byref(lat))
        if st == GW_NOT_READY:
            return None
        self._keep.pop(ticket, None)
        if st == GW_ERR_INVALID:
            raise GWError(st, f"gw_poll: unknown or already reported ticket {ticket}")
        return st, list(stats), lat.value

    def last_error(self) -> str:
        return self.lib.gw_server_last_error(self.h).decode()

    def info(self):
        q, c, b = ctypes.c_long(), ctypes.c_long(), ctypes.c_size_t()
        self.lib.gw_server_info(self.h, ctypes.byref(q), ctypes.byref(c), ctypes.byref(b))
        return q.value, c.value, b.value
