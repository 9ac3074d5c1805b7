"""Exact dense Z[y] multiplication on GB300 (arXiv 1612.05778, CVL_p^2 form).

A thin ctypes binding over the C ABI of ``include/ipm.h`` (``libipm.so``,
built in-tree by ``paper_1612_05778_gb300.build``).  It only marshals
arguments: every step of a product runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  There is no CPU fallback: if
the library is missing, importing the binding's entry points raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libipm.so")

IPM_SYNC = 1
IPM_COSTMODEL = 2
IPM_GRAPH = 4
IPM_TENSOR_STAGES = 8  # radix-16 stages on the INT8 tensor cores (see include/ipm.h)
IPM_VALIDATE = 16      # every single product checked at a random point mod 2^61 - 1
IPM_PERSISTENT = 32    # batched calls as one persistent launch over a device work queue

STATUS = {0: "IPM_OK", 1: "IPM_ERR_ARG", 2: "IPM_ERR_BOUND", 3: "IPM_ERR_NOMEM",
          4: "IPM_ERR_CUDA", 5: "IPM_ERR_TIMEOUT", 6: "IPM_ERR_UNSUPPORTED", 7: "IPM_ERR_MISMATCH"}


class IpmError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s failed: %s (%d)" % (what, STATUS.get(status, "?"), status))
        self.status = status


class Shape(ctypes.Structure):
    _fields_ = [("deg_a", ctypes.c_int64), ("deg_b", ctypes.c_int64),
                ("bits_a", ctypes.c_uint32), ("bits_b", ctypes.c_uint32)]


class Params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("M", ctypes.c_int32), ("r", ctypes.c_int32),
                ("y2", ctypes.c_int32), ("s", ctypes.c_int32), ("y1b", ctypes.c_int32),
                ("kron", ctypes.c_int32), ("school", ctypes.c_int32), ("ks", ctypes.c_int32),
                ("kara", ctypes.c_int32), ("bigp", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("na", ctypes.c_int64), ("nb", ctypes.c_int64), ("nc", ctypes.c_int64),
                ("la", ctypes.c_int32), ("lb", ctypes.c_int32), ("lc", ctypes.c_int32),
                ("K", ctypes.c_int32), ("M", ctypes.c_int32), ("N", ctypes.c_int32),
                ("r", ctypes.c_int32), ("Y", ctypes.c_int64), ("Y1", ctypes.c_int64),
                ("Y2", ctypes.c_int64), ("S", ctypes.c_int32), ("Y1b", ctypes.c_int64),
                ("primes", ctypes.c_uint32 * 8),
                ("log2_modulus", ctypes.c_double), ("log2_bound", ctypes.c_double),
                ("workspace_bytes", ctypes.c_size_t), ("kron", ctypes.c_int32),
                ("kron_w", ctypes.c_int32), ("kron_na", ctypes.c_int64), ("kron_nb", ctypes.c_int64),
                ("kron_bits_a", ctypes.c_uint32), ("kron_bits_b", ctypes.c_uint32),
                ("school", ctypes.c_int32), ("ks", ctypes.c_int32), ("ks_w", ctypes.c_int32),
                ("kara", ctypes.c_int32), ("bigp", ctypes.c_int32)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "primes"}
        d["primes"] = [int(self.primes[i]) for i in range(self.r)]
        return d


FEATURES = 19
MLP_HIDDEN = 32
MLP_PARAMS = MLP_HIDDEN * FEATURES + MLP_HIDDEN * MLP_HIDDEN + 3 * MLP_HIDDEN + 1
MLP_FLOATS = 2 * FEATURES + 2 + MLP_PARAMS


class Candidate(ctypes.Structure):
    _fields_ = [("params", Params), ("info", PlanInfo), ("features", ctypes.c_float * FEATURES)]


class Operands(ctypes.Structure):
    _fields_ = [("a", ctypes.c_void_p), ("a_neg", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("b_neg", ctypes.c_void_p), ("c", ctypes.c_void_p), ("c_neg", ctypes.c_void_p)]


_lib = None


def load_library(path: str | None = None):
    """Load libipm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libipm.so is missing (%s): run paper_1612_05778_gb300.build.build()" % p)
    lib = ctypes.CDLL(p)
    V, I32, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32
    lib.ipm_choose.argtypes = [ctypes.POINTER(Shape), ctypes.POINTER(Params), ctypes.POINTER(PlanInfo)]
    lib.ipm_plan.argtypes = [ctypes.POINTER(V), ctypes.POINTER(Shape), I32, U32]
    lib.ipm_plan_ex.argtypes = [ctypes.POINTER(V), ctypes.POINTER(Shape), I32, U32, ctypes.POINTER(Params)]
    lib.ipm_get_info.argtypes = [V, I32, ctypes.POINTER(PlanInfo)]
    lib.ipm_mul.argtypes = [V, V, V, V, V, V, V, V]
    lib.ipm_mul_host.argtypes = [V, V, V, V, V, V, V, V]
    lib.ipm_mul_host_async.argtypes = [V, V, V, V, V, V, V, V]
    lib.ipm_mul_batched.argtypes = [V, ctypes.POINTER(Operands), I32, V]
    lib.ipm_sync.argtypes = [V, V]
    lib.ipm_set_wait_limit.argtypes = [V, ctypes.c_uint64]
    lib.ipm_debug_hold.argtypes = [V, I32]
    lib.ipm_destroy.argtypes = [V]
    lib.ipm_set_profiling.argtypes = [V, I32]
    lib.ipm_phase_ms.argtypes = [V, ctypes.POINTER(ctypes.c_float), I32]
    lib.ipm_mul_noalloc.argtypes = [ctypes.POINTER(Shape), V, V, V, V, V, V, V]
    lib.ipm_candidates.argtypes = [ctypes.POINTER(Shape), ctypes.POINTER(Candidate), I32]
    lib.ipm_candidates.restype = I32
    F32P = ctypes.POINTER(ctypes.c_float)
    lib.ipm_mlp_train.argtypes = [F32P, F32P, I32, I32, ctypes.c_float, ctypes.c_uint64, F32P, F32P]
    lib.ipm_mlp_grad.argtypes = [F32P, F32P, F32P, I32, F32P, F32P]
    lib.ipm_mlp_predict.argtypes = [F32P, F32P, I32, F32P]
    lib.ipm_set_cost_model.argtypes = [F32P, I32]
    lib.ipm_set_tuned.argtypes = [ctypes.POINTER(Shape), ctypes.POINTER(Params), I32]
    lib.ipm_dispatch.argtypes = [ctypes.POINTER(Shape), ctypes.POINTER(Params), ctypes.POINTER(I32)]
    lib.ipm_validate.argtypes = [ctypes.POINTER(Shape), V, V, V, V, V, V, ctypes.c_uint64, V]
    lib.ipm_taylor_plan.argtypes = [ctypes.POINTER(V), ctypes.c_int64, U32, U32]
    lib.ipm_taylor_limbs.argtypes = [V, ctypes.POINTER(I32)]
    lib.ipm_taylor_shift.argtypes = [V, V, V, V, V, V]
    lib.ipm_taylor_sync.argtypes = [V, V]
    lib.ipm_taylor_destroy.argtypes = [V]
    lib.ipm_strerror.argtypes = [ctypes.c_int]
    lib.ipm_strerror.restype = ctypes.c_char_p
    lib.ipm_launch_count.restype = ctypes.c_int64
    for name in ("ipm_choose", "ipm_plan", "ipm_plan_ex", "ipm_get_info", "ipm_mul", "ipm_mul_host",
                 "ipm_mul_host_async",
                 "ipm_mul_batched", "ipm_sync", "ipm_destroy", "ipm_set_profiling", "ipm_phase_ms",
                 "ipm_mul_noalloc", "ipm_mlp_train", "ipm_mlp_grad", "ipm_mlp_predict",
                 "ipm_set_cost_model", "ipm_set_tuned", "ipm_dispatch", "ipm_validate", "ipm_taylor_plan", "ipm_taylor_limbs",
                 "ipm_taylor_shift", "ipm_taylor_sync", "ipm_taylor_destroy"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(st: int, what: str):
    if st != 0:
        raise IpmError(st, what)


def _params(K=0, M=0, r=0, y2=0, s=0, y1b=0, kron=0, school=0, ks=0, kara=0, bigp=0):
    if not (K or M or r or y2 or s or y1b or kron or school or ks or kara or bigp):
        return None
    return Params(K, M, r, y2, s, y1b, kron, school, ks, kara, bigp)


def choose(na: int, nb: int, bits_a: int, bits_b: int, **overrides) -> dict:
    """Host-only planner query (no GPU): the plan ipm_plan would build."""
    lib = load_library()
    info = PlanInfo()
    prm = _params(**overrides)
    _check(lib.ipm_choose(ctypes.byref(Shape(na - 1, nb - 1, bits_a, bits_b)),
                          ctypes.byref(prm) if prm else None, ctypes.byref(info)), "ipm_choose")
    return info.as_dict()


def candidates(na: int, nb: int, bits_a: int, bits_b: int):
    """Candidate plans of a shape (host only): list of dicts with the override
    set ('params'), the resulting plan ('info') and the cost-model features."""
    lib = load_library()
    shape = Shape(na - 1, nb - 1, bits_a, bits_b)
    n = lib.ipm_candidates(ctypes.byref(shape), None, 0)
    if n < 0:
        raise IpmError(-n, "ipm_candidates")
    arr = (Candidate * max(n, 1))()
    lib.ipm_candidates(ctypes.byref(shape), arr, n)
    out = []
    for c in arr[:n]:
        prm = {k: getattr(c.params, k) for k, _ in Params._fields_ if getattr(c.params, k)}
        out.append({"params": prm, "info": c.info.as_dict(), "features": [float(x) for x in c.features]})
    return out


def _f32(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if n is not None and a.size != n:
        raise ValueError("expected %d floats, got %d" % (n, a.size))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def mlp_train(X, y, epochs: int = 3000, lr: float = 3e-3, seed: int = 0):
    """Train the cost-model network on the GPU: returns (model, final mean loss)."""
    lib = load_library()
    X, xp = _f32(X)
    y, yp = _f32(y)
    n = int(y.size)
    if X.shape != (n, FEATURES):
        raise ValueError("X must be (n, %d)" % FEATURES)
    model = np.zeros(MLP_FLOATS, dtype=np.float32)
    loss = ctypes.c_float()
    _check(lib.ipm_mlp_train(xp, yp, n, epochs, lr, seed,
                             model.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss)),
           "ipm_mlp_train")
    return model, float(loss.value)


def mlp_grad(model, X, y):
    """(summed loss, gradient over the MLP_PARAMS parameters) from the GPU kernel."""
    lib = load_library()
    model, mp = _f32(model, MLP_FLOATS)
    X, xp = _f32(X)
    y, yp = _f32(y)
    g = np.zeros(MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    _check(lib.ipm_mlp_grad(mp, xp, yp, int(y.size), g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                            ctypes.byref(loss)), "ipm_mlp_grad")
    return float(loss.value), g


def mlp_predict(model, X):
    """Predictions of the network for the rows of X (GPU kernel)."""
    lib = load_library()
    model, mp = _f32(model, MLP_FLOATS)
    X, xp = _f32(X)
    n = X.size // FEATURES
    out = np.zeros(n, dtype=np.float32)
    _check(lib.ipm_mlp_predict(mp, xp, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
           "ipm_mlp_predict")
    return out


def set_cost_model(model):
    """Install a model for IPM_COSTMODEL plans (None uninstalls)."""
    lib = load_library()
    if model is None:
        _check(lib.ipm_set_cost_model(None, 0), "ipm_set_cost_model")
        return
    model, mp = _f32(model, MLP_FLOATS)
    _check(lib.ipm_set_cost_model(mp, MLP_FLOATS), "ipm_set_cost_model")


def set_tuned(entries):
    """Replace the tuning table: entries = [((na, nb, bits_a, bits_b), params dict), ...]."""
    lib = load_library()
    n = len(entries)
    shapes = (Shape * max(n, 1))(*[Shape(na - 1, nb - 1, ba, bb) for (na, nb, ba, bb), _ in entries])
    prms = (Params * max(n, 1))(*[Params(*(p.get(k, 0) for k, _ in Params._fields_)) for _, p in entries])
    _check(lib.ipm_set_tuned(shapes, prms, n), "ipm_set_tuned")


def dispatch(na: int, nb: int, bits_a: int, bits_b: int):
    """(params dict, source) that IPM_COSTMODEL gives a shape; source is
    'planner', 'table' or 'model'."""
    lib = load_library()
    prm = Params()
    src = ctypes.c_int32()
    _check(lib.ipm_dispatch(ctypes.byref(Shape(na - 1, nb - 1, bits_a, bits_b)), ctypes.byref(prm),
                            ctypes.byref(src)), "ipm_dispatch")
    return ({k: getattr(prm, k) for k, _ in Params._fields_ if getattr(prm, k)},
            ("planner", "table", "model")[src.value])


def launch_count() -> int:
    return int(load_library().ipm_launch_count())


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _dptr(t, dtype, shape=None):
    import torch
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor of %s" % dtype)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (shape, tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A plan for products of fixed shapes (one shape for mul, several for
    mul_batched).  Each shape is (na, nb, bits_a, bits_b) with na, nb the
    coefficient counts; limb tensors are int32 views of the uint32 limbs
    (torch has no uint32 arithmetic; the bits are what matter)."""

    def __init__(self, shapes, flags: int = 0, **overrides):
        lib = load_library()
        if isinstance(shapes, tuple):
            shapes = [shapes]
        arr = (Shape * len(shapes))(*[Shape(na - 1, nb - 1, ba, bb) for na, nb, ba, bb in shapes])
        prm = _params(**overrides)
        h = ctypes.c_void_p()
        _check(lib.ipm_plan_ex(ctypes.byref(h), arr, len(shapes), flags,
                               ctypes.byref(prm) if prm else None), "ipm_plan")
        self._h = h
        self._lib = lib
        self.shapes = list(shapes)
        self.infos = []
        for i in range(len(shapes)):
            info = PlanInfo()
            _check(lib.ipm_get_info(h, i, ctypes.byref(info)), "ipm_get_info")
            self.infos.append(info.as_dict())

    @property
    def info(self) -> dict:
        return self.infos[0]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.ipm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty_output(self, index: int = 0):
        import torch
        I = self.infos[index]
        return (torch.empty((I["nc"], I["lc"]), dtype=torch.int32, device="cuda"),
                torch.empty((I["nc"],), dtype=torch.uint8, device="cuda"))

    def mul(self, a, a_neg, b, b_neg, c=None, c_neg=None, stream=None):
        """c = a*b on the device; tensors: limbs int32 (n, L), signs uint8 (n,)."""
        import torch
        I = self.info
        if c is None or c_neg is None:
            c, c_neg = self.empty_output()
        args = [_dptr(a, torch.int32, (I["na"], I["la"])), _dptr(a_neg, torch.uint8, (I["na"],)),
                _dptr(b, torch.int32, (I["nb"], I["lb"])), _dptr(b_neg, torch.uint8, (I["nb"],)),
                _dptr(c, torch.int32, (I["nc"], I["lc"])), _dptr(c_neg, torch.uint8, (I["nc"],))]
        _check(self._lib.ipm_mul(self._h, *args, _stream_handle(stream)), "ipm_mul")
        return c, c_neg

    def mul_host(self, a: np.ndarray, a_neg: np.ndarray, b: np.ndarray, b_neg: np.ndarray,
                 c: np.ndarray | None = None, c_neg: np.ndarray | None = None, stream=None):
        """c = a*b with host (numpy) buffers; waits for the result."""
        I = self.info
        a = np.ascontiguousarray(a, dtype=np.uint32)
        b = np.ascontiguousarray(b, dtype=np.uint32)
        a_neg = np.ascontiguousarray(a_neg, dtype=np.uint8)
        b_neg = np.ascontiguousarray(b_neg, dtype=np.uint8)
        if a.shape != (I["na"], I["la"]) or b.shape != (I["nb"], I["lb"]):
            raise ValueError("operand shapes do not match the plan")
        if c is None:
            c = np.empty((I["nc"], I["lc"]), dtype=np.uint32)
        if c_neg is None:
            c_neg = np.empty((I["nc"],), dtype=np.uint8)
        P = lambda x: ctypes.c_void_p(x.ctypes.data)  # noqa: E731
        _check(self._lib.ipm_mul_host(self._h, P(a), P(a_neg), P(b), P(b_neg), P(c), P(c_neg),
                                      _stream_handle(stream)), "ipm_mul_host")
        return c, c_neg

    def mul_host_async(self, a: np.ndarray, a_neg: np.ndarray, b: np.ndarray, b_neg: np.ndarray,
                       c: np.ndarray, c_neg: np.ndarray, stream=None):
        """Enqueue c = a*b with host (numpy, preferably pinned) buffers on
        `stream` and return at once; call sync(stream) before reading c.  The
        buffers must stay alive until then."""
        I = self.info
        for x, shape, dt in ((a, (I["na"], I["la"]), np.uint32), (b, (I["nb"], I["lb"]), np.uint32),
                             (a_neg, (I["na"],), np.uint8), (b_neg, (I["nb"],), np.uint8),
                             (c, (I["nc"], I["lc"]), np.uint32), (c_neg, (I["nc"],), np.uint8)):
            if x.shape != shape or x.dtype != dt or not x.flags.c_contiguous:
                raise ValueError("host buffers must be contiguous %s arrays of shape %s" % (dt.__name__, shape))
        P = lambda x: ctypes.c_void_p(x.ctypes.data)  # noqa: E731
        _check(self._lib.ipm_mul_host_async(self._h, P(a), P(a_neg), P(b), P(b_neg), P(c), P(c_neg),
                                            _stream_handle(stream)), "ipm_mul_host_async")

    def batch_args(self, operands, outputs):
        """Validate a batch once and return its host array of device pointers
        (ipm_operands[n]), reusable by mul_batched while the tensors live."""
        import torch
        n = len(self.shapes)
        if len(operands) != n or len(outputs) != n:
            raise ValueError("need one operand set and one output per plan shape")
        arr = (Operands * n)()
        for i, ((a, an, b, bn), (c, cn)) in enumerate(zip(operands, outputs)):
            I = self.infos[i]
            arr[i] = Operands(_dptr(a, torch.int32, (I["na"], I["la"])).value,
                              _dptr(an, torch.uint8, (I["na"],)).value,
                              _dptr(b, torch.int32, (I["nb"], I["lb"])).value,
                              _dptr(bn, torch.uint8, (I["nb"],)).value,
                              _dptr(c, torch.int32, (I["nc"], I["lc"])).value,
                              _dptr(cn, torch.uint8, (I["nc"],)).value)
        return arr

    def mul_batched(self, operands, outputs=None, stream=None):
        """operands: list of (a, a_neg, b, b_neg) device tensors matching the
        plan's shapes (returns the list of (c, c_neg)), or an array made by
        batch_args (returns None)."""
        n = len(self.shapes)
        if isinstance(operands, ctypes.Array):
            if len(operands) != n:
                raise ValueError("need one operand set per plan shape")
            _check(self._lib.ipm_mul_batched(self._h, operands, n, _stream_handle(stream)), "ipm_mul_batched")
            return None
        if outputs is None:
            outputs = [self.empty_output(i) for i in range(n)]
        arr = self.batch_args(operands, outputs)
        _check(self._lib.ipm_mul_batched(self._h, arr, n, _stream_handle(stream)), "ipm_mul_batched")
        return outputs

    def set_profiling(self, enable: bool = True):
        """Record CUDA events around each of the three passes of every product."""
        _check(self._lib.ipm_set_profiling(self._h, 1 if enable else 0), "ipm_set_profiling")

    def phase_ms(self):
        """(forward, middle, inverse) pass durations of the latest product, in ms."""
        out = (ctypes.c_float * 3)()
        _check(self._lib.ipm_phase_ms(self._h, out, 3), "ipm_phase_ms")
        return [float(x) for x in out]

    def sync(self, stream=None):
        """Wait for the stream and raise on a device-side error (e.g. IPM_ERR_BOUND)."""
        _check(self._lib.ipm_sync(self._h, _stream_handle(stream)), "ipm_sync")

    def set_wait_limit(self, microseconds: int):
        """IPM_PERSISTENT plans: limit of each device-side dependency wait."""
        _check(self._lib.ipm_set_wait_limit(self._h, microseconds), "ipm_set_wait_limit")

    def debug_hold(self, product: int):
        """IPM_PERSISTENT plans, for tests of the timeout path: make product
        `product`'s later phases wait for a tile that never exists (-1:
        release)."""
        _check(self._lib.ipm_debug_hold(self._h, product), "ipm_debug_hold")


class TaylorShift:
    """g(x) = f(x + 1) for f with n coefficients below 2^bits in magnitude
    (ipm_taylor_plan / ipm_taylor_shift): g has n coefficients of `limbs`
    = ceil((bits + n) / 32) limbs."""

    def __init__(self, n: int, bits: int, flags: int = 0):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.ipm_taylor_plan(ctypes.byref(h), n - 1, bits, flags), "ipm_taylor_plan")
        self._h, self._lib, self.n, self.bits = h, lib, n, bits
        lg = ctypes.c_int32()
        _check(lib.ipm_taylor_limbs(h, ctypes.byref(lg)), "ipm_taylor_limbs")
        self.limbs = lg.value

    def shift(self, f, f_neg, g=None, g_neg=None, stream=None):
        import torch
        if g is None or g_neg is None:
            g = torch.empty((self.n, self.limbs), dtype=torch.int32, device="cuda")
            g_neg = torch.empty((self.n,), dtype=torch.uint8, device="cuda")
        args = [_dptr(f, torch.int32, (self.n, (self.bits + 31) // 32)), _dptr(f_neg, torch.uint8, (self.n,)),
                _dptr(g, torch.int32, (self.n, self.limbs)), _dptr(g_neg, torch.uint8, (self.n,))]
        _check(self._lib.ipm_taylor_shift(self._h, *args, _stream_handle(stream)), "ipm_taylor_shift")
        return g, g_neg

    def sync(self, stream=None):
        _check(self._lib.ipm_taylor_sync(self._h, _stream_handle(stream)), "ipm_taylor_sync")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.ipm_taylor_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# Size of the static device scratch of mul_noalloc (IPM_NOALLOC_SCRATCH_BYTES).
NOALLOC_SCRATCH_BYTES = 32 << 20


def output_limbs(na: int, nb: int, bits_a: int, bits_b: int) -> int:
    """Limbs per output coefficient, Lc = ceil((bits_a + bits_b +
    ceil(log2 min(na, nb))) / 32): |c_k| <= min(na, nb) (2^bits_a - 1)
    (2^bits_b - 1) < 2^(bits_a + bits_b + ceil(log2 min(na, nb))).  The
    planner uses the same formula (ipm_plan_info.lc)."""
    mn = min(na, nb)
    lg = (mn - 1).bit_length() if mn > 1 else 0  # ceil(log2 mn)
    return (bits_a + bits_b + lg + 31) // 32


def _check_free_shapes(na, nb, bits_a, bits_b, a, a_neg, b, b_neg, c, c_neg):
    """Shapes of the operands and of the output of a plan-free call, checked
    on the host before any pointer is taken or the library is called: a c
    narrower than Lc limbs would be written past its end by the kernels."""
    if na < 1 or nb < 1 or bits_a < 1 or bits_b < 1:
        raise ValueError("need na, nb >= 1 and bit bounds >= 1")
    la, lb = (bits_a + 31) // 32, (bits_b + 31) // 32
    nc, lc = na + nb - 1, output_limbs(na, nb, bits_a, bits_b)
    want = {"a": (a, (na, la)), "a_neg": (a_neg, (na,)), "b": (b, (nb, lb)), "b_neg": (b_neg, (nb,)),
            "c": (c, (nc, lc)), "c_neg": (c_neg, (nc,))}
    for name, (t, shape) in want.items():
        if tuple(t.shape) != shape:
            raise ValueError("%s must have shape %s, got %s" % (name, shape, tuple(t.shape)))
    return la, lb, nc, lc


def mul_noalloc(na: int, nb: int, bits_a: int, bits_b: int, a, a_neg, b, b_neg, c, c_neg,
                stream=None):
    """c = a*b without allocating anything, for callers that may not
    allocate device memory while they run: allocator-free or latency-bound
    services (cudaMalloc can synchronise the device) and plugins whose host
    application owns all memory and hands over only the buffers.  All
    tensors are caller-owned CUDA tensors (limbs int32 (n, L), signs uint8
    (n,)); c must be (na + nb - 1, output_limbs(...)), checked here before
    the call.  Scratch comes from one static device array shared by every
    call; calls are serialised by a host lock and each waits for its
    stream.  Raises IpmError on failure (IPM_ERR_UNSUPPORTED when the
    product's scratch exceeds the array)."""
    la, lb, nc, lc = _check_free_shapes(na, nb, bits_a, bits_b, a, a_neg, b, b_neg, c, c_neg)
    import torch
    lib = load_library()
    args = [_dptr(a, torch.int32, (na, la)), _dptr(a_neg, torch.uint8, (na,)),
            _dptr(b, torch.int32, (nb, lb)), _dptr(b_neg, torch.uint8, (nb,)),
            _dptr(c, torch.int32, (nc, lc)), _dptr(c_neg, torch.uint8, (nc,))]
    _check(lib.ipm_mul_noalloc(ctypes.byref(Shape(na - 1, nb - 1, bits_a, bits_b)), *args,
                               _stream_handle(stream)), "ipm_mul_noalloc")
    return c, c_neg


def validate(na: int, nb: int, bits_a: int, bits_b: int, a, a_neg, b, b_neg, c, c_neg, seed: int = 1,
             stream=None) -> bool:
    """ipm_validate: True when c(t) = a(t) b(t) modulo q = 2^61 - 1 at the
    point `seed` selects.  The exact product always passes.  A wrong c is
    caught with probability at least 1 - deg(c)/q whenever c - a*b is
    non-zero modulo q (any single changed limb or sign is); an error that
    is 0 modulo q is never caught.  CUDA tensors as for Plan.mul, shapes
    checked on the host first; waits."""
    la, lb, nc, lc = _check_free_shapes(na, nb, bits_a, bits_b, a, a_neg, b, b_neg, c, c_neg)
    import torch
    lib = load_library()
    args = [_dptr(a, torch.int32, (na, la)), _dptr(a_neg, torch.uint8, (na,)),
            _dptr(b, torch.int32, (nb, lb)), _dptr(b_neg, torch.uint8, (nb,)),
            _dptr(c, torch.int32, (nc, lc)), _dptr(c_neg, torch.uint8, (nc,))]
    st = lib.ipm_validate(ctypes.byref(Shape(na - 1, nb - 1, bits_a, bits_b)), *args,
                          ctypes.c_uint64(seed), _stream_handle(stream))
    if st == 7:
        return False
    _check(st, "ipm_validate")
    return True


def to_device(limbs: np.ndarray, neg: np.ndarray):
    """numpy (uint32 limbs, uint8 signs) -> CUDA tensors (int32 view, uint8)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(limbs, dtype=np.uint32).view(np.int32)).cuda()
    s = torch.from_numpy(np.ascontiguousarray(neg, dtype=np.uint8)).cuda()
    return t, s


def to_host(c, c_neg):
    """CUDA tensors -> numpy (uint32 limbs, uint8 signs)."""
    return (c.cpu().numpy().view(np.uint32), c_neg.cpu().numpy())


__all__ = ["Plan", "TaylorShift", "choose", "load_library", "launch_count", "to_device", "to_host", "IpmError",
           "IPM_SYNC", "IPM_COSTMODEL", "IPM_GRAPH", "IPM_TENSOR_STAGES", "IPM_VALIDATE", "IPM_PERSISTENT", "validate", "LIB_PATH", "mul_noalloc", "output_limbs", "NOALLOC_SCRATCH_BYTES", "candidates",
           "mlp_train", "mlp_grad", "mlp_predict", "set_cost_model", "set_tuned", "dispatch"]
