"""CPU oracle for exact dense Z[y] multiplication -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the oracle legs of ``bench.py``
may import this package.  The CUDA library and its Python binding never
import it; the two share no code.

The oracle is the plain definition c_k = sum_{i+j=k} a_i b_j over Z (§1 and
§2 of arXiv 1612.05778), computed by ``ipm_oracle.c`` with its own bigint
(schoolbook limb products into signed accumulators); for full outputs at
large sizes the same c is read off the integer product a(2^s) b(2^s)
(Kronecker substitution) done with the oracle's own Karatsuba.  ``build()`` compiles it
with gcc into ``liboracle.so`` next to this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ipm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, pthreads) and return the .so path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int32
            lib.orc_polymul_mut.argtypes = [i64, i32, P, P, i64, i32, P, P, i32, P, P, i32,
                                            ctypes.c_int]
            lib.orc_polymul_mut.restype = ctypes.c_int
            lib.orc_coeffs.argtypes = [i64, P, i64, i32, P, P, i64, i32, P, P, i32, P, P, i32]
            lib.orc_coeffs.restype = ctypes.c_int
            lib.orc_polymul_kron.argtypes = [i64, i32, P, P, i64, i32, P, P, i32, P, P, i32]
            lib.orc_polymul_kron.restype = ctypes.c_int
            lib.orc_kara_mul.argtypes = [i64, P, P, P, i32]
            lib.orc_kara_mul.restype = ctypes.c_int
            lib.orc_eval_mod.argtypes = [i64, i32, P, P, ctypes.c_uint64, ctypes.c_uint64]
            lib.orc_eval_mod.restype = ctypes.c_uint64
            _lib = lib
    return _lib


def _ptr(x: np.ndarray):
    return x.ctypes.data_as(ctypes.c_void_p)


def _prep(limbs, neg):
    limbs = np.ascontiguousarray(limbs, dtype=np.uint32)
    neg = np.ascontiguousarray(neg, dtype=np.uint8)
    if limbs.ndim != 2 or neg.shape != (limbs.shape[0],):
        raise ValueError("operand must be (n, L) limbs with (n,) signs")
    return limbs, neg


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def polymul(a, b, lc: int, threads: int | None = None, mutation: int = 0):
    """Full product c = a*b; returns (limbs (na+nb-1, lc) u32, neg u8)."""
    (al, an), (bl, bn) = _prep(*a), _prep(*b)
    na, la = al.shape
    nb, lb = bl.shape
    nc = na + nb - 1
    c = np.zeros((nc, lc), dtype=np.uint32)
    cn = np.zeros(nc, dtype=np.uint8)
    st = _load().orc_polymul_mut(na, la, _ptr(al), _ptr(an), nb, lb, _ptr(bl), _ptr(bn),
                                 lc, _ptr(c), _ptr(cn), threads or default_threads(), mutation)
    if st != 0:
        raise RuntimeError("oracle polymul failed with status %d" % st)
    return c, cn


def polymul_kron(a, b, lc: int, threads: int | None = None):
    """Full product c = a*b by Kronecker substitution (a(2^s) b(2^s), slots
    of s = 32 (lc + 1) bits) and the oracle's own threaded Karatsuba; the
    same result as polymul, for sizes where the schoolbook is out of
    reach.  Returns (limbs (na+nb-1, lc) u32, neg u8)."""
    (al, an), (bl, bn) = _prep(*a), _prep(*b)
    na, la = al.shape
    nb, lb = bl.shape
    nc = na + nb - 1
    c = np.zeros((nc, lc), dtype=np.uint32)
    cn = np.zeros(nc, dtype=np.uint8)
    st = _load().orc_polymul_kron(na, la, _ptr(al), _ptr(an), nb, lb, _ptr(bl), _ptr(bn),
                                  lc, _ptr(c), _ptr(cn), threads or default_threads())
    if st != 0:
        raise RuntimeError("oracle polymul_kron failed with status %d" % st)
    return c, cn


def kara_mul(x: int, y: int, threads: int = 1) -> int:
    """x * y for non-negative Python integers through the oracle's
    Karatsuba (the integer product inside polymul_kron)."""
    n = max(x.bit_length(), y.bit_length(), 1)
    n32 = (n + 31) // 32
    n32 += n32 & 1
    xa = np.frombuffer(x.to_bytes(4 * n32, "little"), dtype=np.uint32).copy()
    ya = np.frombuffer(y.to_bytes(4 * n32, "little"), dtype=np.uint32).copy()
    r = np.zeros(2 * n32, dtype=np.uint32)
    st = _load().orc_kara_mul(n32, _ptr(xa), _ptr(ya), _ptr(r), threads)
    if st != 0:
        raise RuntimeError("oracle kara_mul failed with status %d" % st)
    return int.from_bytes(r.tobytes(), "little")


def coeffs(ks, a, b, lc: int, threads: int | None = None):
    """Selected coefficients c_k for k in ks; returns (limbs (len(ks), lc), neg)."""
    (al, an), (bl, bn) = _prep(*a), _prep(*b)
    ks = np.ascontiguousarray(ks, dtype=np.int64)
    na, la = al.shape
    nb, lb = bl.shape
    c = np.zeros((len(ks), lc), dtype=np.uint32)
    cn = np.zeros(len(ks), dtype=np.uint8)
    st = _load().orc_coeffs(len(ks), _ptr(ks), na, la, _ptr(al), _ptr(an), nb, lb, _ptr(bl),
                            _ptr(bn), lc, _ptr(c), _ptr(cn), threads or default_threads())
    if st != 0:
        raise RuntimeError("oracle coeffs failed with status %d" % st)
    return c, cn


def eval_mod(x, t: int, q: int) -> int:
    """sum_k x_k t^k mod q for the sign-magnitude operand x (q < 2**62)."""
    xl, xn = _prep(*x)
    n, l = xl.shape
    return int(_load().orc_eval_mod(n, l, _ptr(xl), _ptr(xn), t % q, q))
