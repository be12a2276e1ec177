"""ctypes wrapper of the plain-C oracle in ``csrc/oracle_hw.c`` (test infrastructure only).

``build()`` compiles it with gcc (-O2, OpenMP) into ``oracle/_build/``; the other
functions take canonical numpy arrays (see ``synthetic``) and return numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "csrc" / "oracle_hw.c"
_OUT = _HERE / "_build" / "liboracle_hw.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile the C oracle (seconds).  Returns the path of the shared library."""
    if _OUT.exists() and not force and _OUT.stat().st_mtime >= _SRC.stat().st_mtime:
        return _OUT
    _OUT.parent.mkdir(exist_ok=True)
    tmp = _OUT.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", str(_SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_hw_apply.argtypes = [dp, dp, dp, ip, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.oracle_cgnr.argtypes = [dp, dp, ip, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    dp, ip, dp]
        lib.oracle_sign_apply.argtypes = [dp, dp, ip, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, dp, dp, ip, dp]
        lib.oracle_sign_apply_many.argtypes = [dp, dp, ip, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, ip, dp]
        for f in (lib.oracle_hw_apply, lib.oracle_cgnr, lib.oracle_sign_apply, lib.oracle_sign_apply_many):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(U):
    lt, lz, ly, lx = U.shape[1:5]
    return (ctypes.c_int * 4)(lx, ly, lz, lt)


def hw_apply(U, psi, m0, r=1.0, bc_t=-1):
    """H_W psi for one canonical spinor (Lt, Lz, Ly, Lx, 4, 3)."""
    lib = _load()
    U = np.ascontiguousarray(U, dtype=np.complex128)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    lib.oracle_hw_apply(_dp(U), _dp(psi), _dp(out), _dims(U), m0, r, int(bc_t))
    return out


def sign_apply(U, b, z, c, c0, m0, r=1.0, bc_t=-1, tol=1e-13, maxiter=200000, keep_nodes=False, strict=True):
    """S_N b = c0 b + sum_j c_j (z_j - H_W)^-1 b with one CGNR solve per node (OpenMP).

    Returns (out, iterations per node, true relative residual per node[, y_j]).  With
    strict=False a node that reaches maxiter is not an error: its iterate after maxiter
    steps enters the sum and its true residual is reported (bounded timing samples)."""
    lib = _load()
    U = np.ascontiguousarray(U, dtype=np.complex128)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    z = np.ascontiguousarray(z, dtype=np.complex128)
    c = np.ascontiguousarray(c, dtype=np.complex128)
    n = len(z)
    out = np.empty_like(b)
    ys = np.empty((n,) + b.shape, dtype=np.complex128) if keep_nodes else None
    iters = (ctypes.c_int * n)()
    res = np.zeros(n)
    c0 = complex(c0)
    rc = lib.oracle_sign_apply(_dp(U), _dp(b), _dims(U), m0, r, int(bc_t), n, _dp(z), _dp(c),
                               c0.real, c0.imag, tol, maxiter, _dp(out),
                               _dp(ys) if ys is not None else None, iters, _dp(res))
    if rc and strict:
        raise RuntimeError("C oracle: a node did not converge")
    if keep_nodes:
        return out, np.array(iters[:]), res, ys
    return out, np.array(iters[:]), res


def sign_apply_many(U, B, z, c, c0, m0, r=1.0, bc_t=-1, tol=1e-13, maxiter=200000):
    """S_N b_r for every source b_r of B (nsrc canonical spinors), one CGNR solve per
    (source, node) pair, OpenMP over all pairs.  Returns (out, iterations[nsrc, n],
    true relative residuals[nsrc, n])."""
    lib = _load()
    U = np.ascontiguousarray(U, dtype=np.complex128)
    B = np.ascontiguousarray(B, dtype=np.complex128)
    z = np.ascontiguousarray(z, dtype=np.complex128)
    c = np.ascontiguousarray(c, dtype=np.complex128)
    nsrc, n = B.shape[0], len(z)
    out = np.empty_like(B)
    iters = (ctypes.c_int * (nsrc * n))()
    res = np.zeros(nsrc * n)
    c0 = complex(c0)
    rc = lib.oracle_sign_apply_many(_dp(U), _dp(B), _dims(U), m0, r, int(bc_t), nsrc, n, _dp(z), _dp(c),
                                    c0.real, c0.imag, tol, maxiter, _dp(out), iters, _dp(res))
    if rc:
        raise RuntimeError("C oracle: a solve did not converge")
    return out, np.array(iters[:]).reshape(nsrc, n), res.reshape(nsrc, n)
