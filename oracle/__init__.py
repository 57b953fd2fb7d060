"""FP64 CPU oracle for periodic tricubic B-spline orbital evaluation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The CUDA library never links, loads or calls it, and this package imports
nothing from the CUDA library's package.

``spo_eval`` wraps ``spo_oracle.c`` (plain C, FP64, OpenMP over positions),
which writes out the textbook cubic B-spline definition: every output is the
plain 64-term window sum of weight products times coefficients (arXiv
1708.02645, Sec. 3 for the orbitals phi_i(r) in the Slater matrix and their
gradients and Laplacians needed by Alg. 1; Sec. 6.1 for the Bspline-v,
Bspline-vgh and SPO-vgl routines; Sec. 6.2 for the read-only 4-D table).

Parity status: pinned by ``tests/test_oracle_pins.py``: the evaluator by
closed forms, brute force and invariants; the condition sums ``condition``
and ``spo_ratio_condition`` (which set the per-element error bounds of the
GPU tests) by their closed forms for tables with |c| constant, a brute-force
sum of |B3 products| |c| over all images, beta_V = V for c >= 0 and
beta_ratio = ratio for non-negative rows and c.  ``tests/test_oracle_mutants.py``
plants slips in both and requires a pin to fail for each.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spo_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KIND_V, KIND_VGL, KIND_VGH = 0, 1, 2
N_COMPONENTS = {KIND_V: 1, KIND_VGL: 5, KIND_VGH: 10}


def build(force: bool = False) -> str:
    """Compile spo_oracle.c into liboracle.so next to it (gcc, -O2, OpenMP).

    -ffp-contract=off keeps every multiply and add separately rounded on both
    x86-64 and AArch64, so the oracle gives the same bits on either host.
    """
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path: str):
    lib = ctypes.CDLL(path)
    lib.oracle_spo_eval.restype = ctypes.c_int
    lib.oracle_spo_eval.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long,
        ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p, ctypes.c_int,
        ctypes.c_void_p, ctypes.c_int]
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_num_threads.argtypes = []
    lib.oracle_spo_condition.restype = ctypes.c_int
    lib.oracle_spo_condition.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long,
        ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB)
    return _lib


def load_variant(path: str):
    """Bind another build of spo_oracle.c (the tests compile deliberately
    broken copies to show that the pins catch each planted mistake)."""
    return _bind(path)


def num_threads() -> int:
    """OpenMP threads the oracle uses by default on this host."""
    return int(_load().oracle_num_threads())


def spo_eval(coefs: np.ndarray, pos: np.ndarray, kind: int = KIND_VGH,
             nthreads: int = 0, lib=None) -> np.ndarray:
    """All N orbitals (and derivatives) at P positions, in FP64.

    coefs: [nx, ny, nz, N] coefficient table (any float dtype; promoted to
           FP64 exactly).
    pos:   [P, 3] Cartesian positions on the periodic unit cube (promoted to
           FP64 exactly).
    kind:  KIND_V -> [P, N]; KIND_VGL -> [P, 5, N] (v, gx, gy, gz, lap);
           KIND_VGH -> [P, 10, N] (v, gx, gy, gz, hxx, hxy, hxz, hyy, hyz, hzz).
    """
    lib = lib if lib is not None else _load()
    c = np.ascontiguousarray(coefs, dtype=np.float64)
    if c.ndim != 4:
        raise ValueError("coefs must be [nx, ny, nz, N]")
    nx, ny, nz, N = c.shape
    r = np.ascontiguousarray(np.asarray(pos).reshape(-1, 3), dtype=np.float64)
    P = r.shape[0]
    nc = N_COMPONENTS[kind]
    out = np.empty((P, nc, N), dtype=np.float64)
    rc = lib.oracle_spo_eval(nx, ny, nz, N, c.ctypes.data, P, r.ctypes.data, kind,
                             out.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_spo_eval failed with code {rc}")
    return out[:, 0, :] if kind == KIND_V else out


def condition(coefs: np.ndarray, pos: np.ndarray, kind: int = KIND_VGH,
              nthreads: int = 0) -> np.ndarray:
    """Condition sums beta = sum |W| |c| over the window, shaped like the
    output of spo_eval for `kind`.  For the Laplacian, beta is the sum of the
    three diagonal Hessian betas.  A correctly implemented FP32 evaluation of
    the same sums errs by at most a small multiple of 2^-24 * beta."""
    lib = _load()
    c = np.ascontiguousarray(coefs, dtype=np.float64)
    nx, ny, nz, N = c.shape
    r = np.ascontiguousarray(np.asarray(pos).reshape(-1, 3), dtype=np.float64)
    P = r.shape[0]
    b = np.empty((P, 10, N), dtype=np.float64)
    rc = lib.oracle_spo_condition(nx, ny, nz, N, c.ctypes.data, P, r.ctypes.data,
                                  b.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_spo_condition failed with code {rc}")
    if kind == KIND_VGH:
        return b
    if kind == KIND_V:
        return b[:, 0, :]
    return np.concatenate([b[:, :4], (b[:, 4] + b[:, 7] + b[:, 9])[:, None]], axis=1)


def spo_ratio(coefs: np.ndarray, pos: np.ndarray, rows: np.ndarray, row_of=None) -> np.ndarray:
    """Determinant ratios rho_p = sum_j rows[r(p), j] phi_j(pos_p) in FP64.

    arXiv 1708.02645, Sec. 3, eq. md_lemma: moving electron k to r' changes
    column k of A (A(i,j) = phi_i(r_j)); det(A')/det(A) is the dot product
    of row k of A^-1 with the orbital values at r'.  rows: [R, N] (the A^-1
    rows); row_of: [P] row index per position (None: row p).
    """
    v = spo_eval(coefs, pos, KIND_V)                        # [P, N], FP64
    rows = np.asarray(rows, dtype=np.float64)
    idx = np.arange(v.shape[0]) if row_of is None else np.asarray(row_of)
    return np.einsum("pj,pj->p", rows[idx], v)


def spo_ratio_condition(coefs: np.ndarray, pos: np.ndarray, rows: np.ndarray,
                        row_of=None) -> np.ndarray:
    """sum_j |rows[r(p), j]| beta_j(p), with beta the V condition sums: the
    scale of the rounding error of any FP32 evaluation of the ratio."""
    b = condition(coefs, pos, KIND_V)
    rows = np.abs(np.asarray(rows, dtype=np.float64))
    idx = np.arange(b.shape[0]) if row_of is None else np.asarray(row_of)
    return np.einsum("pj,pj->p", rows[idx], b)


def prefilter(samples: np.ndarray) -> np.ndarray:
    """Interpolating B-spline coefficients of periodic grid samples.

    The coefficients the spline of which passes through the samples at the
    grid nodes: along every axis the spline's value at node m is
    (c[m-1] + 4 c[m] + c[m+1]) / 6 (B3 at offsets -1, 0, 1), so c is the
    samples with that circulant operator inverted on each axis.  The inverse
    is taken exactly in Fourier space: the operator's eigenvalue at
    frequency k is (4 + 2 cos(2 pi k / n)) / 6 (the reading of the
    coefficients-vs-samples question that prefilters, with the DFT divided
    by prod_d (2 + cos th_d) / 3).  samples: [nx, ny, nz, N]; FP64 result."""
    c = np.asarray(samples, dtype=np.float64)
    for ax in range(3):
        n = c.shape[ax]
        sym = (4.0 + 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n)) / 6.0
        shape = [1] * c.ndim
        shape[ax] = n
        c = np.real(np.fft.ifft(np.fft.fft(c, axis=ax) / sym.reshape(shape), axis=ax))
    return c
