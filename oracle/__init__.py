"""FP64 CPU oracle for the LiFE hot path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  The CUDA library never calls it and shares no code with it.

Thin ctypes wrapper over ``oracle.c`` (plain double-precision loops written from
the paper's definitions; see that file's header for the equation each routine
follows).  Array conventions: D is a flat column-major vector ``D[θ + Nθ·a]``;
signals are flat column-major ``y[θ + Nθ·v]``; Phi is four parallel COO arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_OMP_SRC = os.path.join(_HERE, "oracle_omp.c")
_OMP_LIB = os.path.join(_HERE, "liboracle_omp.so")
_lib = None
_omp = None

ORDER_VOXEL, ORDER_FIBER, ORDER_ATOM = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, -O2, no FP contraction so both host ISAs round alike)
    and liboracle_omp.so (the same arithmetic on all host cores, OpenMP)."""
    for src, lib, extra in ((_SRC, _LIB, []), (_OMP_SRC, _OMP_LIB, ["-fopenmp"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            tmp = lib + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", *extra, "-o", tmp, src,
                                   "-lm"])
            os.replace(tmp, lib)
    return _LIB


class _SbbState(ctypes.Structure):
    _fields_ = [("it", ctypes.c_int64), ("alpha", ctypes.c_double), ("obj", ctypes.c_double),
                ("gg", ctypes.c_double), ("gg0", ctypes.c_double), ("vv", ctypes.c_double),
                ("uu", ctypes.c_double), ("eq", ctypes.c_int32), ("converged", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.oracle_dictionary.argtypes = [i32, i32, P, P, dbl, dbl, P, P]
        lib.oracle_canon.argtypes = [i64, P, P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, i32,
                                     P, P, P, P]
        lib.oracle_canon.restype = i64
        lib.oracle_dsc.argtypes = [i64, P, P, P, P, i32, P, P, i64, P]
        lib.oracle_wc.argtypes = [i64, P, P, P, P, i32, P, P, i64, P]
        lib.oracle_grad_D.argtypes = [i64, P, P, P, P, i32, i32, P, P, P]
        lib.oracle_sbb_step.argtypes = [i64, P, P, P, P, i32, P, i64, i64, P, P, dbl, i32,
                                        ctypes.POINTER(_SbbState), P]
        lib.oracle_sbb_solve.argtypes = [i64, P, P, P, P, i32, P, i64, i64, P, P, dbl, i32, i64,
                                         ctypes.POINTER(_SbbState), P]
        lib.oracle_voxel_rmse.argtypes = [i32, i64, P, P]
        lib.oracle_voxel_rmse.restype = dbl
        lib.oracle_prune.argtypes = [i64, P, ctypes.c_float, P, P]
        lib.oracle_prune.restype = i64
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    return ctypes.c_void_p(a.ctypes.data)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


@dataclass
class Phi:
    """Phi as parallel COO arrays (atom, voxel, fascicle, value)."""
    atom: np.ndarray
    voxel: np.ndarray
    fasc: np.ndarray
    val: np.ndarray

    def __len__(self):
        return int(self.atom.shape[0])


# Every wrapper below binds each converted array to a local name before the C
# call, so that no temporary copy is freed while the C code still reads it.

def dictionary(grad_dirs, atom_dirs, bval: float, lam: float):
    """D (flat column-major, Nθ·Na) and dD/dλ, both demeaned per column."""
    g, u = _f64(grad_dirs), _f64(atom_dirs)
    nt, na = g.shape[0], u.shape[0]
    D = np.empty(nt * na, np.float64)
    dD = np.empty(nt * na, np.float64)
    _load().oracle_dictionary(nt, na, _p(g), _p(u), float(bval), float(lam), _p(D), _p(dD))
    return D, dD


def canon(atom, voxel, fasc, val, n_atoms, n_voxels, n_fasc, order=ORDER_VOXEL) -> Phi:
    """Restructured Phi: sorted by the chosen dimension, duplicates merged (FP64
    sum, one rounding to float32)."""
    a, v, f = _i32(atom), _i32(voxel), _i32(fasc)
    x = np.ascontiguousarray(val, dtype=np.float32)
    n = a.shape[0]
    oa, ov, of = (np.empty(n, np.int32) for _ in range(3))
    ox = np.empty(n, np.float32)
    m = _load().oracle_canon(n, _p(a), _p(v), _p(f), _p(x), n_atoms, n_voxels, n_fasc, order,
                             _p(oa), _p(ov), _p(of), _p(ox))
    if m < 0:
        raise ValueError("oracle_canon: index out of range or non-finite value")
    return Phi(oa[:m].copy(), ov[:m].copy(), of[:m].copy(), ox[:m].copy())


def _phi_args(phi: Phi):
    return _i32(phi.atom), _i32(phi.voxel), _i32(phi.fasc), _f64(phi.val)


def dsc(phi: Phi, D, w, n_theta: int, n_voxels: int) -> np.ndarray:
    """y = M w in FP64 (flat column-major)."""
    y = np.empty(n_theta * n_voxels, np.float64)
    a, v, f, val = _phi_args(phi)
    Dd, wd = _f64(D), _f64(w)
    _load().oracle_dsc(len(phi), _p(a), _p(v), _p(f), _p(val), n_theta, _p(Dd), _p(wd), n_voxels, _p(y))
    return y


def wc(phi: Phi, D, r, n_theta: int, n_fasc: int) -> np.ndarray:
    """g = M^T r in FP64."""
    g = np.empty(n_fasc, np.float64)
    a, v, f, val = _phi_args(phi)
    Dd, rd = _f64(D), _f64(r)
    _load().oracle_wc(len(phi), _p(a), _p(v), _p(f), _p(val), n_theta, _p(Dd), _p(rd), n_fasc, _p(g))
    return g


def grad_D(phi: Phi, w, e, n_theta: int, n_atoms: int) -> np.ndarray:
    """dL/dD (flat column-major) for L = ½‖r - M(D) w‖², given e = M w - r."""
    gD = np.empty(n_theta * n_atoms, np.float64)
    a, v, f, val = _phi_args(phi)
    wd, ed = _f64(w), _f64(e)
    _load().oracle_grad_D(len(phi), _p(a), _p(v), _p(f), _p(val), n_theta, n_atoms, _p(wd), _p(ed), _p(gD))
    return gD


def loss_grads(phi: Phi, D, dD_dlam, w, r, n_theta, n_atoms, n_voxels, n_fasc):
    """L = ½‖r - M(D) w‖² and its gradients w.r.t. w, D and λ (through dD/dλ)."""
    e = dsc(phi, D, w, n_theta, n_voxels) - _f64(r)
    L = 0.5 * float(e @ e)
    gw = wc(phi, D, e, n_theta, n_fasc)
    gD = grad_D(phi, w, e, n_theta, n_atoms)
    glam = float(gD @ _f64(dD_dlam))
    return L, gw, gD, glam


class SbbState:
    """SBB-NNLS state: iteration count, last alpha, last dot products."""

    def __init__(self):
        self.s = _SbbState(it=0, alpha=1.0, obj=0.0, gg=0.0, gg0=0.0, vv=0.0, uu=0.0, eq=0, converged=0)

    def __getattr__(self, k):
        return getattr(self.__dict__["s"], k)

    def as_dict(self):
        return {k: getattr(self.s, k) for k, _ in _SbbState._fields_}


def sbb_step(phi: Phi, D, b, w, n_theta, n_voxels, n_fasc, state: SbbState, tol=0.0, eq7_on_even=True):
    """One SBB-NNLS iteration; updates ``w`` (float64 array) in place."""
    assert w.dtype == np.float64 and w.flags.c_contiguous
    work = np.empty(2 * n_theta * n_voxels + 2 * n_fasc, np.float64)
    a, v, f, val = _phi_args(phi)
    Dd, bd = _f64(D), _f64(b)
    _load().oracle_sbb_step(len(phi), _p(a), _p(v), _p(f), _p(val), n_theta, _p(Dd), n_voxels, n_fasc, _p(bd),
                            _p(w), float(tol), 1 if eq7_on_even else 0, ctypes.byref(state.s), _p(work))
    return state


def sbb_solve(phi: Phi, D, b, w, n_theta, n_voxels, n_fasc, max_iter, tol=0.0, eq7_on_even=True, state=None):
    """Up to ``max_iter`` SBB-NNLS iterations from ``w`` (float64, updated in place)."""
    state = state or SbbState()
    assert w.dtype == np.float64 and w.flags.c_contiguous
    work = np.empty(2 * n_theta * n_voxels + 2 * n_fasc, np.float64)
    a, v, f, val = _phi_args(phi)
    Dd, bd = _f64(D), _f64(b)
    _load().oracle_sbb_solve(len(phi), _p(a), _p(v), _p(f), _p(val), n_theta, _p(Dd), n_voxels, n_fasc, _p(bd),
                             _p(w), float(tol), 1 if eq7_on_even else 0, int(max_iter), ctypes.byref(state.s),
                             _p(work))
    return state


def problem_signal(phi: Phi, D, w_true, noise, n_theta, n_voxels):
    """b = M w_true + noise, rounded to float32 (the measured, demeaned signal)."""
    return (dsc(phi, D, w_true, n_theta, n_voxels) + _f64(noise)).astype(np.float32)


def voxel_rmse(e, n_theta: int, n_voxels: int):
    """(rmse [Nv], Σ e²): per-voxel root-mean-square of a residual over θ."""
    ed = _f64(e)
    assert ed.size == n_theta * n_voxels
    rmse = np.empty(n_voxels, np.float64)
    total = _load().oracle_voxel_rmse(n_theta, n_voxels, _p(ed), _p(rmse))
    return rmse, float(total)


def prune(w, threshold: float = 0.0):
    """(keep mask uint8 [Nf], kept fascicle ids int32): fascicles with w > threshold."""
    wf = np.ascontiguousarray(w, dtype=np.float32)
    keep = np.empty(wf.size, np.uint8)
    kept = np.empty(max(wf.size, 1), np.int32)
    n = _load().oracle_prune(wf.size, _p(wf), float(threshold), _p(keep), _p(kept))
    return keep, kept[:n].copy()


# ------------------------------------------------------------ all host cores

def _load_omp():
    global _omp
    if _omp is None:
        build()
        lib = ctypes.CDLL(_OMP_LIB)
        P, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.oracle_omp_threads.restype = i32
        lib.oracle_omp_set_threads.argtypes = [i32]
        lib.oracle_omp_group.argtypes = [i64, P, i64, P, P]
        lib.oracle_omp_dsc.argtypes = [P, P, P, P, P, i32, P, P, i64, P]
        lib.oracle_omp_wc.argtypes = [P, P, P, P, P, i32, P, P, i64, P]
        lib.oracle_omp_sbb_step.argtypes = [P, P, P, P, P, P, P, P, i32, P, i64, i64, P, P, dbl, i32,
                                            ctypes.POINTER(_SbbState), P]
        _omp = lib
    return _omp


def omp_threads() -> int:
    """Host threads the OpenMP baseline uses (OMP_NUM_THREADS, else all cores)."""
    return int(_load_omp().oracle_omp_threads())


def omp_set_threads(n: int):
    """Threads for the following OpenMP baseline calls."""
    _load_omp().oracle_omp_set_threads(int(n))


class OmpProblem:
    """Phi grouped by voxel (DSC) and by fascicle (WC) for the all-cores baseline.
    Raw COO entries are accepted as they are: repeated (a, v, f) entries add up."""

    def __init__(self, atom, voxel, fasc, val, n_theta, n_voxels, n_fasc):
        L = _load_omp()
        self.atom, self.voxel, self.fasc = _i32(atom), _i32(voxel), _i32(fasc)
        self.val = _f64(val)
        self.nt, self.nv, self.nf = int(n_theta), int(n_voxels), int(n_fasc)
        n = self.atom.size
        self.vptr = np.empty(self.nv + 1, np.int64)
        self.vperm = np.empty(max(n, 1), np.int64)
        self.fptr = np.empty(self.nf + 1, np.int64)
        self.fperm = np.empty(max(n, 1), np.int64)
        L.oracle_omp_group(n, _p(self.voxel), self.nv, _p(self.vptr), _p(self.vperm))
        L.oracle_omp_group(n, _p(self.fasc), self.nf, _p(self.fptr), _p(self.fperm))

    def dsc(self, D, x):
        y = np.empty(self.nt * self.nv, np.float64)
        Dd, xd = _f64(D), _f64(x)
        _load_omp().oracle_omp_dsc(_p(self.vptr), _p(self.vperm), _p(self.atom), _p(self.fasc), _p(self.val),
                                   self.nt, _p(Dd), _p(xd), self.nv, _p(y))
        return y

    def wc(self, D, r):
        g = np.empty(self.nf, np.float64)
        Dd, rd = _f64(D), _f64(r)
        _load_omp().oracle_omp_wc(_p(self.fptr), _p(self.fperm), _p(self.atom), _p(self.voxel), _p(self.val),
                                  self.nt, _p(Dd), _p(rd), self.nf, _p(g))
        return g

    def sbb_step(self, D, b, w, state: SbbState, tol=0.0, eq7_on_even=True, work=None):
        """One SBB-NNLS iteration on all cores; updates ``w`` (float64) in place."""
        assert w.dtype == np.float64 and w.flags.c_contiguous
        if work is None:
            work = np.empty(2 * self.nt * self.nv + 2 * self.nf, np.float64)
        Dd, bd = _f64(D), _f64(b)
        _load_omp().oracle_omp_sbb_step(_p(self.vptr), _p(self.vperm), _p(self.fptr), _p(self.fperm),
                                        _p(self.atom), _p(self.voxel), _p(self.fasc), _p(self.val), self.nt, _p(Dd),
                                        self.nv, self.nf, _p(bd), _p(w), float(tol), 1 if eq7_on_even else 0,
                                        ctypes.byref(state.s), _p(work))
        return state
