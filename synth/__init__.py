"""Seeded synthetic LiFE inputs (tractography-shaped), shared by the oracle and the CUDA path.

This module holds the input recipe only: gradient/atom direction sets, persistent
random walks that emit raw Phi entries (duplicates not merged), ground-truth
weights and Gaussian noise.  None of the method's arithmetic lives here: the
dictionary D, duplicate merging, ``M w`` and ``M^T r`` are computed by whoever
consumes the problem (the oracle in tests, the CUDA library in the product path).

The walk model follows the problem statement of the LiFE paper (Sec. 2.1: voxels,
fascicles, gradient directions; Eq. 3: a fascicle contributes one dictionary atom
per voxel it crosses) with the shapes of its workloads (Nθ = 96 directions at
b = 2000 s/mm², 10^5 - 10^6 voxels, up to 5·10^5 fascicles; Sec. 6, Table 9).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "walks.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

SEED_BASE = 1905062340


def build(force: bool = False) -> str:
    """Compile libsynth.so with gcc (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
        lib.synth_fibonacci_sphere.argtypes = [i32, P]
        lib.synth_fibonacci_hemisphere.argtypes = [i32, P]
        lib.synth_voxel_ids.argtypes = [i32, i32, i32, i32, P]
        lib.synth_voxel_ids.restype = i64
        lib.synth_walk_lengths.argtypes = [u64, i64, i32, i32, P]
        lib.synth_walks.argtypes = [u64, i64, P, P, i32, i32, i32, P, i32, i32, P, dbl, dbl, dbl, P, P, P, P]
        lib.synth_w_true.argtypes = [u64, i64, dbl, P]
        lib.synth_noise.argtypes = [u64, i64, dbl, P]
        lib.synth_loguniform_int.argtypes = [u64, i64, i64, i64]
        lib.synth_loguniform_int.restype = i64
        lib.synth_uniform_int.argtypes = [u64, i64, i64, i64]
        lib.synth_uniform_int.restype = i64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def fibonacci_sphere(n: int) -> np.ndarray:
    out = np.zeros((n, 3), np.float64)
    _load().synth_fibonacci_sphere(n, _ptr(out))
    return out


def fibonacci_hemisphere(n: int) -> np.ndarray:
    out = np.zeros((n, 3), np.float64)
    _load().synth_fibonacci_hemisphere(n, _ptr(out))
    return out


@dataclass
class Problem:
    """One synthetic LiFE problem.

    ``coo_*`` is the raw Phi list in walk order (one entry per walk step, duplicate
    (atom, voxel, fascicle) triples NOT merged).  ``noise`` is column-major
    ``[θ + Nθ·v]`` like the signal.  ``voxel_ijk`` holds each voxel's grid
    coordinates.  Units: bval in ms/µm², lam in µm²/ms.
    """
    name: str
    seed: int
    n_theta: int
    n_atoms: int
    n_voxels: int
    n_fasc: int
    grid: tuple
    grad_dirs: np.ndarray
    atom_dirs: np.ndarray
    bval: float
    lam: float
    coo_atom: np.ndarray
    coo_voxel: np.ndarray
    coo_fasc: np.ndarray
    coo_val: np.ndarray
    w_true: np.ndarray
    noise: np.ndarray
    voxel_ijk: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_raw(self) -> int:
        return int(self.coo_atom.shape[0])


def make_problem(name: str = "custom", *, seed: int, n_theta: int = 96, n_atoms: int = 360,
                 grid=(16, 16, 16), mask: bool = False, n_fasc: int = 2000,
                 steps=(40, 80), step_len=(0.5, 1.0), persist: float = 0.3,
                 bval: float = 2.0, lam: float = 1.7, zero_frac: float = 0.3,
                 sigma: float = 0.01, with_noise: bool = True) -> Problem:
    lib = _load()
    nx, ny, nz = (int(x) for x in grid)
    vox_id = np.empty(nx * ny * nz, np.int32)
    nv = int(lib.synth_voxel_ids(nx, ny, nz, 1 if mask else 0, _ptr(vox_id)))
    lin = np.nonzero(vox_id >= 0)[0]
    ijk = np.stack([lin % nx, (lin // nx) % ny, lin // (nx * ny)], axis=1).astype(np.int32)
    g = fibonacci_sphere(n_theta)
    u = fibonacci_hemisphere(n_atoms)
    lens = np.empty(n_fasc, np.int32)
    lib.synth_walk_lengths(seed, n_fasc, int(steps[0]), int(steps[1]), _ptr(lens))
    off = np.zeros(n_fasc + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    n_raw = int(off[-1])
    atom = np.empty(n_raw, np.int32)
    vox = np.empty(n_raw, np.int32)
    fas = np.empty(n_raw, np.int32)
    val = np.empty(n_raw, np.float32)
    u_c = np.ascontiguousarray(u)  # kept alive across the C call
    lib.synth_walks(seed, n_fasc, _ptr(lens), _ptr(off), nx, ny, nz, _ptr(vox_id), 1 if mask else 0,
                    n_atoms, _ptr(u_c), persist, float(step_len[0]), float(step_len[1]),
                    _ptr(atom), _ptr(vox), _ptr(fas), _ptr(val))
    w_true = np.empty(n_fasc, np.float32)
    lib.synth_w_true(seed, n_fasc, zero_frac, _ptr(w_true))
    noise = np.zeros(n_theta * nv, np.float32)
    if with_noise:
        lib.synth_noise(seed, n_theta * nv, sigma, _ptr(noise))
    return Problem(name=name, seed=seed, n_theta=n_theta, n_atoms=n_atoms, n_voxels=nv, n_fasc=n_fasc,
                   grid=(nx, ny, nz), grad_dirs=g, atom_dirs=u, bval=bval, lam=lam,
                   coo_atom=atom, coo_voxel=vox, coo_fasc=fas, coo_val=val, w_true=w_true,
                   noise=noise, voxel_ijk=ijk,
                   meta=dict(mask=mask, steps=tuple(steps), step_len=tuple(step_len), persist=persist,
                             zero_frac=zero_frac, sigma=sigma))


# The five workloads.  Sizes follow the paper's data (Nθ = 96, b = 2000 s/mm²,
# Sec. 6.1; Nf up to 5·10^5 and 1.4-2.6·10^5 voxels, Table 9).
CONFIGS = {
    "tiny": dict(grid=(16, 16, 16), mask=False, n_fasc=2000, steps=(40, 80)),
    "medium": dict(grid=(64, 64, 64), mask=False, n_fasc=50000, steps=(30, 150)),
    "paper": dict(grid=(96, 96, 72), mask=True, n_fasc=500000, steps=(20, 300)),
    "grad": dict(grid=(16, 16, 16), mask=False, n_fasc=2000, steps=(40, 80)),
    # paper density (entries per voxel and per fascicle) at about a third of the
    # size: the case profiled with hardware counters
    "paper_small": dict(grid=(64, 64, 48), mask=True, n_fasc=150000, steps=(20, 300)),
}
CONFIG_INDEX = {"tiny": 1, "medium": 2, "paper": 3, "grad": 4, "batched": 5, "paper_small": 6}


def config_problem(name: str, **overrides) -> Problem:
    kw = dict(CONFIGS[name])
    kw.update(overrides)
    seed = kw.pop("seed", SEED_BASE + CONFIG_INDEX[name])
    return make_problem(name, seed=seed, **kw)


def batched_shapes(n: int = 16, seed: int = SEED_BASE + 5):
    """Shapes of the batched workload: Nf log-uniform in [1e4, 2e5], cubic grid
    edge uniform in [32, 80], walks of 30-150 steps, no mask."""
    lib = _load()
    out = []
    for k in range(n):
        nf = int(lib.synth_loguniform_int(seed, k, 10000, 200000))
        edge = int(lib.synth_uniform_int(seed, k, 32, 80))
        out.append(dict(grid=(edge, edge, edge), mask=False, n_fasc=nf, steps=(30, 150), seed=seed * 100 + k))
    return out


def batched_problems(n: int = 16, seed: int = SEED_BASE + 5, scale: float = 1.0):
    """The batched workload's problems; ``scale`` < 1 shrinks Nf and the grid edge
    (for quick tests) while keeping the uneven size mix."""
    probs = []
    for k, s in enumerate(batched_shapes(n, seed)):
        s = dict(s)
        sd = s.pop("seed")
        if scale != 1.0:
            e = max(8, int(round(s["grid"][0] * scale ** (1 / 3))))
            s["grid"] = (e, e, e)
            s["n_fasc"] = max(50, int(s["n_fasc"] * scale))
        probs.append(make_problem(f"batched{k}", seed=sd, **s))
    return probs
