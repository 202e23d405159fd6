"""Hybrid restructuring on the CUDA-core path (the voxel layout with each voxel's
entries reordered by atom, Sec. 4.1.2), through the C ABI against the FP64 oracle.

The run-compressed kernels apply D's column once per run of equal atoms inside a
voxel; the entrywise kernels once per entry (simt_kernels 1: both entrywise, 2:
both by runs, 0: the default mix, DSC by runs and WC by entries).  Both must meet the FP32 gate
(relative L2 1e-5) on shapes whose runs cross the 32-lane windows, on zero
weights inside runs, on Nθ that is not a multiple of 32, and on a voxel holding a
single long run; the autotuner's timed choice between them must leave results
within the same gate.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


@pytest.fixture(scope="module")
def life():
    import paper_1905_06234_gb300 as L
    L.load(build_if_missing=True)
    return L


def runs_problem(nt, na, nv, nf, nnz, seed, run_len):
    """Random Phi whose atoms repeat in runs of about run_len inside each voxel."""
    rng = np.random.default_rng(seed)
    v = rng.integers(0, nv, nnz).astype(np.int32)
    base = rng.integers(0, na, nnz)
    a = (base // max(run_len, 1) * max(run_len, 1) % na).astype(np.int32) if run_len > 1 else base.astype(np.int32)
    a = np.minimum(a, na - 1).astype(np.int32)
    f = rng.integers(0, nf, nnz).astype(np.int32)
    x = rng.uniform(0.5, 1.0, nnz).astype(np.float32)
    return a, v, f, x


def check(life, idx, phi, D32, nt, nv, nf, seed):
    rng = np.random.default_rng(seed)
    w = rng.random(nf).astype(np.float32)
    w[rng.random(nf) < 0.3] = 0.0
    r = rng.standard_normal(nt * nv).astype(np.float32)
    D = torch.from_numpy(D32).cuda()
    y, _ = life.life_dsc(idx, D, torch.from_numpy(w).cuda())
    g, _ = life.life_wc(idx, D, torch.from_numpy(r).cuda())
    torch.cuda.synchronize()
    life.life_check_device_status()
    ey = rel(y.cpu().numpy(), oracle.dsc(phi, D32, w, nt, nv))
    eg = rel(g.cpu().numpy(), oracle.wc(phi, D32, r, nt, nf))
    assert ey <= TOL and eg <= TOL, (ey, eg)
    return ey, eg


@pytest.mark.parametrize("kernels,bits", [(0, 1), (1, 0), (2, 3)])
@pytest.mark.parametrize("shape", [(96, 360, 500, 400, 60000, 1), (96, 60, 200, 3000, 80000, 6),
                                   (33, 40, 300, 1000, 30000, 9), (7, 5, 50, 2000, 20000, 2)])
def test_run_and_entrywise_kernels(life, kernels, bits, shape):
    nt, na, nv, nf, nnz, run_len = shape
    a, v, f, x = runs_problem(nt, na, nv, nf, nnz, seed=nnz + run_len, run_len=run_len)
    phi = oracle.canon(a, v, f, x, na, nv, nf)
    D32 = np.random.default_rng(2).standard_normal(nt * na).astype(np.float32)
    idx = life.index_from_arrays(a, v, f, x, nt, na, nv, nf, precision=life.LIFE_FP32, algo=life.LIFE_ALGO_SIMT,
                                 simt_kernels=kernels)
    assert idx.info()["simt_runs"] == bits
    check(life, idx, phi, D32, nt, nv, nf, seed=run_len)


@pytest.mark.parametrize("kernels", [0, 2])
def test_single_long_run(life, kernels):
    """One voxel whose 300 entries all share one atom: one run across ten 32-lane windows."""
    nt, na, nv, nf = 96, 360, 4, 500
    f = np.arange(300, dtype=np.int32)
    a = np.full(300, 17, np.int32)
    v = np.full(300, 2, np.int32)
    x = np.linspace(0.5, 1.0, 300).astype(np.float32)
    phi = oracle.canon(a, v, f, x, na, nv, nf)
    D32 = np.random.default_rng(3).standard_normal(nt * na).astype(np.float32)
    idx = life.index_from_arrays(a, v, f, x, nt, na, nv, nf, precision=life.LIFE_FP32, algo=life.LIFE_ALGO_SIMT,
                                 simt_kernels=kernels)
    check(life, idx, phi, D32, nt, nv, nf, seed=5)


def test_autotuned_restructuring(life):
    p = synth.config_problem("tiny")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    idx = life.upload_problem(p, precision=life.LIFE_FP32, algo=life.LIFE_ALGO_SIMT, autotune=True)
    info = idx.info()
    assert info["tuned"] == 1 and info["simt_runs"] in (0, 1, 2, 3)
    check(life, idx, phi, D32, p.n_theta, p.n_voxels, p.n_fasc, seed=7)
