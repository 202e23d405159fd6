"""Connectome evaluation outputs on the GPU (life_prune, life_voxel_rmse) against
the FP64 oracle, through the C ABI.

Pruning is index work and must match bit for bit (keep mask, kept list and
count, the pruned weights).  The per-voxel RMSE sums in FP64 on both sides and
rounds once to float32, so the two may differ only in the summation order of the
FP64 sum: at most one float32 ulp (relative 2^-23) per voxel.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests._golden import read_sections

pytestmark = pytest.mark.gpu

ULP_REL = 2.0 ** -23


@pytest.fixture(scope="module")
def life():
    import paper_1905_06234_gb300 as L
    L.load(build_if_missing=True)
    return L


def _golden():
    s = read_sections("evaluate_small.txt")
    nt, nv = (int(x) for x in s["dims"][0])
    flat = lambda k: np.array([x for row in s[k] for x in row], np.float64)
    return nt, nv, flat


def test_voxel_rmse_golden(life):
    nt, nv, flat = _golden()
    e = torch.tensor(flat("e"), dtype=torch.float32, device="cuda")
    rmse, ss = life.life_voxel_rmse(e, nt, nv)
    torch.cuda.synchronize()
    np.testing.assert_allclose(rmse.cpu().numpy(), flat("rmse"), rtol=ULP_REL, atol=0)
    assert float(ss.item()) == flat("total")[0]


@pytest.mark.parametrize("nt,nv", [(1, 5), (31, 1000), (33, 777), (96, 20000), (150, 257), (96, 0)])
def test_voxel_rmse_vs_oracle(life, nt, nv):
    rng = np.random.default_rng(nt * 1000 + nv)
    e = (rng.standard_normal(nt * nv) * rng.choice([1e-3, 1.0, 1e3], nt * nv)).astype(np.float32)
    rmse, ss = life.life_voxel_rmse(torch.from_numpy(e).cuda(), nt, nv)
    torch.cuda.synchronize()
    ref, total = oracle.voxel_rmse(e, nt, nv)
    got = rmse.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, ref.astype(np.float32).astype(np.float64), rtol=ULP_REL, atol=0)
    assert abs(float(ss.item()) - total) <= 1e-12 * max(total, 1e-300)


def _check_prune(life, w, thr):
    keep_ref, kept_ref = oracle.prune(w, thr)
    keep, kept, w_pruned = life.life_prune(torch.from_numpy(w).cuda(), thr)
    torch.cuda.synchronize()
    assert np.array_equal(keep.cpu().numpy(), keep_ref)
    assert np.array_equal(kept.cpu().numpy(), kept_ref)
    wp_ref = np.where(keep_ref == 1, w, np.float32(0)).astype(np.float32)
    assert np.array_equal(w_pruned.cpu().numpy().view(np.uint32), wp_ref.view(np.uint32))


def test_prune_golden(life):
    _, _, flat = _golden()
    w = flat("w").astype(np.float32)
    for thr in (0.0, 0.25):
        _check_prune(life, w, thr)


@pytest.mark.parametrize("nf", [0, 1, 1000, 1 << 20, 500_000])
def test_prune_vs_oracle(life, nf):
    rng = np.random.default_rng(nf + 11)
    w = rng.random(nf).astype(np.float32)
    w[rng.random(nf) < 0.3] = 0.0
    neg = rng.random(nf) < 0.01
    w[neg] = -rng.random(int(neg.sum())).astype(np.float32)
    w[rng.random(nf) < 0.001] = np.nan
    for thr in (0.0, 0.5, np.float32(0.3)):
        _check_prune(life, w, float(thr))


def test_evaluate_pruned_connectome(life):
    """Prune an SBB-NNLS solution, predict with the pruned weights, and compare the
    per-voxel prediction error with the oracle's on the same pruned weights."""
    p = synth.config_problem("tiny")
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    D64, _ = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
    D32 = D64.astype(np.float32)
    b = oracle.problem_signal(phi, D32, p.w_true, p.noise, p.n_theta, p.n_voxels)
    idx = life.upload_problem(p, precision=life.LIFE_FP32)
    D = torch.from_numpy(D32).cuda()
    bt = torch.from_numpy(b).cuda()
    w = torch.ones(p.n_fasc, dtype=torch.float32, device="cuda")
    st = life.new_sbb_state()
    ws = life.new_sbb_workspace(idx)
    life.life_sbbnnls_solve(idx, D, bt, w, 50, st, ws)
    out = life.evaluate_connectome(idx, D, w, bt)
    torch.cuda.synchronize()
    life.life_check_device_status()
    wn = w.cpu().numpy()
    keep_ref, kept_ref = oracle.prune(wn, 0.0)
    assert np.array_equal(out["kept"].cpu().numpy(), kept_ref)
    assert 0 < kept_ref.size < p.n_fasc  # the solve zeroed some fascicles
    wp = np.where(keep_ref == 1, wn, 0.0)
    e_ref = oracle.dsc(phi, D32, wp, p.n_theta, p.n_voxels) - b
    rmse_ref, total = oracle.voxel_rmse(e_ref, p.n_theta, p.n_voxels)
    got = out["rmse"].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - rmse_ref) <= 1e-4 * np.linalg.norm(rmse_ref)
    g_ref = np.sqrt(total / (p.n_theta * p.n_voxels))
    assert abs(out["global_rmse"] - g_ref) <= 1e-4 * g_ref
    idx.close()
