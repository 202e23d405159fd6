"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The paper-scale workload (79.5M merged entries) is too large for the oracle to
recompute every output within a test, so sampled outputs are checked: the oracle
evaluates y[:, v] for 48 random voxels from the raw entries of those voxels, and
g[f] for 48 random fascicles from the raw entries of those fascicles.  The
medium workload is checked in full, including one SBB-NNLS iteration.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_BF16 = 3e-3
U_BF16 = 2.0 ** -8
U_TC = 2 * U_BF16 + 2.0 ** -11   # BF16 Phi value and D, FP16 operand (S or r)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def life():
    import paper_1905_06234_gb300 as L
    L.load(build_if_missing=True)
    return L


@pytest.fixture(scope="module")
def paper():
    p = synth.config_problem("paper")
    return p


def sampled_check(life, p, idx, D32, tol, bf16):
    rng = np.random.default_rng(42)
    w = p.w_true.copy()
    r = rng.standard_normal(p.n_theta * p.n_voxels).astype(np.float32)
    D = torch.from_numpy(D32).cuda()
    y, _ = life.life_dsc(idx, D, torch.from_numpy(w).cuda())
    g, _ = life.life_wc(idx, D, torch.from_numpy(r).cuda())
    torch.cuda.synchronize()
    life.life_check_device_status()
    y = y.cpu().numpy()
    g = g.cpu().numpy()
    nt = p.n_theta
    vs = np.sort(rng.choice(p.n_voxels, 48, replace=False))
    sel = np.isin(p.coo_voxel, vs)
    phi_v = oracle.Phi(p.coo_atom[sel], p.coo_voxel[sel], p.coo_fasc[sel], p.coo_val[sel])
    y_ref = oracle.dsc(phi_v, D32, w, nt, p.n_voxels).reshape(p.n_voxels, nt)[vs]
    y_got = y.reshape(p.n_voxels, nt)[vs]
    fs = np.sort(rng.choice(p.n_fasc, 48, replace=False))
    self_ = np.isin(p.coo_fasc, fs)
    phi_f = oracle.Phi(p.coo_atom[self_], p.coo_voxel[self_], p.coo_fasc[self_], p.coo_val[self_])
    g_ref = oracle.wc(phi_f, D32, r, nt, p.n_fasc)[fs]
    errs = dict(y=rel(y_got, y_ref), g=rel(g[fs], g_ref))
    assert errs["y"] <= tol and errs["g"] <= tol, errs
    if bf16:
        a = np.abs
        yb = oracle.dsc(oracle.Phi(phi_v.atom, phi_v.voxel, phi_v.fasc, a(phi_v.val)), a(D32), a(w), nt,
                        p.n_voxels).reshape(p.n_voxels, nt)[vs]
        gb = oracle.wc(oracle.Phi(phi_f.atom, phi_f.voxel, phi_f.fasc, a(phi_f.val)), a(D32), a(r), nt, p.n_fasc)[fs]
        assert (np.abs(y_got - y_ref) <= 1.25 * U_TC * yb).all()
        assert (np.abs(g[fs] - g_ref) <= 1.25 * U_TC * gb).all()
    return errs


def test_paper_scale_fp32_simt(life, paper):
    p = paper
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    idx = life.upload_problem(p, precision=life.LIFE_FP32, algo=life.LIFE_ALGO_SIMT)
    assert idx.nnz > 79_000_000
    print("paper fp32", sampled_check(life, p, idx, D32, TOL_FP32, bf16=False))
    idx.close()


def test_paper_scale_bf16_tc(life, paper):
    p = paper
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    idx = life.upload_problem(p, precision=life.LIFE_BF16, algo=life.LIFE_ALGO_TC)
    info = idx.info()
    assert info["algo"] == life.LIFE_ALGO_TC and info["brick_edge"] == 8
    print("paper bf16", sampled_check(life, p, idx, D32, TOL_BF16, bf16=True), info["n_bricks"], info["n_tiles"])
    idx.close()


def test_paper_scale_fp32_tc(life, paper):
    """FP32 storage on the tensor cores (split FP16 operands) at the FP32 tolerance."""
    p = paper
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    idx = life.upload_problem(p, precision=life.LIFE_FP32, algo=life.LIFE_ALGO_TC)
    info = idx.info()
    assert info["algo"] == life.LIFE_ALGO_TC and info["precision"] == life.LIFE_FP32
    print("paper fp32-tc", sampled_check(life, p, idx, D32, TOL_FP32, bf16=False))
    idx.close()


@pytest.mark.parametrize("precision", ["fp32", "fp32-tc", "bf16"])
def test_medium_full_and_sbb_step(life, precision):
    p = synth.config_problem("medium")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    b = oracle.problem_signal(phi, D32, p.w_true, p.noise, p.n_theta, p.n_voxels)
    bf = precision == "bf16"
    tc = precision != "fp32"
    idx = life.upload_problem(p, precision=life.LIFE_BF16 if bf else life.LIFE_FP32,
                              algo=life.LIFE_ALGO_TC if tc else life.LIFE_ALGO_SIMT)
    tol = TOL_BF16 if bf else TOL_FP32
    D = torch.from_numpy(D32).cuda()
    y, _ = life.life_dsc(idx, D, torch.from_numpy(p.w_true).cuda())
    g, _ = life.life_wc(idx, D, torch.from_numpy(b).cuda())
    torch.cuda.synchronize()
    life.life_check_device_status()
    ey = rel(y.cpu().numpy(), oracle.dsc(phi, D32, p.w_true, p.n_theta, p.n_voxels))
    eg = rel(g.cpu().numpy(), oracle.wc(phi, D32, b, p.n_theta, p.n_fasc))
    assert ey <= tol and eg <= tol, (ey, eg)
    # one SBB-NNLS iteration from w = 1 against the oracle iteration
    w = torch.ones(p.n_fasc, device="cuda")
    st, ws = life.new_sbb_state(), life.new_sbb_workspace(idx)
    life.life_sbbnnls_step(idx, D, torch.from_numpy(b).cuda(), w, st, ws)
    torch.cuda.synchronize()
    w_ref = np.ones(p.n_fasc)
    ost = oracle.sbb_step(phi, D32, b, w_ref, p.n_theta, p.n_voxels, p.n_fasc, oracle.SbbState())
    gst = life.read_sbb_state(st)
    # FP32 on the tensor cores: the step's dot products carry its DSC error (a few
    # 1e-6 of |Mw|) amplified by |Mw| / |e| and the cancellation in M^T e
    stol = 3e-2 if bf else (1e-3 if tc else 1e-4)
    for k in ("obj", "gg", "vv", "alpha"):
        assert abs(gst[k] - getattr(ost, k)) <= stol * abs(getattr(ost, k)), (k, gst[k], getattr(ost, k))
    assert rel(w.cpu().numpy(), w_ref) <= (3e-2 if bf else 1e-4)
    print(precision, "medium", ey, eg)
