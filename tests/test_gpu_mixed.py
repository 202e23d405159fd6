"""Solves continued from a stopped state (life_sbb_state_resume): reduced-precision
(BF16 tensor-core) iterations to a loose tolerance, then full-precision (FP32)
iterations on the same problem's FP32 index to the final tolerance, from the
same weights and state.  The stopping test stays relative to the first projected
gradient, the iteration count continues, and the result meets the tolerance the
FP32 solve alone meets, at an objective as low as that solve's (both reach the
NNLS optimum to within the tolerance).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1905_06234_gb300._native import SBB_STATE_BYTES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def life():
    import paper_1905_06234_gb300 as L
    L.load(build_if_missing=True)
    return L


@pytest.mark.parametrize("hi_algo", ["simt", "tc"])
def test_bf16_then_fp32_single(life, hi_algo):
    """The FP32 phase on the CUDA cores or on the tensor cores (split FP16 operands)."""
    p = synth.config_problem("tiny")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    b = torch.from_numpy(oracle.problem_signal(phi, D32, p.w_true, p.noise, p.n_theta, p.n_voxels)).cuda()
    D = torch.from_numpy(D32).cuda()
    lo = life.upload_problem(p, precision=life.LIFE_BF16, algo=life.LIFE_ALGO_TC)
    hi = life.upload_problem(p, precision=life.LIFE_FP32,
                             algo=life.LIFE_ALGO_SIMT if hi_algo == "simt" else life.LIFE_ALGO_TC)
    tol = 1e-4
    # FP32 alone
    w_ref = torch.ones(p.n_fasc, device="cuda")
    st_ref, ws_hi = life.new_sbb_state(), life.new_sbb_workspace(hi)
    life.life_sbbnnls_solve(hi, D, b, w_ref, 500, st_ref, ws_hi, tol=tol)
    # BF16 to 1e-3, then FP32 to 1e-4 from the same w and state
    w = torch.ones(p.n_fasc, device="cuda")
    st, ws_lo = life.new_sbb_state(), life.new_sbb_workspace(lo)
    life.life_sbbnnls_solve(lo, D, b, w, 500, st, ws_lo, tol=1e-3)
    s1 = life.read_sbb_state(st)
    assert s1["converged"] == 1
    life.life_sbb_state_resume(st)
    s1b = life.read_sbb_state(st)
    assert s1b["converged"] == 0 and s1b["it"] == s1["it"] and s1b["gg0"] == s1["gg0"]
    life.life_sbbnnls_solve(hi, D, b, w, 500, st, life.new_sbb_workspace(hi), tol=tol)
    torch.cuda.synchronize()
    life.life_check_device_status()
    s2, sr = life.read_sbb_state(st), life.read_sbb_state(st_ref)
    assert s2["converged"] == 1 and s2["it"] > s1["it"]
    assert np.sqrt(s2["gg"]) <= tol * np.sqrt(s2["gg0"])
    assert sr["converged"] == 1
    # the objective the continued solve stops at is as low as the FP32 solve's (the
    # two stop at different points of the same small neighbourhood of the optimum)
    assert s2["obj"] <= sr["obj"] * (1 + 1e-3), (s2["obj"], sr["obj"])
    # and the weights are KKT points to the tolerance: projected gradient checked on the oracle
    wn = w.double().cpu().numpy()
    e = oracle.dsc(phi, D32, wn, p.n_theta, p.n_voxels) - b.double().cpu().numpy()
    g = oracle.wc(phi, D32, e, p.n_theta, p.n_fasc)
    gt = np.where((wn == 0) & (g > 0), 0.0, g)
    g0 = oracle.wc(phi, D32, oracle.dsc(phi, D32, np.ones(p.n_fasc), p.n_theta, p.n_voxels)
                   - b.double().cpu().numpy(), p.n_theta, p.n_fasc)
    assert np.linalg.norm(gt) <= 2 * tol * np.linalg.norm(g0)


def test_resume_many_states(life):
    st = life.new_batch_states(3)
    raw = st.cpu().numpy().copy()
    conv_off = SBB_STATE_BYTES - 4
    for k in range(3):
        raw[k * SBB_STATE_BYTES + conv_off:(k + 1) * SBB_STATE_BYTES] = np.frombuffer(
            np.int32(1).tobytes(), np.uint8)
    st.copy_(torch.from_numpy(raw))
    assert all(x["converged"] == 1 for x in life.read_batch_states(st, 3))
    life.life_sbb_state_resume(st, 3)
    assert all(x["converged"] == 0 and x["it"] == 0 and x["alpha"] == 1.0 for x in life.read_batch_states(st, 3))
