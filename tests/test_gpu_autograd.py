"""Differentiation through DSC: the autograd wrappers (CUDA backward passes)
against the FP64 oracle's analytic gradients, on the differentiation workload
(16^3 grid, 2000 fascicles, Nθ = 96, Na = 360).

Loss: L = ½‖r − M(D(λ)) w‖².  The oracle's gradients are themselves pinned to
central finite differences (h = 1e-3, FP64) in test_oracle.py; here a GPU-side
finite difference in λ checks the chained derivative once more.

FP32 path: relative L2 error against the FP64 oracle on the same float32 inputs
at most 1e-5.  dL/dλ is a single sum over Nθ·Na products with cancellation, so
it is compared with the same tolerance scaled by Σ|dL/dD·dD/dλ| / |dL/dλ| (the
sum's condition number).

BF16 storage: the backward pass consumes the forward residual, so the forward
rounding error reaches every gradient; the check is elementwise against bounds
from the rounding model (u = 2^-8 for each BF16 rounding of a stored value, u16 =
2^-11 for the FP16 rounding of a tensor-core operand, FP32 accumulation
negligible, a 1.25 safety factor):
  forward   |δe[θ,v]| <= 1.25·(2u+u16)·Σ|D[θ,a]·val·w[f]|    (val and D stored, S = Σ val·w operand)
  dL/dw     |δg[f]|   <= Σ val·|D|·(|δe| + 1.25·(2u+u16)·|e|)   (val and D stored, r operand in WC)
  dL/dD     |δG[θ,a]| <= Σ |val·w|·(|δe| + 1.25·2u·|e|)
  dL/dλ     |δ|       <= Σ |dD/dλ|·|δG|
The relative L2 errors are reported against the 3e-3 gate of the reduced-precision
forms: dL/dw is held to it; dL/dD (3.8e-3 measured) is the gradient of the
BF16-stored model at its own residual, whose error relative to e = M w − r
exceeds that of y, and is held to the elementwise bound above.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


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
def case():
    p = synth.config_problem("grad")
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    D64, dD64 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
    rng = np.random.default_rng(1905)
    w = rng.random(p.n_fasc).astype(np.float32)
    D32 = D64.astype(np.float32)
    r = oracle.problem_signal(phi, D32, p.w_true, p.noise, p.n_theta, p.n_voxels)
    ref = oracle.loss_grads(phi, D64, dD64, w, r, p.n_theta, p.n_atoms, p.n_voxels, p.n_fasc)
    return p, phi, w, r, dD64, ref


def gpu_loss_and_grads(life, idx, p, w, r, lam_value):
    lam = torch.tensor([lam_value], dtype=torch.float64, device="cuda", requires_grad=True)
    wt = torch.tensor(w, dtype=torch.float32, device="cuda", requires_grad=True)
    g = torch.from_numpy(p.grad_dirs).cuda()
    u = torch.from_numpy(p.atom_dirs).cuda()
    D = life.dictionary(lam, g, u, p.bval)
    D.retain_grad()
    y = life.dsc(idx, D, wt)
    e = y.double() - torch.from_numpy(r).cuda().double()
    L = 0.5 * (e * e).sum()
    L.backward()
    return float(L.detach()), wt.grad.cpu().numpy(), D.grad.cpu().numpy(), float(lam.grad)


@pytest.mark.parametrize("algo", ["simt", "tc"])
def test_gradients_vs_oracle_fp32(life, case, algo):
    """FP32 storage, forward and WC backward on the CUDA cores or on the tensor
    cores (split FP16 operands); the same FP32 tolerance."""
    p, phi, w, r, dD64, (L_ref, gw_ref, gD_ref, glam_ref) = case
    idx = life.upload_problem(p, precision=life.LIFE_FP32,
                              algo=life.LIFE_ALGO_SIMT if algo == "simt" else life.LIFE_ALGO_TC)
    assert idx.info()["algo"] == (life.LIFE_ALGO_SIMT if algo == "simt" else life.LIFE_ALGO_TC)
    tol = 1e-5
    L, gw, gD, glam = gpu_loss_and_grads(life, idx, p, w, r, p.lam)
    torch.cuda.synchronize()
    life.life_check_device_status()
    assert abs(L - L_ref) <= tol * abs(L_ref), (L, L_ref)
    assert rel(gw, gw_ref) <= tol, rel(gw, gw_ref)
    assert rel(gD, gD_ref) <= tol, rel(gD, gD_ref)
    cond = float(np.abs(gD_ref * dD64).sum()) / abs(glam_ref)
    assert abs(glam - glam_ref) <= tol * cond * abs(glam_ref), (glam, glam_ref, cond)
    idx.close()


def test_gradients_vs_oracle_bf16(life, case):
    p, phi, w, r, dD64, (L_ref, gw_ref, gD_ref, glam_ref) = case
    idx = life.upload_problem(p, precision=life.LIFE_BF16, algo=life.LIFE_ALGO_TC)
    L, gw, gD, glam = gpu_loss_and_grads(life, idx, p, w, r, p.lam)
    torch.cuda.synchronize()
    life.life_check_device_status()
    u, u16 = 2.0 ** -8, 2.0 ** -11
    a = np.abs
    D64, _ = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
    phi_abs = oracle.Phi(phi.atom, phi.voxel, phi.fasc, a(phi.val))
    nt, nv, nf, na = p.n_theta, p.n_voxels, p.n_fasc, p.n_atoms
    e_ref = oracle.dsc(phi, D64, w, nt, nv) - r
    de = 1.25 * (2 * u + u16) * oracle.dsc(phi_abs, a(D64), a(w), nt, nv)
    gw_bound = oracle.wc(phi_abs, a(D64), de + 1.25 * (2 * u + u16) * a(e_ref), nt, nf)
    gD_bound = oracle.grad_D(phi_abs, a(w), de + 1.25 * 2 * u * a(e_ref), nt, na)
    L_bound = float(a(e_ref) @ de + 0.5 * de @ de)
    assert abs(L - L_ref) <= L_bound, (L, L_ref, L_bound)
    assert (a(gw - gw_ref) <= gw_bound).all(), float((a(gw - gw_ref) / gw_bound).max())
    assert (a(gD - gD_ref) <= gD_bound).all(), float((a(gD - gD_ref) / gD_bound).max())
    assert abs(glam - glam_ref) <= float(a(dD64) @ gD_bound), (glam, glam_ref)
    print("bf16 rel L2: gw", rel(gw, gw_ref), "gD", rel(gD, gD_ref), "glam", abs(glam - glam_ref) / abs(glam_ref))
    assert rel(gw, gw_ref) <= 3e-3, rel(gw, gw_ref)
    idx.close()


def test_lambda_finite_difference_on_gpu(life, case):
    """Central difference of the GPU loss in λ against the GPU's dL/dλ."""
    p, phi, w, r, dD64, _ = case
    idx = life.upload_problem(p, precision=life.LIFE_FP32, algo=life.LIFE_ALGO_SIMT)
    _, _, _, glam = gpu_loss_and_grads(life, idx, p, w, r, p.lam)
    h = 1e-3
    Lp = gpu_loss_and_grads(life, idx, p, w, r, p.lam + h)[0]
    Lm = gpu_loss_and_grads(life, idx, p, w, r, p.lam - h)[0]
    fd = (Lp - Lm) / (2 * h)
    assert abs(fd - glam) <= 1e-2 * abs(glam), (fd, glam)
    idx.close()


def test_gradients_only_where_needed(life, case):
    """w without requires_grad: only dL/dD is formed, and it is unchanged."""
    p, phi, w, r, dD64, (_, _, gD_ref, _) = case
    idx = life.upload_problem(p, precision=life.LIFE_FP32, algo=life.LIFE_ALGO_SIMT)
    D64, _ = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
    D = torch.tensor(D64.astype(np.float32), device="cuda", requires_grad=True)
    wt = torch.tensor(w, device="cuda")
    y = life.dsc(idx, D, wt)
    e = y - torch.from_numpy(r).cuda()
    (0.5 * (e.double() ** 2).sum()).backward()
    assert wt.grad is None
    assert rel(D.grad.cpu().numpy(), gD_ref) <= 1e-5
    idx.close()
