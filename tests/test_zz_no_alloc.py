"""life_dsc_grad_D_noalloc: dL/dD for callers that may not allocate device memory
while they run (code under CUDA-graph capture, allocation-free real-time loops).

It must give the allocating entry point's result, call after call, while keeping
its scratch in the library's fixed device array.  This file is collected last so
that a run stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_grad_D_noalloc_matches_allocating_call_twice():
    import paper_1905_06234_gb300 as life
    life.load(build_if_missing=True)
    p = synth.config_problem("grad")
    idx = life.upload_problem(p)
    n_sig, n_d = p.n_theta * p.n_voxels, p.n_theta * p.n_atoms
    # without the atom-sorted layout the call refuses (and allocates nothing)
    out = torch.empty(n_d, dtype=torch.float32, device="cuda")
    with pytest.raises(life.LifeError) as e:
        life.life_dsc_grad_D_noalloc(idx, torch.zeros(n_sig, device="cuda"), torch.zeros(p.n_fasc, device="cuda"),
                                     out)
    assert e.value.status == 1  # LIFE_EINVAL
    rng = np.random.default_rng(11)
    ins = [(torch.from_numpy(rng.standard_normal(n_sig).astype(np.float32)).cuda(),
            torch.from_numpy(rng.random(p.n_fasc).astype(np.float32)).cuda()) for _ in range(2)]
    # set-up: the allocating call builds the atom-sorted layout
    refs = [life.life_dsc_grad_D(idx, gy, w).clone() for gy, w in ins]
    for (gy, w), ref in zip(ins, refs):
        got = life.life_dsc_grad_D_noalloc(idx, gy, w, out)
        torch.cuda.synchronize()
        assert rel(got.cpu().numpy(), ref.cpu().numpy()) <= TOL_FP32
    # and against the FP64 oracle for the second input
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    gy, w = ins[1]
    want = oracle.grad_D(phi, w.cpu().numpy(), gy.cpu().numpy(), p.n_theta, p.n_atoms)
    assert rel(out.cpu().numpy(), want) <= TOL_FP32
    idx.close()


def test_grad_D_noalloc_rejects_oversized_scratch():
    import paper_1905_06234_gb300 as life
    life.load(build_if_missing=True)
    # 256 directions x about 6200 atom chunks (1.58M distinct entries) exceeds the 2^20-float array
    nt, na, nv, nf, n = 256, 16, 64, 4000, 2_000_000
    rng = np.random.default_rng(2)
    idx = life.index_from_arrays(rng.integers(0, na, n).astype(np.int32), rng.integers(0, nv, n).astype(np.int32),
                                 rng.integers(0, nf, n).astype(np.int32), np.ones(n, np.float32), nt, na, nv, nf)
    gy = torch.zeros(nt * nv, device="cuda")
    w = torch.zeros(nf, device="cuda")
    life.life_dsc_grad_D(idx, gy, w)
    with pytest.raises(life.LifeError) as e:
        life.life_dsc_grad_D_noalloc(idx, gy, w, torch.empty(nt * na, device="cuda"))
    assert e.value.status == 2  # LIFE_ERANGE
    idx.close()
