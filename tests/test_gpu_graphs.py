"""Cached CUDA graphs of the SBB-NNLS entry points (Algorithm 1 as device code).

life_sbbnnls_step replays one captured iteration; life_sbbnnls_solve replays a
conditional WHILE graph of the same iteration.  Both run the same kernels in the
same order, so k steps and a k-iteration solve from the same start agree up to
the order in which the WC's global float reductions land (one per voxel segment
or brick table, in the order the blocks finish): a few ulps after k iterations
in FP32.  With BF16 storage a weight that moves by an ulp can move the FP16
rounding of a run sum S (2^-11 relative), so the iterates agree to the BF16
path's own tolerance.
Rebuilding the layout (life_index_autotune) must drop the cached graphs: a solve
after it matches a fresh index built with the parameters it chose.
"""

TOL_FP32 = 1e-5   # relative, per weight and per FP64 scalar of the state
TOL_BF16 = 3e-3
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def life():
    import paper_1905_06234_gb300 as L
    L.load(build_if_missing=True)
    return L


def setup(life, p, precision, algo, brick_dim=0):
    idx = life.upload_problem(p, precision=precision, algo=algo, brick_dim=brick_dim)
    g = torch.from_numpy(p.grad_dirs)
    u = torch.from_numpy(p.atom_dirs)
    D, _ = life.life_dictionary(g, u, p.bval, p.lam)
    gen = torch.Generator(device="cuda").manual_seed(3)
    b = torch.rand(p.n_theta * p.n_voxels, device="cuda", generator=gen)
    return idx, D, b


def run_steps(life, idx, D, b, n, k):
    w = torch.ones(n, device="cuda")
    st, ws = life.new_sbb_state(), life.new_sbb_workspace(idx)
    for _ in range(k):
        life.life_sbbnnls_step(idx, D, b, w, st, ws)
    torch.cuda.synchronize()
    life.life_check_device_status()
    return w.cpu().numpy(), life.read_sbb_state(st)


def run_solve(life, idx, D, b, n, k):
    w = torch.ones(n, device="cuda")
    st, ws = life.new_sbb_state(), life.new_sbb_workspace(idx)
    life.life_sbbnnls_solve(idx, D, b, w, k, st, ws)
    torch.cuda.synchronize()
    life.life_check_device_status()
    return w.cpu().numpy(), life.read_sbb_state(st)


def same_run(w1, s1, w2, s2, tol):
    """Same iterate up to the order of the WC's float reductions."""
    assert s1["it"] == s2["it"] and s1["eq"] == s2["eq"] and s1["converged"] == s2["converged"]
    for k in ("alpha", "obj", "gg", "gg0", "vv", "uu"):
        assert abs(s1[k] - s2[k]) <= tol * max(abs(s1[k]), abs(s2[k]), 1e-300), (k, s1[k], s2[k])
    scale = float(np.abs(w2).max())
    assert np.allclose(w1, w2, rtol=tol, atol=tol * scale)
    assert ((w1 == 0) == (w2 == 0)).mean() > 0.99   # the same active set, bar weights at the boundary


@pytest.mark.parametrize("path", ["fp32-simt", "fp32-tc", "bf16-tc"])
def test_step_graph_matches_solve(life, path):
    p = synth.config_problem("tiny")
    prec = life.LIFE_BF16 if path == "bf16-tc" else life.LIFE_FP32
    algo = life.LIFE_ALGO_SIMT if path == "fp32-simt" else life.LIFE_ALGO_TC
    idx, D, b = setup(life, p, prec, algo)
    w1, st1 = run_steps(life, idx, D, b, p.n_fasc, 7)
    w2, st2 = run_solve(life, idx, D, b, p.n_fasc, 7)
    tol = TOL_BF16 if path == "bf16-tc" else TOL_FP32
    assert st1["it"] == 7
    same_run(w1, st1, w2, st2, tol)
    # the step graph is replayed for the same buffers, and rebuilt for new ones
    w3, st3 = run_steps(life, idx, D, b, p.n_fasc, 7)
    same_run(w1, st1, w3, st3, tol)


def test_autotune_drops_cached_graphs(life):
    p = synth.config_problem("tiny")
    idx, D, b = setup(life, p, life.LIFE_BF16, life.LIFE_ALGO_TC)
    w = torch.ones(p.n_fasc, device="cuda")
    st, ws = life.new_sbb_state(), life.new_sbb_workspace(idx)
    life.life_sbbnnls_solve(idx, D, b, w, 5, st, ws)
    life.life_sbbnnls_step(idx, D, b, w, st, ws)
    torch.cuda.synchronize()
    life.life_index_autotune(idx)           # rebuilds the tile layout
    info = idx.info()
    assert info["tuned"] == 1
    # the same buffers again, from the same start
    w.fill_(1.0)
    life.life_sbb_state_init(st)
    life.life_sbbnnls_solve(idx, D, b, w, 6, st, ws)
    life.life_sbbnnls_step(idx, D, b, w, st, ws)
    torch.cuda.synchronize()
    life.life_check_device_status()
    got_w, got_st = w.cpu().numpy(), life.read_sbb_state(st)
    # a fresh index with the layout the autotuner chose
    fresh, D2, b2 = setup(life, p, life.LIFE_BF16, life.LIFE_ALGO_TC, brick_dim=info["brick_edge"])
    assert fresh.info()["brick_edge"] == info["brick_edge"]
    w_ref = torch.ones(p.n_fasc, device="cuda")
    st_ref, ws_ref = life.new_sbb_state(), life.new_sbb_workspace(fresh)
    life.life_sbbnnls_solve(fresh, D2, b2, w_ref, 6, st_ref, ws_ref)
    life.life_sbbnnls_step(fresh, D2, b2, w_ref, st_ref, ws_ref)
    torch.cuda.synchronize()
    life.life_check_device_status()
    assert got_st["it"] == 7
    same_run(got_w, got_st, w_ref.cpu().numpy(), life.read_sbb_state(st_ref), TOL_BF16)
