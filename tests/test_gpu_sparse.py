"""Sparse-w-aware DSC on the tensor-core path (the live-entry stream), through the
C ABI, against the FP64 oracle and against an index that always streams every
entry (the default; sparse_dsc enables the live-entry stream).

A zero weight contributes nothing to y = M w (Sec. 4.2.1), so a DSC whose input is
sparse may stream only the entries of fascicles with a non-zero input.  The
checks: the number of entries in the live-entry stream equals, exactly, the
number of merged Phi entries whose fascicle has a non-zero input; results stay
within the same BF16 rounding bounds as the full stream; the device-side choice
of stream (rebuild, reuse, fall back to the full stream) follows the input's
support; SBB-NNLS iterations from a sparse w agree with the oracle teacher-forced.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.test_gpu_tc import TOL_BF16, dev, rel, rounding_bounds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def life():
    import paper_1905_06234_gb300 as L
    L.load(build_if_missing=True)
    return L


@pytest.fixture(scope="module")
def case(life):
    p = synth.config_problem("tiny")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    return p, D32, phi


def tc(life, p, dense=False):
    idx = life.upload_problem(p, precision=life.LIFE_BF16, algo=life.LIFE_ALGO_TC, sparse_dsc=not dense)
    assert idx.info()["algo"] == life.LIFE_ALGO_TC
    return idx


def live_entries(phi, w):
    return int((w[phi.fasc] != 0).sum())


def check_y(life, idx, phi, D32, w, nt, nv, nf):
    y, _ = life.life_dsc(idx, dev(D32), dev(w))
    torch.cuda.synchronize()
    life.life_check_device_status()
    y = y.cpu().numpy()
    y_ref = oracle.dsc(phi, D32, w, nt, nv)
    yb, _ = rounding_bounds(phi, D32, w, np.zeros(nt * nv, np.float32), nt, nv, nf)
    assert (np.abs(y - y_ref) <= yb + 1e-30).all(), float((np.abs(y - y_ref) / (yb + 1e-30)).max())
    return y, y_ref


@pytest.mark.parametrize("zero_frac", [0.3, 0.7, 0.95])
def test_sparse_dsc_vs_oracle_and_full_stream(life, case, zero_frac):
    p, D32, phi = case
    nt, nv, nf = p.n_theta, p.n_voxels, p.n_fasc
    rng = np.random.default_rng(int(zero_frac * 100))
    w = rng.random(nf).astype(np.float32)
    w[rng.random(nf) < zero_frac] = 0.0
    idx, idx_full = tc(life, p), tc(life, p, dense=True)
    y, y_ref = check_y(life, idx, phi, D32, w, nt, nv, nf)
    y_full, _ = check_y(life, idx_full, phi, D32, w, nt, nv, nf)
    st = life.life_index_sparse_stats(idx)
    assert st["entries"] == len(phi)
    # at most 92 % of the brick-table slots non-zero: the call rebuilt and used the live stream
    assert st["rebuilds"] == 1 and st["compact_calls"] == 1, st
    assert st["live_entries"] == live_entries(phi, w), (st, live_entries(phi, w))
    assert life.life_index_sparse_stats(idx_full)["calls"] == 0
    assert rel(y, y_ref) <= TOL_BF16 and rel(y_full, y_ref) <= TOL_BF16
    # the same S values up to the association of FP32 run sums: a BF16 rounding at most
    assert rel(y, y_full) <= 2 * TOL_BF16
    idx.close()
    idx_full.close()


def test_sparse_dsc_stream_choice(life, case):
    p, D32, phi = case
    nt, nv, nf = p.n_theta, p.n_voxels, p.n_fasc
    rng = np.random.default_rng(21)
    idx = tc(life, p)
    w1 = rng.random(nf).astype(np.float32)
    w1[rng.random(nf) < 0.6] = 0.0
    check_y(life, idx, phi, D32, w1, nt, nv, nf)
    s = life.life_index_sparse_stats(idx)
    assert (s["rebuilds"], s["compact_calls"]) == (1, 1)
    # a subset of the live set, shrunk by under 10 %: reused as is
    w2 = w1.copy()
    nz = np.nonzero(w1)[0]
    w2[nz[: max(1, len(nz) // 20)]] = 0.0
    check_y(life, idx, phi, D32, w2, nt, nv, nf)
    s = life.life_index_sparse_stats(idx)
    assert (s["rebuilds"], s["compact_calls"]) == (1, 2), s
    assert s["live_entries"] == live_entries(phi, w1)
    # a fascicle outside the live set: stale, rebuilt for the new support
    w3 = w1.copy()
    z = np.nonzero((w1 == 0) & (np.bincount(phi.fasc, minlength=nf) > 0))[0]
    w3[z[0]] = 0.5
    check_y(life, idx, phi, D32, w3, nt, nv, nf)
    s = life.life_index_sparse_stats(idx)
    assert (s["rebuilds"], s["compact_calls"]) == (2, 3), s
    assert s["live_entries"] == live_entries(phi, w3)
    # a dense input streams every entry and leaves the live stream alone
    w4 = rng.random(nf).astype(np.float32) + 0.1
    check_y(life, idx, phi, D32, w4, nt, nv, nf)
    s = life.life_index_sparse_stats(idx)
    assert (s["rebuilds"], s["compact_calls"], s["calls"]) == (2, 3, 4), s
    # all-zero input: an empty live stream, y = 0 exactly
    y0, _ = life.life_dsc(idx, dev(D32), torch.zeros(nf, device="cuda"))
    torch.cuda.synchronize()
    life.life_check_device_status()
    assert float(y0.abs().max()) == 0.0
    assert life.life_index_sparse_stats(idx)["live_entries"] == 0
    # a NaN weight is live: NaN exactly where the oracle has it
    w5 = w1.copy()
    w5[int(phi.fasc[len(phi.fasc) // 2])] = np.nan
    y5, _ = life.life_dsc(idx, dev(D32), dev(w5))
    torch.cuda.synchronize()
    with np.errstate(invalid="ignore"):
        y5_ref = oracle.dsc(phi, D32, w5, nt, nv)
    np.testing.assert_array_equal(np.isnan(y5.cpu().numpy()), np.isnan(y5_ref))
    idx.close()


def test_sparse_sbb_teacher_forced(life, case):
    """SBB-NNLS from a w with 70 % zeros: the projected gradient is sparse, so the
    step's second DSC rebuilds and both DSCs stream the live entries; every step
    agrees with the oracle's step taken from the same w."""
    p, D32, phi = case
    nt, nv, nf = p.n_theta, p.n_voxels, p.n_fasc
    b = oracle.problem_signal(phi, D32, p.w_true, p.noise, nt, nv)
    rng = np.random.default_rng(5)
    w0 = p.w_true.astype(np.float32).copy()
    w0[rng.random(nf) < 0.6] = 0.0
    idx = tc(life, p)
    w = dev(w0)
    st, ws = life.new_sbb_state(), life.new_sbb_workspace(idx)
    ost = oracle.SbbState()
    worst = 0.0
    for _ in range(6):
        w_in = w.double().cpu().numpy().copy()
        prev = life.read_sbb_state(st)
        ost.s.it, ost.s.alpha, ost.s.gg0 = prev["it"], prev["alpha"], prev["gg0"]
        life.life_sbbnnls_step(idx, dev(D32), dev(b), w, st, ws)
        torch.cuda.synchronize()
        oracle.sbb_step(phi, D32, b, w_in, nt, nv, nf, ost)
        gst = life.read_sbb_state(st)
        assert gst["eq"] == ost.eq
        for k in ("obj", "gg", "vv", "alpha"):
            worst = max(worst, abs(gst[k] - getattr(ost, k)) / abs(getattr(ost, k)))
    life.life_check_device_status()
    s = life.life_index_sparse_stats(idx)
    assert s["rebuilds"] >= 1 and s["compact_calls"] >= 2, s
    assert worst <= 3e-2, worst
    idx.close()
