"""Batched solve: several problems of uneven size concatenated into one
block-diagonal index and iterated together (one graph launch per solve).

Checked against (a) the FP64 oracle on each problem (index bit for bit, DSC and
WC to 1e-5 / 3e-3, SBB objective after a fixed number of iterations) and (b) the
same problems solved one after the other with life_sbbnnls_solve: the batch runs
the same kernels on the same tiles, so each problem's iteration count and
convergence must match exactly and its iterate to within summation-order drift.
The problems are the batched workload's shapes scaled down (Nf and grid edge)
so the oracle finishes in seconds.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_BF16 = 3e-3


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def life():
    import paper_1905_06234_gb300 as L
    L.load(build_if_missing=True)
    return L


class Batch:
    def __init__(self, n=5, scale=0.01):
        self.probs = synth.batched_problems(n, scale=scale)
        p0 = self.probs[0]
        D64, _ = oracle.dictionary(p0.grad_dirs, p0.atom_dirs, p0.bval, p0.lam)
        self.D32 = D64.astype(np.float32)
        self.phis, self.bs = [], []
        for p in self.probs:
            phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
            self.phis.append(phi)
            self.bs.append(oracle.problem_signal(phi, self.D32, p.w_true, p.noise, p.n_theta, p.n_voxels))


@pytest.fixture(scope="module")
def bt():
    return Batch()


def make(life, bt, precision, **kw):
    bf = precision == "bf16"
    idxs = [life.upload_problem(p, precision=life.LIFE_BF16 if bf else life.LIFE_FP32,
                                algo=life.LIFE_ALGO_TC if bf else life.LIFE_ALGO_SIMT) for p in bt.probs]
    return idxs, life.life_batch_create(idxs, **kw)


def test_batch_index_is_concatenation(life, bt):
    idxs, batch = make(life, bt, "bf16")
    info = batch.info()
    n = len(bt.probs)
    assert info["n"] == n and info["algo"] == life.LIFE_ALGO_TC
    assert batch.vox_off == list(np.cumsum([0] + [p.n_voxels for p in bt.probs]))
    assert batch.fasc_off == list(np.cumsum([0] + [p.n_fasc for p in bt.probs]))
    assert info["nnz"] == sum(len(ph) for ph in bt.phis)
    a, v, f, x = (t.cpu().numpy() for t in life.life_index_export(batch.index, life.LIFE_LAYOUT_VOXEL))
    ra = np.concatenate([ph.atom for ph in bt.phis])
    rv = np.concatenate([ph.voxel + batch.vox_off[k] for k, ph in enumerate(bt.phis)])
    rf = np.concatenate([ph.fasc + batch.fasc_off[k] for k, ph in enumerate(bt.phis)])
    rx = np.concatenate([ph.val for ph in bt.phis])
    assert np.array_equal(a, ra) and np.array_equal(v, rv) and np.array_equal(f, rf)
    assert np.array_equal(x.view(np.uint32), rx.view(np.uint32))
    # no brick mixes two problems
    t = life.life_index_export_tiles(batch.index)
    tile_vox = t["tile_vox"].cpu().numpy().reshape(-1, 128)
    btp = t["brick_tile_ptr"].cpu().numpy()
    prob_of = np.searchsorted(np.asarray(batch.vox_off), np.arange(batch.vox_off[-1]), side="right") - 1
    for b in range(len(btp) - 1):
        rows = tile_vox[btp[b]:btp[b + 1]].ravel()
        assert len(set(prob_of[rows[rows >= 0]])) == 1


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batch_spmv_per_problem(life, bt, precision):
    idxs, batch = make(life, bt, precision)
    tol = TOL_BF16 if precision == "bf16" else TOL_FP32
    rng = np.random.default_rng(55)
    nt = bt.probs[0].n_theta
    ws = [rng.random(p.n_fasc).astype(np.float32) for p in bt.probs]
    rs = [rng.standard_normal(nt * p.n_voxels).astype(np.float32) for p in bt.probs]
    D = dev(bt.D32)
    y, _ = life.life_dsc(batch.index, D, dev(np.concatenate(ws)))
    g, _ = life.life_wc(batch.index, D, dev(np.concatenate(rs)))
    torch.cuda.synchronize()
    life.life_check_device_status()
    y, g = y.cpu().numpy(), g.cpu().numpy()
    for k, p in enumerate(bt.probs):
        yk = y[nt * batch.vox_off[k]:nt * batch.vox_off[k + 1]]
        gk = g[batch.fasc_off[k]:batch.fasc_off[k + 1]]
        assert rel(yk, oracle.dsc(bt.phis[k], bt.D32, ws[k], nt, p.n_voxels)) <= tol
        assert rel(gk, oracle.wc(bt.phis[k], bt.D32, rs[k], nt, p.n_fasc)) <= tol


def batch_solve(life, batch, bt, max_iter, tol, eq7=True, w0=None, st=None, wsp=None):
    n = len(bt.probs)
    bs = [dev(b) for b in bt.bs]
    ws = w0 if w0 is not None else [torch.ones(p.n_fasc, device="cuda") for p in bt.probs]
    st = st if st is not None else life.new_batch_states(n)
    wsp = wsp if wsp is not None else life.new_batch_workspace(batch)
    life.life_batch_solve(batch, dev(bt.D32), bs, ws, max_iter, st, wsp, tol=tol, eq7_on_even=eq7)
    torch.cuda.synchronize()
    life.life_check_device_status()
    return ws, life.read_batch_states(st, n), st, wsp


def sequential_solve(life, idxs, bt, max_iter, tol, eq7=True):
    out = []
    for k, p in enumerate(bt.probs):
        w = torch.ones(p.n_fasc, device="cuda")
        st, ws = life.new_sbb_state(), life.new_sbb_workspace(idxs[k])
        life.life_sbbnnls_solve(idxs[k], dev(bt.D32), dev(bt.bs[k]), w, max_iter, st, ws, tol=tol,
                                eq7_on_even=eq7)
        torch.cuda.synchronize()
        out.append((w, life.read_sbb_state(st)))
    return out


def test_batch_solve_matches_sequential_fp32(life, bt):
    """Eight free-running iterations agree closely: same kernels, same tiles,
    same per-problem arithmetic; only the order of WC's atomic sums and of the
    FP64 partial sums differs, and that drift grows slowly over the iterations."""
    idxs, batch = make(life, bt, "fp32")
    ws, sts, _, _ = batch_solve(life, batch, bt, 8, 0.0)
    seq = sequential_solve(life, idxs, bt, 8, 0.0)
    for k in range(len(bt.probs)):
        w_ref, s_ref = seq[k]
        assert sts[k]["it"] == s_ref["it"] == 8 and sts[k]["eq"] == s_ref["eq"]
        for key in ("obj", "gg", "vv", "uu", "alpha"):
            assert abs(sts[k][key] - s_ref[key]) <= 1e-4 * abs(s_ref[key]), (k, key)
        assert rel(ws[k].cpu().numpy(), w_ref.cpu().numpy()) <= 1e-4
        assert float(ws[k].min()) >= 0.0


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batch_step_teacher_forced(life, bt, precision):
    """Each batched iteration against a single-problem iteration started from the
    batch's own iterate and state, so drift cannot accumulate.

    FP32 (CUDA cores): per-voxel sums in the same order on both sides, so only
    WC's atomic order differs.  BF16 (tensor cores): a run sum Σ val·w of one
    (atom, row) is split at 8-entry slot boundaries, which sit at different
    offsets of the combined stream than of the problem's own stream, so the FP32
    association differs and, now and then, one BF16 rounding of an S cell lands on
    the other neighbour (a 2^-8 relative change of one term of one voxel).  The
    same happens in v' = M g~ when g differs in its last bits (atomic order).
    Both results satisfy the BF16 error bounds; the bounds below allow a few such
    flips."""
    idxs, batch = make(life, bt, precision)
    bf = precision == "bf16"
    n = len(bt.probs)
    D = dev(bt.D32)
    bs = [dev(b) for b in bt.bs]
    ws = [torch.ones(p.n_fasc, device="cuda") for p in bt.probs]
    st = life.new_batch_states(n)
    wsp = life.new_batch_workspace(batch)
    single_ws = [life.new_sbb_workspace(ix) for ix in idxs]
    SB = life._native.SBB_STATE_BYTES
    for it in range(6):
        w_in = [w.clone() for w in ws]
        st_in = [st[k * SB:(k + 1) * SB].clone() for k in range(n)]
        life.life_batch_solve(batch, D, bs, ws, 1, st, wsp)
        for k in range(n):
            life.life_sbbnnls_step(idxs[k], D, bs[k], w_in[k], st_in[k], single_ws[k])
        torch.cuda.synchronize()
        got = life.read_batch_states(st, n)
        for k in range(n):
            ref = life.read_sbb_state(st_in[k])
            assert got[k]["it"] == ref["it"] == it + 1 and got[k]["eq"] == ref["eq"]
            for key in ("obj", "gg"):
                tol = 2e-4 if bf else 1e-6
                assert abs(got[k][key] - ref[key]) <= tol * abs(ref[key]), (it, k, key, got[k][key], ref[key])
            for key in ("vv", "uu", "alpha"):
                tol = 5e-3 if bf else 1e-5
                assert abs(got[k][key] - ref[key]) <= tol * abs(ref[key]), (it, k, key, got[k][key], ref[key])
            assert rel(ws[k].cpu().numpy(), w_in[k].cpu().numpy()) <= (5e-3 if bf else 1e-5)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batch_staggered_convergence(life, bt, precision):
    """Problems stop on their own (‖g~‖ <= 1e-3·‖g~_0‖) at different iterations
    while the others go on, and a stopped problem stays frozen.  On the FP32 path
    each stop and objective agree with the problem solved alone.  With BF16
    storage two runs drift apart through WC's atomic sums and single BF16
    roundings, and the non-monotone BB iteration (Eq. 7/8) reaches the threshold
    at a different point of its oscillation, so there only the stopping rule
    itself is checked."""
    idxs, batch = make(life, bt, precision)
    bf = precision == "bf16"
    ws, sts, st, wsp = batch_solve(life, batch, bt, 300, 1e-3)
    its = [s["it"] for s in sts]
    assert all(s["converged"] == 1 for s in sts) and len(set(its)) > 1, its
    w_before = [w.clone() for w in ws]
    st_before = st.clone()
    ws2, _, st2, _ = batch_solve(life, batch, bt, 10, 1e-3, w0=ws, st=st, wsp=wsp)
    assert all(torch.equal(x, y) for x, y in zip(ws2, w_before)) and torch.equal(st2, st_before)
    seq = sequential_solve(life, idxs, bt, 300, 1e-3)
    for k in range(len(bt.probs)):
        w_ref, s_ref = seq[k]
        assert s_ref["converged"] == 1
        assert np.sqrt(sts[k]["gg"]) <= 1e-3 * np.sqrt(sts[k]["gg0"]) and sts[k]["eq"] == 0
        if bf:
            print("bf16 stop", k, sts[k]["it"], s_ref["it"], sts[k]["obj"], s_ref["obj"])
        else:
            assert abs(sts[k]["it"] - s_ref["it"]) <= 1, (k, sts[k]["it"], s_ref["it"])
            assert abs(sts[k]["obj"] - s_ref["obj"]) <= 1e-4 * s_ref["obj"], (k, sts[k]["obj"], s_ref["obj"])
        assert float(ws[k].min()) >= 0.0


def test_batch_eq8_first_reading(life, bt):
    idxs, batch = make(life, bt, "fp32")
    ws, sts, _, _ = batch_solve(life, batch, bt, 9, 0.0, eq7=False)
    seq = sequential_solve(life, idxs, bt, 9, 0.0, eq7=False)
    for k in range(len(bt.probs)):
        assert sts[k]["it"] == 9 and sts[k]["eq"] == 8 == seq[k][1]["eq"]
        assert rel(ws[k].cpu().numpy(), seq[k][0].cpu().numpy()) <= 1e-4


def test_batch_solve_vs_oracle(life, bt):
    idxs, batch = make(life, bt, "fp32")
    ws, sts, _, _ = batch_solve(life, batch, bt, 30, 0.0)
    for k, p in enumerate(bt.probs):
        w_ref = np.ones(p.n_fasc)
        ost = oracle.sbb_solve(bt.phis[k], bt.D32, bt.bs[k], w_ref, p.n_theta, p.n_voxels, p.n_fasc, 30)
        assert sts[k]["it"] == 30
        assert abs(sts[k]["obj"] - ost.obj) <= 1e-3 * ost.obj, (k, sts[k]["obj"], ost.obj)


def test_batch_max_iter_and_continuation(life, bt):
    idxs, batch = make(life, bt, "fp32")
    ws, sts, st, wsp = batch_solve(life, batch, bt, 7, 0.0)
    assert all(s["it"] == 7 for s in sts)
    ws, sts, _, _ = batch_solve(life, batch, bt, 5, 0.0, w0=ws, st=st, wsp=wsp)
    assert all(s["it"] == 12 for s in sts)
    seq = sequential_solve(life, idxs, bt, 12, 0.0)
    for k in range(len(bt.probs)):
        assert rel(ws[k].cpu().numpy(), seq[k][0].cpu().numpy()) <= 1e-4


def test_batch_errors(life, bt):
    idx_a = life.upload_problem(bt.probs[0])
    p = bt.probs[1]
    idx_b = life.index_from_arrays(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, 64, p.n_atoms, p.n_voxels,
                                   p.n_fasc)
    with pytest.raises(life.LifeError):
        life.life_batch_create([idx_a, idx_b])          # different Nθ
    with pytest.raises(life.LifeError):
        life.life_batch_create([])


def test_autotune_index_and_batch(life, bt):
    p = synth.config_problem("tiny")
    idx = life.upload_problem(p, precision=life.LIFE_BF16, algo=life.LIFE_ALGO_TC)
    info = life.life_index_autotune(idx)
    assert info["tuned"] == 1 and info["wc_groups"] in (1, 2, 4) and 1 <= info["brick_edge"] <= 12
    D64, _ = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
    D32 = D64.astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    rng = np.random.default_rng(8)
    w = rng.random(p.n_fasc).astype(np.float32)
    r = rng.standard_normal(p.n_theta * p.n_voxels).astype(np.float32)
    y, _ = life.life_dsc(idx, dev(D32), dev(w))
    g, _ = life.life_wc(idx, dev(D32), dev(r))
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), oracle.dsc(phi, D32, w, p.n_theta, p.n_voxels)) <= TOL_BF16
    assert rel(g.cpu().numpy(), oracle.wc(phi, D32, r, p.n_theta, p.n_fasc)) <= TOL_BF16
    idxs, batch = make(life, bt, "bf16", autotune=True)
    binfo = batch.info()
    assert binfo["tuned"] == 1 and binfo["wc_groups"] in (1, 2, 4)
    # the tuned combined layout still computes every problem's DSC and WC
    nt = bt.probs[0].n_theta
    ws_ = [rng.random(p.n_fasc).astype(np.float32) for p in bt.probs]
    rs_ = [rng.standard_normal(nt * p.n_voxels).astype(np.float32) for p in bt.probs]
    y, _ = life.life_dsc(batch.index, dev(bt.D32), dev(np.concatenate(ws_)))
    g, _ = life.life_wc(batch.index, dev(bt.D32), dev(np.concatenate(rs_)))
    torch.cuda.synchronize()
    y, g = y.cpu().numpy(), g.cpu().numpy()
    for k, q in enumerate(bt.probs):
        yk = y[nt * batch.vox_off[k]:nt * batch.vox_off[k + 1]]
        gk = g[batch.fasc_off[k]:batch.fasc_off[k + 1]]
        assert rel(yk, oracle.dsc(bt.phis[k], bt.D32, ws_[k], nt, q.n_voxels)) <= TOL_BF16
        assert rel(gk, oracle.wc(bt.phis[k], bt.D32, rs_[k], nt, q.n_fasc)) <= TOL_BF16
    # and the solve on it: two iterations agree with the problems solved alone
    ws, sts, _, _ = batch_solve(life, batch, bt, 2, 0.0)
    seq = sequential_solve(life, idxs, bt, 2, 0.0)
    for k in range(len(bt.probs)):
        assert abs(sts[k]["obj"] - seq[k][1]["obj"]) <= 1e-3 * seq[k][1]["obj"]
