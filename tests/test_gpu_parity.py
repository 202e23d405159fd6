"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances (relative L2 error against the FP64 oracle on the same float32 inputs):
FP32 path 1e-5, reduced-precision (BF16 storage) path 3e-3.  Index restructuring is
compared bit for bit.
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
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


@pytest.fixture(scope="module")
def life():
    import paper_1905_06234_gb300 as L
    L.load(build_if_missing=True)
    return L


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


class Case:
    """A problem with its oracle-side inputs (dictionary, merged Phi, signal)."""

    def __init__(self, p):
        self.p = p
        D64, dD = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
        self.D32 = D64.astype(np.float32)
        self.dD32 = dD.astype(np.float32)
        self.phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
        self.b = oracle.problem_signal(self.phi, self.D32, p.w_true, p.noise, p.n_theta, p.n_voxels)


@pytest.fixture(scope="module")
def tiny():
    return Case(synth.config_problem("tiny"))


def raw_problem(nt, na, nv, nf, nnz, seed, dup_frac=0.2, empty_frac=0.1):
    """Uniform random Phi with duplicates and some empty voxels/fascicles."""
    rng = np.random.default_rng(seed)
    live_v = rng.permutation(nv)[: max(1, int(nv * (1 - empty_frac)))]
    live_f = rng.permutation(nf)[: max(1, int(nf * (1 - empty_frac)))]
    a = rng.integers(0, na, nnz).astype(np.int32)
    v = live_v[rng.integers(0, len(live_v), nnz)].astype(np.int32)
    f = live_f[rng.integers(0, len(live_f), nnz)].astype(np.int32)
    ndup = int(nnz * dup_frac)
    if ndup and nnz > 1:
        src = rng.integers(0, nnz, ndup)
        dst = rng.integers(0, nnz, ndup)
        a[dst], v[dst], f[dst] = a[src], v[src], f[src]
    x = rng.uniform(0.5, 1.0, nnz).astype(np.float32)
    return a, v, f, x


# ------------------------------------------------------------- index build

@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_index_bit_exact_tiny(life, tiny, precision):
    p = tiny.p
    prec = life.LIFE_FP32 if precision == "fp32" else life.LIFE_BF16
    idx = life.upload_problem(p, precision=prec)
    assert idx.nnz == len(tiny.phi)
    for layout, order in ((life.LIFE_LAYOUT_VOXEL, oracle.ORDER_VOXEL), (life.LIFE_LAYOUT_FIBER, oracle.ORDER_FIBER),
                          (life.LIFE_LAYOUT_ATOM, oracle.ORDER_ATOM)):
        ref = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc, order)
        a, v, f, x = (t.cpu().numpy() for t in life.life_index_export(idx, layout))
        np.testing.assert_array_equal(a, ref.atom)
        np.testing.assert_array_equal(v, ref.voxel)
        np.testing.assert_array_equal(f, ref.fasc)
        np.testing.assert_array_equal(x.view(np.uint32), ref.val.view(np.uint32))


@pytest.mark.parametrize("shape", [(7, 5, 3, 4, 1), (96, 360, 1000, 300, 5000), (33, 4096, 70, 9, 3000),
                                   (1, 1, 1, 1, 50), (150, 31, 257, 1031, 20011)])
def test_index_bit_exact_random(life, shape):
    nt, na, nv, nf, nnz = shape
    a, v, f, x = raw_problem(nt, na, nv, nf, nnz, seed=nnz)
    idx = life.index_from_arrays(a, v, f, x, nt, na, nv, nf)
    for layout, order in ((life.LIFE_LAYOUT_VOXEL, 0), (life.LIFE_LAYOUT_FIBER, 1), (life.LIFE_LAYOUT_ATOM, 2)):
        ref = oracle.canon(a, v, f, x, na, nv, nf, order)
        ga, gv, gf, gx = (t.cpu().numpy() for t in life.life_index_export(idx, layout))
        np.testing.assert_array_equal(ga, ref.atom)
        np.testing.assert_array_equal(gv, ref.voxel)
        np.testing.assert_array_equal(gf, ref.fasc)
        np.testing.assert_array_equal(gx.view(np.uint32), ref.val.view(np.uint32))


def test_index_errors_and_empty(life):
    a = np.array([0, 5], np.int32)
    v = np.zeros(2, np.int32)
    f = np.zeros(2, np.int32)
    x = np.ones(2, np.float32)
    with pytest.raises(life.LifeError) as e:
        life.index_from_arrays(a, v, f, x, 4, 4, 1, 1)
    assert e.value.status == 2  # LIFE_ERANGE
    with pytest.raises(life.LifeError) as e:
        life.index_from_arrays(a[:1], v[:1], f[:1], np.array([np.inf], np.float32), 4, 4, 1, 1)
    assert e.value.status == 1  # LIFE_EINVAL
    idx = life.index_from_arrays(a[:0], v[:0], f[:0], x[:0], 4, 4, 3, 2)
    assert idx.nnz == 0
    D = torch.ones(16, device="cuda")
    y, ss = life.life_dsc(idx, D, torch.ones(2, device="cuda"), sumsq=True)
    g, _ = life.life_wc(idx, D, torch.ones(12, device="cuda"))
    torch.cuda.synchronize()
    assert float(y.abs().max()) == 0.0 and float(g.abs().max()) == 0.0 and float(ss) == 0.0
    # every raw entry a duplicate of one triple: merged into one coefficient
    n = 1000
    idx = life.index_from_arrays(np.full(n, 2, np.int32), np.full(n, 1, np.int32), np.full(n, 3, np.int32),
                                 np.full(n, 0.75, np.float32), 4, 4, 3, 5)
    assert idx.nnz == 1
    _, _, _, xx = life.life_index_export(idx)
    assert float(xx[0]) == 750.0


# --------------------------------------------------------------- SpMVs

def check_spmv(life, case_phi, D32, nt, na, nv, nf, idx, tol, seed=0):
    rng = np.random.default_rng(seed)
    w = rng.random(nf).astype(np.float32)
    w[rng.random(nf) < 0.3] = 0.0                      # sparse w: the zero-skip path
    r = rng.standard_normal(nt * nv).astype(np.float32)
    b = rng.standard_normal(nt * nv).astype(np.float32)
    D = dev(D32)
    y, ss = life.life_dsc(idx, D, dev(w), sumsq=True)
    e, sse = life.life_dsc(idx, D, dev(w), b=dev(b), sumsq=True)
    g, ssg = life.life_wc(idx, D, dev(r), sumsq=True)
    torch.cuda.synchronize()
    y_ref = oracle.dsc(case_phi, D32, w, nt, nv)
    g_ref = oracle.wc(case_phi, D32, r, nt, nf)
    errs = dict(y=rel(y.cpu().numpy(), y_ref), e=rel(e.cpu().numpy(), y_ref - b), g=rel(g.cpu().numpy(), g_ref))
    assert errs["y"] <= tol and errs["e"] <= tol and errs["g"] <= tol, errs
    assert abs(float(ss) - y_ref @ y_ref) <= 2 * tol * max(y_ref @ y_ref, 1e-30)
    assert abs(float(sse) - (y_ref - b) @ (y_ref - b)) <= 2 * tol * max((y_ref - b) @ (y_ref - b), 1e-30)
    assert abs(float(ssg) - g_ref @ g_ref) <= 2 * tol * max(g_ref @ g_ref, 1e-30)
    return errs


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_spmv_tiny(life, tiny, precision):
    p = tiny.p
    prec = life.LIFE_FP32 if precision == "fp32" else life.LIFE_BF16
    idx = life.upload_problem(p, precision=prec)
    tol = TOL_FP32 if precision == "fp32" else TOL_BF16
    errs = check_spmv(life, tiny.phi, tiny.D32, p.n_theta, p.n_atoms, p.n_voxels, p.n_fasc, idx, tol)
    print(precision, errs)


@pytest.mark.parametrize("shape", [(1, 1, 5, 3, 40), (31, 7, 50, 20, 700), (32, 360, 300, 100, 4000),
                                   (33, 360, 129, 77, 6000), (96, 360, 1000, 300, 30000),
                                   (150, 50, 200, 80, 9000), (96, 4096, 100, 50, 8000),
                                   (64, 600, 10, 2000, 20000)])
def test_spmv_shapes_fp32(life, shape):
    nt, na, nv, nf, nnz = shape
    a, v, f, x = raw_problem(nt, na, nv, nf, nnz, seed=nnz + nt)
    phi = oracle.canon(a, v, f, x, na, nv, nf)
    rng = np.random.default_rng(1)
    D32 = rng.standard_normal(nt * na).astype(np.float32)
    idx = life.index_from_arrays(a, v, f, x, nt, na, nv, nf)
    check_spmv(life, phi, D32, nt, na, nv, nf, idx, TOL_FP32)


def test_spmv_giant_voxel(life):
    # one voxel holds most nonzeros: the load-imbalance case
    nt, na, nv, nf = 96, 360, 64, 5000
    rng = np.random.default_rng(3)
    n = 60000
    v = np.where(rng.random(n) < 0.9, 17, rng.integers(0, nv, n)).astype(np.int32)
    a = rng.integers(0, na, n).astype(np.int32)
    f = rng.integers(0, nf, n).astype(np.int32)
    x = rng.uniform(0.5, 1, n).astype(np.float32)
    phi = oracle.canon(a, v, f, x, na, nv, nf)
    D32 = rng.standard_normal(nt * na).astype(np.float32)
    idx = life.index_from_arrays(a, v, f, x, nt, na, nv, nf)
    check_spmv(life, phi, D32, nt, na, nv, nf, idx, TOL_FP32)


def test_adjoint_and_demeaned_columns(life, tiny):
    p = tiny.p
    idx = life.upload_problem(p)
    rng = np.random.default_rng(9)
    w = rng.random(p.n_fasc).astype(np.float32)
    r = rng.standard_normal(p.n_theta * p.n_voxels).astype(np.float32)
    D = dev(tiny.D32)
    y, _ = life.life_dsc(idx, D, dev(w))
    g, _ = life.life_wc(idx, D, dev(r))
    y, g = y.double().cpu().numpy(), g.double().cpu().numpy()
    lhs, rhs = y @ r, w.astype(np.float64) @ g
    assert abs(lhs - rhs) <= 1e-5 * (np.abs(y) @ np.abs(r))
    col = y.reshape(p.n_voxels, p.n_theta).sum(axis=1)     # demeaned D: Σ_θ y = 0
    assert np.abs(col).max() <= 1e-5 * np.abs(y).max()


def test_dictionary_gpu(life, tiny):
    p = tiny.p
    D, dD = life.life_dictionary(torch.from_numpy(p.grad_dirs), torch.from_numpy(p.atom_dirs), p.bval, p.lam)
    D64, dD64 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
    assert np.abs(D.cpu().numpy() - D64).max() <= 1e-6
    assert np.abs(dD.cpu().numpy() - dD64).max() <= 1e-5


def test_grad_D(life, tiny):
    p = tiny.p
    idx = life.upload_problem(p)
    rng = np.random.default_rng(4)
    w = rng.random(p.n_fasc).astype(np.float32)
    gy = rng.standard_normal(p.n_theta * p.n_voxels).astype(np.float32)
    gD = life.life_dsc_grad_D(idx, dev(gy), dev(w))
    ref = oracle.grad_D(tiny.phi, w, gy, p.n_theta, p.n_atoms)
    assert rel(gD.cpu().numpy(), ref) <= TOL_FP32
    gD2 = life.life_dsc_grad_D(idx, dev(gy), dev(w))
    assert torch.equal(gD, gD2)                         # deterministic split, no atomics


# ----------------------------------------------------------------- SBB

def test_sbb_teacher_forced_steps(life, tiny):
    """Each GPU iteration against the oracle iteration started from the GPU's own
    iterate and state (so drift between the two trajectories cannot accumulate)."""
    p = tiny.p
    idx = life.upload_problem(p)
    D = dev(tiny.D32)
    b = dev(tiny.b)
    w = torch.ones(p.n_fasc, device="cuda")
    st = life.new_sbb_state()
    ws = life.new_sbb_workspace(idx)
    ost = oracle.SbbState()
    worst = {}
    for it in range(12):
        w_in = w.double().cpu().numpy().copy()
        prev = life.read_sbb_state(st)
        ost.s.it, ost.s.alpha, ost.s.gg0 = prev["it"], prev["alpha"], prev["gg0"]
        life.life_sbbnnls_step(idx, D, b, w, st, ws)
        torch.cuda.synchronize()
        oracle.sbb_step(tiny.phi, tiny.D32, tiny.b, w_in, p.n_theta, p.n_voxels, p.n_fasc, ost)
        gst = life.read_sbb_state(st)
        assert gst["it"] == it + 1 and gst["eq"] == ost.eq == (7 if it % 2 == 0 else 8)
        for k in ("obj", "gg", "vv", "uu", "alpha"):
            ref = getattr(ost, k)
            err = abs(gst[k] - ref) / max(abs(ref), 1e-300)
            worst[k] = max(worst.get(k, 0), err)
        worst["w"] = max(worst.get("w", 0), rel(w.cpu().numpy(), w_in))
        assert (w >= 0).all()
    print(worst)
    assert max(worst[k] for k in ("obj", "gg", "vv", "uu", "alpha")) <= 1e-4, worst
    assert worst["w"] <= 1e-4, worst


def test_sbb_solve_graph_matches_steps(life, tiny):
    p = tiny.p
    idx = life.upload_problem(p)
    D, b = dev(tiny.D32), dev(tiny.b)
    w1 = torch.ones(p.n_fasc, device="cuda")
    st1, ws1 = life.new_sbb_state(), life.new_sbb_workspace(idx)
    for _ in range(20):
        life.life_sbbnnls_step(idx, D, b, w1, st1, ws1)
    w2 = torch.ones(p.n_fasc, device="cuda")
    st2, ws2 = life.new_sbb_state(), life.new_sbb_workspace(idx)
    life.life_sbbnnls_solve(idx, D, b, w2, 20, st2, ws2)
    torch.cuda.synchronize()
    assert life.read_sbb_state(st2)["it"] == 20
    # same kernels, same order: identical up to atomic summation order in WC
    assert rel(w2.cpu().numpy(), w1.cpu().numpy()) <= 1e-5


def test_sbb_objective_vs_oracle_50_iterations(life, tiny):
    p = tiny.p
    idx = life.upload_problem(p)
    D, b = dev(tiny.D32), dev(tiny.b)
    w = torch.ones(p.n_fasc, device="cuda")
    st, ws = life.new_sbb_state(), life.new_sbb_workspace(idx)
    life.life_sbbnnls_solve(idx, D, b, w, 50, st, ws)
    torch.cuda.synchronize()
    w_ref = np.ones(p.n_fasc)
    ost = oracle.sbb_solve(tiny.phi, tiny.D32, tiny.b, w_ref, p.n_theta, p.n_voxels, p.n_fasc, 50)
    gst = life.read_sbb_state(st)
    # the last recorded objective (start of iteration 50) agrees to within trajectory drift
    assert abs(gst["obj"] - ost.obj) <= 1e-3 * ost.obj, (gst["obj"], ost.obj)
    obj0 = 0.5 * float(np.sum((oracle.dsc(tiny.phi, tiny.D32, np.ones(p.n_fasc), p.n_theta, p.n_voxels)
                               - tiny.b) ** 2))
    assert gst["obj"] < 0.2 * obj0


def test_sbb_converges_to_nnls_solution(life):
    p = synth.make_problem("small", seed=7, n_theta=16, n_atoms=30, grid=(3, 3, 3), n_fasc=8, steps=(6, 12))
    D64, _ = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
    D32 = D64.astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    rng = np.random.default_rng(4)
    wt = (rng.random(p.n_fasc) - 0.4)
    b = (oracle.dsc(phi, D32, wt, p.n_theta, p.n_voxels) + 0.05 * rng.standard_normal(p.n_theta * p.n_voxels))
    b = b.astype(np.float32)
    w_ref = np.ones(p.n_fasc)
    ost = oracle.sbb_solve(phi, D32, b, w_ref, p.n_theta, p.n_voxels, p.n_fasc, max_iter=20000, tol=1e-12)
    assert ost.converged
    idx = life.upload_problem(p)
    w = torch.ones(p.n_fasc, device="cuda")
    st, ws = life.new_sbb_state(), life.new_sbb_workspace(idx)
    life.life_sbbnnls_solve(idx, dev(D32), dev(b), w, 5000, st, ws, tol=1e-5)
    torch.cuda.synchronize()
    gst = life.read_sbb_state(st)
    assert gst["converged"] == 1, gst
    wg = w.double().cpu().numpy()
    assert np.abs(wg - w_ref).max() <= 1e-3 * max(1.0, np.abs(w_ref).max())
    assert ((wg == 0) == (w_ref == 0)).all()             # same active set


def test_sbb_converged_state_is_noop(life, tiny):
    p = tiny.p
    idx = life.upload_problem(p)
    D, b = dev(tiny.D32), dev(tiny.b)
    w = torch.ones(p.n_fasc, device="cuda")
    st, ws = life.new_sbb_state(), life.new_sbb_workspace(idx)
    life.life_sbbnnls_step(idx, D, b, w, st, ws, tol=1e9)   # any tol >= 1 stops at iteration 0
    torch.cuda.synchronize()
    s = life.read_sbb_state(st)
    assert s["converged"] == 1 and s["it"] == 0
    assert float(w.min()) == 1.0 and float(w.max()) == 1.0


# ------------------------------------------------------- failure detection

def test_bounded_wait_timeout_is_reported_and_context_survives(life, tiny):
    """A wait that can never complete gives up after its limit, the host reads
    LIFE_ETIMEOUT from the status word (which is then cleared), and the next
    SpMV on the same context is still correct.  Nothing faults."""
    life.life_check_device_status()                       # start clean
    life.life_selftest_bounded_wait(50_000_000)           # 50 ms
    with pytest.raises(life.LifeError) as ei:
        life.life_check_device_status()
    assert ei.value.status == life._native.LIFE_ETIMEOUT
    life.life_check_device_status()                       # cleared
    p = tiny.p
    idx = life.upload_problem(p)
    w = np.random.default_rng(2).random(p.n_fasc).astype(np.float32)
    y, _ = life.life_dsc(idx, dev(tiny.D32), dev(w))
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), oracle.dsc(tiny.phi, tiny.D32, w, p.n_theta, p.n_voxels)) <= TOL_FP32
    with pytest.raises(life.LifeError):
        life.life_selftest_bounded_wait(0)                # argument check
