"""Pins for the FP64 oracle, each against something other than the oracle itself:
hand-derived fixtures, closed forms, invariants, brute force and textbook routines."""
import itertools

import numpy as np
import pytest

import oracle
import synth
from tests._golden import phi_small


# ------------------------------------------------------------------ helpers

def dense_M(phi, D, nt, na, nv, nf):
    """M assembled from Eq. 4: the tensor Phi[a,v,f] contracted with D along atoms,
    giving M[(θ,v), f] with row index θ + Nθ·v."""
    Phi = np.zeros((na, nv, nf))
    np.add.at(Phi, (phi.atom, phi.voxel, phi.fasc), phi.val.astype(np.float64))
    Dm = np.asarray(D, np.float64).reshape(na, nt).T          # D[θ, a]
    M = np.einsum("ta,avf->vtf", Dm, Phi).reshape(nv * nt, nf)
    return M


def small_problem(seed=7, nt=16, na=30, grid=(3, 3, 3), nf=8, steps=(6, 12)):
    p = synth.make_problem("small", seed=seed, n_theta=nt, n_atoms=na, grid=grid, n_fasc=nf, steps=steps)
    D, dD = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    return p, D, dD, phi


# --------------------------------------------------------------- dictionary

def test_dictionary_two_direction_closed_form():
    # g = (e_z, e_x), u = (e_z): c = (1, 0) so D_raw = (exp(-bλ), 1) and the demeaned
    # column is ±(exp(-bλ) - 1)/2.
    g = np.array([[0, 0, 1.0], [1.0, 0, 0]])
    u = np.array([[0, 0, 1.0]])
    b, lam = 2.0, 1.7
    D, dD = oracle.dictionary(g, u, b, lam)
    e = np.exp(-b * lam)
    np.testing.assert_allclose(D, [(e - 1) / 2, (1 - e) / 2], rtol=1e-15)
    # d/dλ of D_raw = (-b e, 0), demeaned: (-b e / 2, +b e / 2)
    np.testing.assert_allclose(dD, [-b * e / 2, b * e / 2], rtol=1e-15)


def test_dictionary_invariants():
    g = synth.fibonacci_sphere(96)
    u = synth.fibonacci_hemisphere(360)
    np.testing.assert_allclose(np.linalg.norm(g, axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-14)
    assert (u[:, 2] > 0).all()
    D, dD = oracle.dictionary(g, u, 2.0, 1.7)
    Dm = D.reshape(360, 96)
    np.testing.assert_allclose(Dm.sum(axis=1), 0.0, atol=1e-12)          # demeaned columns
    D_flip, _ = oracle.dictionary(g, -u, 2.0, 1.7)                        # depends on |g·u| only
    np.testing.assert_array_equal(D, D_flip)
    D0, _ = oracle.dictionary(g, u, 2.0, 0.0)                            # λ = 0: all atoms flat -> 0
    np.testing.assert_allclose(D0, 0.0, atol=1e-15)
    h = 1e-5                                                             # dD/dλ vs central difference
    Dp, _ = oracle.dictionary(g, u, 2.0, 1.7 + h)
    Dn, _ = oracle.dictionary(g, u, 2.0, 1.7 - h)
    np.testing.assert_allclose(dD, (Dp - Dn) / (2 * h), atol=1e-8)


# -------------------------------------------------------------- restructuring

@pytest.mark.parametrize("order,key", [(oracle.ORDER_VOXEL, "voxel"), (oracle.ORDER_FIBER, "fiber"),
                                       (oracle.ORDER_ATOM, "atom")])
def test_canon_golden(order, key):
    G = phi_small()
    a, v, f, x = G["raw"]
    phi = oracle.canon(a, v, f, x, G["na"], G["nv"], G["nf"], order)
    ea, ev, ef, ex = G[key]
    np.testing.assert_array_equal(phi.atom, ea)
    np.testing.assert_array_equal(phi.voxel, ev)
    np.testing.assert_array_equal(phi.fasc, ef)
    np.testing.assert_array_equal(phi.val, ex)


def test_canon_invariants():
    p = synth.config_problem("tiny")
    rng = np.random.default_rng(0)
    perm = rng.permutation(p.n_raw)
    for order, keys in [(0, ("voxel", "atom", "fasc")), (1, ("fasc", "voxel", "atom")), (2, ("atom", "voxel", "fasc"))]:
        phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc, order)
        # strictly increasing lexicographic keys: sorted and duplicate-free
        k = [getattr(phi, n).astype(np.int64) for n in keys]
        big = (k[0] * (1 << 21) + k[1]) * (1 << 21) + k[2]
        assert (np.diff(big) > 0).all()
        # input order does not matter
        phi2 = oracle.canon(p.coo_atom[perm], p.coo_voxel[perm], p.coo_fasc[perm], p.coo_val[perm],
                            p.n_atoms, p.n_voxels, p.n_fasc, order)
        for n in ("atom", "voxel", "fasc", "val"):
            np.testing.assert_array_equal(getattr(phi, n), getattr(phi2, n))
    # merged values = per-triple sums of the raw values (numpy grouping, fp64, one rounding)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc, 0)
    raw_key = (p.coo_voxel.astype(np.int64) * p.n_atoms + p.coo_atom) * p.n_fasc + p.coo_fasc
    uk, inv = np.unique(raw_key, return_inverse=True)
    sums = np.zeros(len(uk))
    np.add.at(sums, inv, p.coo_val.astype(np.float64))
    got_key = (phi.voxel.astype(np.int64) * p.n_atoms + phi.atom) * p.n_fasc + phi.fasc
    np.testing.assert_array_equal(got_key, uk)
    np.testing.assert_array_equal(phi.val, sums.astype(np.float32))
    assert len(phi) < p.n_raw  # the walks do produce duplicates


def test_canon_rejects_bad_input():
    a = np.array([0, 5], np.int32)
    v = np.array([0, 0], np.int32)
    f = np.array([0, 0], np.int32)
    x = np.array([1.0, 1.0], np.float32)
    with pytest.raises(ValueError):
        oracle.canon(a, v, f, x, 4, 1, 1)
    with pytest.raises(ValueError):
        oracle.canon(a[:1], v[:1], f[:1], np.array([np.nan], np.float32), 4, 1, 1)
    phi = oracle.canon(a[:0], v[:0], f[:0], x[:0], 4, 1, 1)
    assert len(phi) == 0


# --------------------------------------------------------------------- SpMVs

def test_spmv_golden():
    G = phi_small()
    a, v, f, x = G["voxel"]
    phi = oracle.Phi(a, v, f, x)
    y = oracle.dsc(phi, G["D"], G["w"], G["nt"], G["nv"])
    np.testing.assert_array_equal(y, G["y"])
    g = oracle.wc(phi, G["D"], G["r"], G["nt"], G["nf"])
    np.testing.assert_array_equal(g, G["g"])
    # the raw list (duplicates unmerged) gives the same products: M is linear in Phi
    ra, rv, rf, rx = G["raw"]
    np.testing.assert_allclose(oracle.dsc(oracle.Phi(ra, rv, rf, rx), G["D"], G["w"], G["nt"], G["nv"]), G["y"])


def test_spmv_dense_equivalence():
    p, D, _, phi = small_problem(seed=11, nt=8, na=10, grid=(3, 3, 3), nf=8)
    M = dense_M(phi, D, p.n_theta, p.n_atoms, p.n_voxels, p.n_fasc)
    rng = np.random.default_rng(1)
    w = rng.random(p.n_fasc)
    r = rng.standard_normal(p.n_theta * p.n_voxels)
    y = oracle.dsc(phi, D, w, p.n_theta, p.n_voxels)
    g = oracle.wc(phi, D, r, p.n_theta, p.n_fasc)
    np.testing.assert_allclose(y, M @ w, rtol=1e-13, atol=1e-14 * np.abs(M @ w).max())
    np.testing.assert_allclose(g, M.T @ r, rtol=1e-13, atol=1e-13 * np.abs(M.T @ r).max())


def test_spmv_adjoint_linearity_demean():
    p = synth.config_problem("tiny")
    D, _ = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    rng = np.random.default_rng(2)
    w1, w2 = rng.random(p.n_fasc), rng.random(p.n_fasc)
    r = rng.standard_normal(p.n_theta * p.n_voxels)
    y1 = oracle.dsc(phi, D, w1, p.n_theta, p.n_voxels)
    g = oracle.wc(phi, D, r, p.n_theta, p.n_fasc)
    lhs, rhs = y1 @ r, w1 @ g
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(y1) @ np.abs(r))              # <Mw, r> = <w, M^T r>
    y2 = oracle.dsc(phi, D, w2, p.n_theta, p.n_voxels)
    y12 = oracle.dsc(phi, D, 2.0 * w1 - 3.0 * w2, p.n_theta, p.n_voxels)
    np.testing.assert_allclose(y12, 2.0 * y1 - 3.0 * y2, atol=1e-12 * np.abs(y1).max())
    # demeaned dictionary columns: each voxel's predicted signal sums to zero over θ
    col = y1.reshape(p.n_voxels, p.n_theta).sum(axis=1)
    assert np.abs(col).max() <= 1e-12 * max(1.0, np.abs(y1).max())


def test_wrapper_converts_inputs_safely():
    # float32 inputs are converted to float64 copies; those copies must stay alive
    # for the whole C call (a dangling copy once corrupted results)
    p = synth.config_problem("tiny")
    D, _ = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    D32 = D.astype(np.float32)
    w32 = np.random.default_rng(0).random(p.n_fasc).astype(np.float32)
    r32 = np.random.default_rng(1).standard_normal(p.n_theta * p.n_voxels).astype(np.float32)
    for _ in range(3):
        y1 = oracle.dsc(phi, D32, w32, p.n_theta, p.n_voxels)
        y2 = oracle.dsc(phi, D32.astype(np.float64), w32.astype(np.float64), p.n_theta, p.n_voxels)
        np.testing.assert_array_equal(y1, y2)
        g1 = oracle.wc(phi, D32, r32, p.n_theta, p.n_fasc)
        g2 = oracle.wc(phi, D32.astype(np.float64), r32.astype(np.float64), p.n_theta, p.n_fasc)
        np.testing.assert_array_equal(g1, g2)


def test_spmv_single_nonzero():
    nt, na, nv, nf = 5, 4, 3, 2
    D = np.arange(1.0, nt * na + 1.0)
    phi = oracle.Phi(np.array([2], np.int32), np.array([1], np.int32), np.array([1], np.int32),
                     np.array([0.75], np.float32))
    w = np.array([10.0, 3.0])
    y = oracle.dsc(phi, D, w, nt, nv)
    exp = np.zeros(nt * nv)
    exp[nt:2 * nt] = 0.75 * 3.0 * D[nt * 2:nt * 3]                          # y[:,1] = val w[1] D[:,2]
    np.testing.assert_array_equal(y, exp)
    r = np.arange(nt * nv, dtype=np.float64)
    g = oracle.wc(phi, D, r, nt, nf)
    np.testing.assert_allclose(g, [0.0, 0.75 * float(D[nt * 2:nt * 3] @ r[nt:2 * nt])], rtol=1e-15)


# ---------------------------------------------------------------- SBB-NNLS

def orthogonal_problem(nt=6, na=5, nf=7, seed=3):
    """Each fascicle owns one voxel with one nonzero: M has orthogonal columns,
    M^T M = diag(c^2) with c_f = val_f ‖D[:, a_f]‖."""
    rng = np.random.default_rng(seed)
    D = rng.standard_normal(nt * na)
    a = rng.integers(0, na, nf).astype(np.int32)
    v = np.arange(nf, dtype=np.int32)
    f = np.arange(nf, dtype=np.int32)
    x = rng.uniform(0.5, 1.0, nf).astype(np.float32)
    phi = oracle.Phi(a, v, f, x)
    c2 = (x.astype(np.float64) ** 2) * np.array([np.sum(D[nt * k:nt * (k + 1)] ** 2) for k in a])
    b = rng.standard_normal(nt * nf)
    Mtb = np.array([x[k] * (D[nt * a[k]:nt * (a[k] + 1)] @ b[nt * k:nt * (k + 1)]) for k in range(nf)])
    return phi, D, b, c2, Mtb, nt, nf


def test_sbb_step_closed_form_alternation():
    phi, D, b, c2, Mtb, nt, nf = orthogonal_problem()
    w = np.array([1.0, 0.0, 2.0, 0.0, 0.5, 0.0, 1.5])
    st = oracle.SbbState()
    for it, rule in [(0, 7), (1, 8), (2, 7)]:
        g = c2 * w - Mtb                                   # M^T (M w - b) with M^T M = diag(c^2)
        gt = np.where((w == 0) & (g > 0), 0.0, g)
        if rule == 7:
            alpha = (gt @ gt) / (c2 * gt @ gt)             # <g~,g~> / <Mg~,Mg~>
        else:
            alpha = (c2 * gt @ gt) / ((c2 ** 2) * gt @ gt) # <Mg~,Mg~> / <M^T M g~, M^T M g~>
        w_exp = np.maximum(w - alpha * gt, 0.0)
        oracle.sbb_step(phi, D, b, w, nt, nf, nf, st)
        assert st.eq == rule and st.it == it + 1
        np.testing.assert_allclose(st.alpha, alpha, rtol=1e-13)
        np.testing.assert_allclose(w, w_exp, rtol=1e-13, atol=1e-14)
    # the other parity reading swaps the rules
    w = np.ones(nf)
    st = oracle.SbbState()
    oracle.sbb_step(phi, D, b, w, nt, nf, nf, st, eq7_on_even=False)
    assert st.eq == 8


def test_sbb_scaled_identity_one_step_is_exact():
    # equal column norms: both rules give alpha = 1/c^2 and one step lands on the
    # NNLS solution [M^T b / c^2]_+ (Newton step for a multiple of the identity)
    nt, nf = 4, 6
    D = np.zeros(nt * 1)
    D[:] = [0.5, -0.5, 0.5, -0.5]                          # ‖D[:,0]‖ = 1
    phi = oracle.Phi(np.zeros(nf, np.int32), np.arange(nf, dtype=np.int32), np.arange(nf, dtype=np.int32),
                     np.full(nf, 0.75, np.float32))
    rng = np.random.default_rng(5)
    b = rng.standard_normal(nt * nf)
    Mtb = np.array([0.75 * (D @ b[nt * k:nt * (k + 1)]) for k in range(nf)])
    w = rng.random(nf) + 0.1
    st = oracle.SbbState()
    oracle.sbb_step(phi, D, b, w, nt, nf, nf, st)
    np.testing.assert_allclose(w, np.maximum(Mtb / 0.75 ** 2, 0.0), rtol=1e-13, atol=1e-15)


def brute_force_nnls(M, b):
    n = M.shape[1]
    best, best_w = np.inf, None
    for k in range(n + 1):
        for S in itertools.combinations(range(n), k):
            w = np.zeros(n)
            if S:
                sol, *_ = np.linalg.lstsq(M[:, S], b, rcond=None)
                if (sol < 0).any():
                    continue
                w[list(S)] = sol
            obj = 0.5 * np.sum((M @ w - b) ** 2)
            if obj < best:
                best, best_w = obj, w
    return best_w, best


def test_sbb_converges_to_exact_nnls():
    p, D, _, phi = small_problem(seed=7)
    M = dense_M(phi, D, p.n_theta, p.n_atoms, p.n_voxels, p.n_fasc)
    rng = np.random.default_rng(4)
    b = M @ (rng.random(p.n_fasc) - 0.4) + 0.05 * rng.standard_normal(M.shape[0])
    w_bf, obj_bf = brute_force_nnls(M, b)
    scipy_opt = pytest.importorskip("scipy.optimize")
    w_sp, _ = scipy_opt.nnls(M, b)
    np.testing.assert_allclose(w_sp, w_bf, atol=1e-9)
    assert (w_bf == 0).any()                               # the constraint is active somewhere
    w = np.ones(p.n_fasc)
    st = oracle.sbb_solve(phi, D, b, w, p.n_theta, p.n_voxels, p.n_fasc, max_iter=20000, tol=1e-13)
    assert st.converged
    np.testing.assert_allclose(w, w_bf, atol=1e-7 * max(1.0, np.abs(w_bf).max()))
    # KKT: w >= 0, gradient >= 0 on the boundary, complementary slackness
    grad = M.T @ (M @ w - b)
    scale = np.abs(M.T @ b).max()
    assert (w >= 0).all()
    assert (grad >= -1e-8 * scale).all()
    assert np.abs(w * grad).max() <= 1e-8 * scale * max(1.0, w.max())


# ---------------------------------------------------------------- gradients

def test_gradients_finite_differences():
    p, D, dD, phi = small_problem(seed=9, nt=12, na=20, grid=(4, 4, 4), nf=10)
    rng = np.random.default_rng(6)
    w = rng.random(p.n_fasc)
    r = rng.standard_normal(p.n_theta * p.n_voxels)
    L, gw, gD, glam = oracle.loss_grads(phi, D, dD, w, r, p.n_theta, p.n_atoms, p.n_voxels, p.n_fasc)

    def loss(wv, Dv):
        e = oracle.dsc(phi, Dv, wv, p.n_theta, p.n_voxels) - r
        return 0.5 * e @ e

    h = 1e-3
    for f in range(p.n_fasc):
        e = np.zeros(p.n_fasc)
        e[f] = h
        fd = (loss(w + e, D) - loss(w - e, D)) / (2 * h)
        assert abs(fd - gw[f]) <= 1e-8 * max(1.0, abs(gw).max())
    for idx in rng.choice(D.size, 25, replace=False):
        e = np.zeros(D.size)
        e[idx] = h
        fd = (loss(w, D + e) - loss(w, D - e)) / (2 * h)
        assert abs(fd - gD[idx]) <= 1e-8 * max(1.0, abs(gD).max())

    def loss_lam(lam):
        Dl, _ = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, lam)
        return loss(w, Dl)

    fd = (loss_lam(p.lam + h) - loss_lam(p.lam - h)) / (2 * h)
    assert abs(fd - glam) <= 1e-5 * max(1.0, abs(glam))


# ------------------------------------------------------------ evaluation


def _evaluate_golden():
    from tests._golden import read_sections
    s = read_sections("evaluate_small.txt")
    nt, nv = (int(x) for x in s["dims"][0])
    flat = lambda k: np.array([x for row in s[k] for x in row], np.float64)
    return nt, nv, s, flat


def test_voxel_rmse_golden():
    nt, nv, s, flat = _evaluate_golden()
    rmse, total = oracle.voxel_rmse(flat("e"), nt, nv)
    np.testing.assert_allclose(rmse, flat("rmse"), rtol=1e-15, atol=0)
    assert total == flat("total")[0]


def test_voxel_rmse_invariants():
    rng = np.random.default_rng(3)
    nt, nv = 7, 50
    e = rng.standard_normal(nt * nv)
    rmse, total = oracle.voxel_rmse(e, nt, nv)
    # Σ_v Nθ·rmse² is the total sum of squares; scaling e scales rmse by |k|
    assert abs(nt * (rmse ** 2).sum() - total) <= 1e-12 * total
    assert abs(total - float(e @ e)) <= 1e-12 * total
    np.testing.assert_allclose(oracle.voxel_rmse(-2.5 * e, nt, nv)[0], 2.5 * rmse, rtol=1e-14)
    # a voxel whose residual is the constant c over θ has rmse |c|
    c = np.repeat(rng.standard_normal(nv), nt)
    np.testing.assert_allclose(oracle.voxel_rmse(c, nt, nv)[0], np.abs(c[::nt]), rtol=1e-15)


def test_prune_golden():
    _, _, s, flat = _evaluate_golden()
    w = flat("w").astype(np.float32)
    for thr, key in ((0.0, "kept_t0"), (0.25, "kept_t025")):
        keep, kept = oracle.prune(w, thr)
        assert kept.tolist() == [int(x) for x in flat(key)]
        assert keep.tolist() == [1 if i in kept else 0 for i in range(w.size)]


def test_prune_invariants():
    rng = np.random.default_rng(4)
    w = rng.standard_normal(1000).astype(np.float32)
    w[rng.random(1000) < 0.3] = 0.0
    keep, kept = oracle.prune(w, 0.0)
    assert (np.diff(kept) > 0).all() and keep.sum() == kept.size
    assert (w[kept] > 0).all() and not (w[keep == 0] > 0).any()
    assert oracle.prune(np.zeros(0, np.float32))[1].size == 0


# ------------------------------------------------------- all-cores baseline


def test_omp_baseline_matches_serial_oracle():
    """The all-cores FP64 baseline (Phi grouped by voxel and by fascicle)
    reproduces the serial oracle's SpMVs and SBB iterations to FP64 rounding on the
    merged Phi, and to the float32 rounding of the merged values on the raw list
    with its repeated (a, v, f) entries."""
    p = synth.make_problem("omp", seed=1905062351, n_theta=24, n_atoms=40, grid=(6, 6, 5), n_fasc=60,
                           steps=(8, 20))
    D, _ = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    assert len(phi) < len(p.coo_atom)  # the raw list repeats some (a, v, f)
    op = oracle.OmpProblem(phi.atom, phi.voxel, phi.fasc, phi.val, p.n_theta, p.n_voxels, p.n_fasc)
    raw = oracle.OmpProblem(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_voxels, p.n_fasc)
    rng = np.random.default_rng(8)
    w = rng.random(p.n_fasc)
    r = rng.standard_normal(p.n_theta * p.n_voxels)
    y_ref = oracle.dsc(phi, D, w, p.n_theta, p.n_voxels)
    g_ref = oracle.wc(phi, D, r, p.n_theta, p.n_fasc)
    np.testing.assert_allclose(op.dsc(D, w), y_ref, rtol=1e-12, atol=1e-12 * np.abs(y_ref).max())
    np.testing.assert_allclose(op.wc(D, r), g_ref, rtol=1e-12, atol=1e-12 * np.abs(g_ref).max())
    assert np.linalg.norm(raw.dsc(D, w) - y_ref) <= 1e-7 * np.linalg.norm(y_ref)
    assert np.linalg.norm(raw.wc(D, r) - g_ref) <= 1e-7 * np.linalg.norm(g_ref)
    b = oracle.problem_signal(phi, D, p.w_true, p.noise, p.n_theta, p.n_voxels)
    w1, w2 = np.ones(p.n_fasc), np.ones(p.n_fasc)
    s1, s2 = oracle.SbbState(), oracle.SbbState()
    for _ in range(10):
        oracle.sbb_step(phi, D, b, w1, p.n_theta, p.n_voxels, p.n_fasc, s1)
        op.sbb_step(D, b, w2, s2)
    assert s1.it == s2.it == 10 and s1.eq == s2.eq
    for k in ("obj", "gg", "vv", "uu", "alpha"):
        assert abs(getattr(s1, k) - getattr(s2, k)) <= 1e-9 * abs(getattr(s1, k))
    np.testing.assert_allclose(w2, w1, rtol=1e-9, atol=1e-12)
    assert oracle.omp_threads() >= 1
