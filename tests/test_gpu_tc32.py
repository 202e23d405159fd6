"""GPU parity of the FP32-storage tensor-core path against the FP64 oracle.

An index built with precision LIFE_FP32 and algo LIFE_ALGO_TC keeps the Phi values
in FP32 and runs DSC on the tensor cores: D·2^kD and S·2^kS (S = Σ val·w per
(atom, voxel), summed in FP32) are split into FP16 hi and lo parts, and
Y = D_hi·S_hi + D_hi·S_lo + D_lo·S_hi is accumulated in FP32 (three MMAs per K
step of 16 atoms).  WC splits D and each tile of r the same way,
Z = D_hi·R_hi + D_hi·R_lo + D_lo·R_hi per 128-atom block and half tile, and sums
val·Z in FP32 brick tables (on the CUDA cores where D's parts and the Z slots do
not fit tensor memory: Nθ = 128 with Na > 256).  Both meet the FP32 path's
tolerance: relative L2 error <= 1e-5 against the FP64 oracle.

Per element, the DSC error is bounded by
  (3·kp/16 + 8) · 2^-23 · Σ_a |D[θ,a]| · Σ_f |val·w[f]|   (x 1.25)
(kp/16 K steps of three accumulating MMAs with at most one FP32 rounding each,
the representation errors 2^-22 of the hi/lo splits and of the dropped
D_lo·S_lo term, the FP32 run sums), plus an absolute 2^-38 · kp · max|D| ·
max|S| for parts that fall below FP16's normal range.  Per fascicle, the WC
error is bounded likewise by
  ((3·np/16 + 8) · 2^-23 + n_f · 2^-24) · Σ_k |val_k| · Σ_θ |D[θ,a_k]| |r[θ,v_k]|   (x 1.25)
(n_f: the fascicle's entries, summed in FP32), plus 2^-38 · np · max|D| · max|r|
· Σ_k |val_k|.
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
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


@pytest.fixture(scope="module")
def life():
    import paper_1905_06234_gb300 as L
    L.load(build_if_missing=True)
    return L


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def tc32_index(life, a, v, f, x, nt, na, nv, nf, ijk=None, **kw):
    idx = life.index_from_arrays(a, v, f, x, nt, na, nv, nf, voxel_ijk=ijk, precision=life.LIFE_FP32,
                                 algo=life.LIFE_ALGO_TC, **kw)
    info = idx.info()
    assert info["algo"] == life.LIFE_ALGO_TC and info["precision"] == life.LIFE_FP32
    return idx


def dsc_bound(phi, D32, w, nt, nv, na):
    kp = (na + 127) // 128 * 128
    u = 1.25 * (3 * kp / 16 + 8) * 2.0 ** -23
    a = np.abs
    yb = oracle.dsc(oracle.Phi(phi.atom, phi.voxel, phi.fasc, a(phi.val)), a(D32), a(w), nt, nv)
    # largest |S| over the (atom, voxel) cells
    key = phi.voxel.astype(np.int64) * na + phi.atom
    smax = np.bincount(key, weights=np.abs(phi.val.astype(np.float64) * w[phi.fasc])).max() if len(phi) else 0.0
    return u * yb + 2.0 ** -38 * kp * float(np.abs(D32).max()) * smax


def wc_bound(phi, D32, r, nt, nf):
    np_ = (nt + 15) // 16 * 16
    cnt = np.bincount(phi.fasc, minlength=nf).astype(np.float64)
    a = np.abs
    gb = oracle.wc(oracle.Phi(phi.atom, phi.voxel, phi.fasc, a(phi.val)), a(D32), a(r), nt, nf)
    u = 1.25 * ((3 * np_ / 16 + 8) * 2.0 ** -23 + cnt * 2.0 ** -24)
    vsum = np.bincount(phi.fasc, weights=np.abs(phi.val.astype(np.float64)), minlength=nf)
    return u * gb + 2.0 ** -38 * np_ * float(np.abs(D32).max()) * float(np.abs(r).max()) * vsum


def run_check(life, idx, phi, D32, nt, na, nv, nf, seed=0, scale=1.0, tol=TOL_FP32, l2=True, check_ss=True):
    rng = np.random.default_rng(seed)
    w = (rng.random(nf) * scale).astype(np.float32)
    w[rng.random(nf) < 0.3] = 0.0
    r = rng.standard_normal(nt * nv).astype(np.float32)
    b = (rng.standard_normal(nt * nv) * scale).astype(np.float32)
    D = dev(D32)
    y, ss = life.life_dsc(idx, D, dev(w), sumsq=True)
    e, sse = life.life_dsc(idx, D, dev(w), b=dev(b), sumsq=True)
    g, ssg = life.life_wc(idx, D, dev(r), sumsq=True)
    torch.cuda.synchronize()
    life.life_check_device_status()
    y = y.cpu().numpy()
    y_ref = oracle.dsc(phi, D32, w, nt, nv)
    g_ref = oracle.wc(phi, D32, r, nt, nf)
    yb = dsc_bound(phi, D32, w, nt, nv, na)
    assert np.isfinite(y).all()
    assert (np.abs(y - y_ref) <= yb + 1e-38).all(), float((np.abs(y - y_ref) / (yb + 1e-38)).max())
    gb = wc_bound(phi, D32, r, nt, nf)
    gg = g.cpu().numpy()
    assert (np.abs(gg - g_ref) <= gb + 1e-38).all(), float((np.abs(gg - g_ref) / (gb + 1e-38)).max())
    errs = dict(y=rel(y, y_ref), e=rel(e.cpu().numpy(), y_ref - b), g=rel(gg, g_ref))
    if l2:
        assert errs["y"] <= tol and errs["e"] <= tol and errs["g"] <= tol, errs
    if l2 and check_ss:   # squares summed in FP32 per thread first: |y| within FP32's square range
        assert abs(float(ss) - y_ref @ y_ref) <= 2 * tol * max(y_ref @ y_ref, 1e-300)
        assert abs(float(sse) - (y_ref - b) @ (y_ref - b)) <= 2 * tol * max((y_ref - b) @ (y_ref - b), 1e-300)
        assert abs(float(ssg) - g_ref @ g_ref) <= 2 * tol * max(g_ref @ g_ref, 1e-300)
    return errs


def raw_problem(nt, na, nv, nf, nnz, seed):
    rng = np.random.default_rng(seed)
    live_v = rng.permutation(nv)[: max(1, int(nv * 0.9))]
    a = rng.integers(0, na, nnz).astype(np.int32)
    v = live_v[rng.integers(0, len(live_v), nnz)].astype(np.int32)
    f = rng.integers(0, nf, nnz).astype(np.int32)
    x = rng.uniform(0.5, 1.0, nnz).astype(np.float32)
    return a, v, f, x


def test_tc32_tiny_workload(life):
    p = synth.config_problem("tiny")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    idx = tc32_index(life, p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_atoms, p.n_voxels,
                     p.n_fasc, ijk=p.voxel_ijk)
    info = idx.info()
    assert info["n_bricks"] == 8 and info["n_tiles"] == 32
    assert info["stream_bytes"] >= 8 * info["nnz"]   # FP32 values: 8 bytes per entry
    print(run_check(life, idx, phi, D32, p.n_theta, p.n_atoms, p.n_voxels, p.n_fasc))


@pytest.mark.parametrize("shape", [(96, 360, 1000, 300, 30000), (16, 7, 130, 50, 2000), (33, 64, 257, 1031, 20011),
                                   (128, 384, 300, 400, 60000), (1, 1, 5, 3, 40), (100, 256, 500, 700, 40000),
                                   (64, 100, 3000, 20000, 150000), (97, 129, 400, 300, 25000)])
def test_tc32_shapes(life, shape):
    nt, na, nv, nf, nnz = shape
    a, v, f, x = raw_problem(nt, na, nv, nf, nnz, seed=nnz + 1)
    phi = oracle.canon(a, v, f, x, na, nv, nf)
    D32 = np.random.default_rng(2).standard_normal(nt * na).astype(np.float32)
    idx = tc32_index(life, a, v, f, x, nt, na, nv, nf)
    run_check(life, idx, phi, D32, nt, na, nv, nf, l2=nt >= 8)


def test_tc32_giant_voxel_and_empty(life):
    nt, na, nv, nf = 96, 360, 700, 3000
    rng = np.random.default_rng(6)
    n = 80000
    v = np.where(rng.random(n) < 0.7, 333, rng.integers(0, 600, n)).astype(np.int32)   # voxels 600.. empty
    a = rng.integers(0, na, n).astype(np.int32)
    f = rng.integers(0, nf, n).astype(np.int32)
    x = rng.uniform(0.5, 1, n).astype(np.float32)
    phi = oracle.canon(a, v, f, x, na, nv, nf)
    D32 = rng.standard_normal(nt * na).astype(np.float32)
    idx = tc32_index(life, a, v, f, x, nt, na, nv, nf)
    run_check(life, idx, phi, D32, nt, na, nv, nf)
    idx0 = tc32_index(life, a[:0], v[:0], f[:0], x[:0], nt, na, nv, nf)
    y, ss = life.life_dsc(idx0, dev(D32), torch.ones(nf, device="cuda"), sumsq=True)
    torch.cuda.synchronize()
    life.life_check_device_status()
    assert float(y.abs().max()) == 0.0 and float(ss) == 0.0


@pytest.mark.parametrize("scale", [1e-30, 1e-12, 1e12, 1e30])
def test_tc32_operand_scales(life, scale):
    """Weights far outside FP16's range: the power-of-two scales of S (from max |w|
    and the largest run of values) and of D keep the FP32-path accuracy."""
    p = synth.config_problem("tiny")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    idx = tc32_index(life, p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_atoms, p.n_voxels,
                     p.n_fasc, ijk=p.voxel_ijk)
    run_check(life, idx, phi, D32, p.n_theta, p.n_atoms, p.n_voxels, p.n_fasc, seed=3, scale=scale,
              check_ss=False)
    # D scaled too: its own exponent moves the other way
    Ds = (D32 * np.float32(1.0 / scale ** 0.5)).astype(np.float32)
    run_check(life, idx, phi, Ds, p.n_theta, p.n_atoms, p.n_voxels, p.n_fasc, seed=4, scale=scale,
              check_ss=False)


def test_tc32_layout_values_are_fp32(life):
    """The tile stream keeps the merged FP32 values bit for bit."""
    p = synth.config_problem("tiny")
    idx = tc32_index(life, p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_atoms, p.n_voxels,
                     p.n_fasc, ijk=p.voxel_ijk)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    t = {k: v.cpu().numpy() for k, v in life.life_index_export_tiles(idx).items()}
    m = idx.info()["nnz"]
    tile_vox = t["tile_vox"]
    va = t["va"][:m].view(np.uint16).astype(np.int64)
    tile = np.repeat(np.arange(len(t["chunk_ptr"]) - 1) // (idx.info()["n_sub"] // 4), np.diff(t["chunk_ptr"]))
    vox = tile_vox[tile * 128 + (va & 127)]
    atom = va >> 7
    # each (voxel, atom) cell's values, as a multiset, are the oracle's merged ones
    got = sorted(zip(vox.tolist(), atom.tolist(), t["val"][:m].view(np.uint32).tolist()))
    ref = sorted(zip(phi.voxel.tolist(), phi.atom.tolist(), phi.val.view(np.uint32).tolist()))
    assert got == ref


def test_tc32_wc_outlier_and_non_finite(life):
    """One voxel's residual 1e5 times the rest sets its brick's R scale: the other
    voxels' values keep their precision in the hi/lo parts (per-fascicle bound and
    1e-5 hold).  A NaN and an inf in r: the fascicles through them come out
    non-finite exactly where the FP64 oracle's do (NaN where it has NaN; an
    infinite one may read NaN, since inf·D_hi + inf·D_lo cancels when the two parts
    of D differ in sign), every other one within the bound."""
    p = synth.config_problem("tiny")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    idx = tc32_index(life, p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_atoms, p.n_voxels,
                     p.n_fasc, ijk=p.voxel_ijk)
    nt, nv, nf = p.n_theta, p.n_voxels, p.n_fasc
    rng = np.random.default_rng(21)
    r = rng.standard_normal(nt * nv).astype(np.float32)
    hot = int(phi.voxel[len(phi.voxel) // 2])
    r[hot * nt:(hot + 1) * nt] *= 1e5
    g, _ = life.life_wc(idx, dev(D32), dev(r))
    torch.cuda.synchronize()
    life.life_check_device_status()
    g = g.cpu().numpy()
    g_ref = oracle.wc(phi, D32, r, nt, nf)
    gb = wc_bound(phi, D32, r, nt, nf)
    assert (np.abs(g - g_ref) <= gb + 1e-38).all(), float((np.abs(g - g_ref) / (gb + 1e-38)).max())
    assert rel(g, g_ref) <= TOL_FP32
    r = rng.standard_normal(nt * nv).astype(np.float32)
    vs = np.unique(phi.voxel)
    r[int(vs[3]) * nt + 5] = np.nan
    r[int(vs[-4]) * nt + 7] = np.inf
    g, _ = life.life_wc(idx, dev(D32), dev(r))
    torch.cuda.synchronize()
    life.life_check_device_status()
    g = g.cpu().numpy()
    with np.errstate(invalid="ignore"):
        g_ref = oracle.wc(phi, D32, r, nt, nf)
    np.testing.assert_array_equal(np.isfinite(g), np.isfinite(g_ref))
    assert np.isnan(g[np.isnan(g_ref)]).all()
    ok = np.isfinite(g_ref)
    assert 0 < (~ok).sum() < nf
    gb = wc_bound(phi, D32, np.where(np.isfinite(r), r, 0.0).astype(np.float32), nt, nf)
    # the bricks holding the NaN / inf read their r unscaled (|r| ~ 1 keeps 22 bits)
    assert (np.abs(g[ok] - g_ref[ok]) <= gb[ok] + 1e-38).all()


def test_tc32_options_rejected(life):
    a, v, f, x = raw_problem(8, 400, 10, 10, 100, seed=1)
    with pytest.raises(life.LifeError) as e:   # D's FP16 parts and the accumulator exceed tensor memory
        tc32_index(life, a, v, f, x, 8, 400, 10, 10)
    assert e.value.status == 6   # LIFE_ENOTSUP
    a, v, f, x = raw_problem(8, 40, 10, 10, 100, seed=2)
    with pytest.raises(life.LifeError) as e:   # the live-entry stream is a BF16-storage feature
        tc32_index(life, a, v, f, x, 8, 40, 10, 10, sparse_dsc=True)
    assert e.value.status == 6


def tiny_signal():
    p = synth.config_problem("tiny")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    b = oracle.problem_signal(phi, D32, p.w_true, p.noise, p.n_theta, p.n_voxels)
    return p, D32, phi, b


def test_tc32_sbb_teacher_forced(life):
    """Each iteration against the oracle's from the same iterate and state.  The
    objective and the new iterate agree to 1e-4.  The dot products of the step
    (<g~,g~>, <Mg~,Mg~>, <M^T M g~, M^T M g~>) and alpha are built from
    e = Mw - b, whose relative error is the DSC's (~3e-6 of |Mw|, eight times the
    CUDA-core kernel's: the tensor cores round the FP32 accumulator once per MMA,
    three MMAs per 16 atoms) times |Mw| / |e|, and then cancel again in M^T e:
    here a few 1e-3, gated at 1e-2."""
    p, D32, phi, b = tiny_signal()
    idx = life.upload_problem(p, precision=life.LIFE_FP32, algo=life.LIFE_ALGO_TC)
    D, bd = dev(D32), dev(b)
    w = torch.ones(p.n_fasc, device="cuda")
    st, ws = life.new_sbb_state(), life.new_sbb_workspace(idx)
    ost = oracle.SbbState()
    worst = {}
    for it in range(12):
        w_in = w.double().cpu().numpy().copy()
        prev = life.read_sbb_state(st)
        ost.s.it, ost.s.alpha, ost.s.gg0 = prev["it"], prev["alpha"], prev["gg0"]
        life.life_sbbnnls_step(idx, D, bd, w, st, ws)
        torch.cuda.synchronize()
        oracle.sbb_step(phi, D32, b, w_in, p.n_theta, p.n_voxels, p.n_fasc, ost)
        gst = life.read_sbb_state(st)
        assert gst["it"] == it + 1 and gst["eq"] == ost.eq
        for k in ("obj", "gg", "vv", "uu", "alpha"):
            ref = getattr(ost, k)
            worst[k] = max(worst.get(k, 0), abs(gst[k] - ref) / max(abs(ref), 1e-300))
        worst["w"] = max(worst.get("w", 0), rel(w.cpu().numpy(), w_in))
    life.life_check_device_status()
    print(worst)
    assert worst["obj"] <= 1e-4 and worst["w"] <= 1e-4, worst
    assert max(worst[k] for k in ("gg", "vv", "uu", "alpha")) <= 1e-2, worst


def test_tc32_converges_to_nnls_solution(life):
    p = synth.make_problem("small", seed=7, n_theta=16, n_atoms=30, grid=(3, 3, 3), n_fasc=8, steps=(6, 12))
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    rng = np.random.default_rng(4)
    wt = rng.random(p.n_fasc) - 0.4
    b = (oracle.dsc(phi, D32, wt, p.n_theta, p.n_voxels) + 0.05 * rng.standard_normal(p.n_theta * p.n_voxels))
    b = b.astype(np.float32)
    w_ref = np.ones(p.n_fasc)
    ost = oracle.sbb_solve(phi, D32, b, w_ref, p.n_theta, p.n_voxels, p.n_fasc, max_iter=20000, tol=1e-12)
    assert ost.converged
    idx = life.upload_problem(p, precision=life.LIFE_FP32, algo=life.LIFE_ALGO_TC)
    w = torch.ones(p.n_fasc, device="cuda")
    st, ws = life.new_sbb_state(), life.new_sbb_workspace(idx)
    life.life_sbbnnls_solve(idx, dev(D32), dev(b), w, 5000, st, ws, tol=1e-5)
    torch.cuda.synchronize()
    life.life_check_device_status()
    gst = life.read_sbb_state(st)
    assert gst["converged"] == 1, gst
    wg = w.double().cpu().numpy()
    assert np.abs(wg - w_ref).max() <= 1e-3 * max(1.0, np.abs(w_ref).max())
    assert ((wg == 0) == (w_ref == 0)).all()


def test_tc32_matches_simt_solve(life):
    """The tiny workload solved to 1e-4 on the FP32 tensor-core index and on the
    FP32 CUDA-core index: both converge, to the same objective within the
    tolerance's neighbourhood of the optimum."""
    p, D32, phi, b = tiny_signal()
    out = {}
    for algo in (life.LIFE_ALGO_TC, life.LIFE_ALGO_SIMT):
        idx = life.upload_problem(p, precision=life.LIFE_FP32, algo=algo)
        w = torch.ones(p.n_fasc, device="cuda")
        st, ws = life.new_sbb_state(), life.new_sbb_workspace(idx)
        life.life_sbbnnls_solve(idx, dev(D32), dev(b), w, 2000, st, ws, tol=1e-4)
        torch.cuda.synchronize()
        life.life_check_device_status()
        out[algo] = life.read_sbb_state(st)
    tc, simt = out[life.LIFE_ALGO_TC], out[life.LIFE_ALGO_SIMT]
    assert tc["converged"] == 1 and simt["converged"] == 1
    assert abs(tc["obj"] - simt["obj"]) <= 1e-3 * simt["obj"], (tc["obj"], simt["obj"])


def test_tc32_batch(life):
    """A batch of FP32 indices on the tensor-core DSC: per-problem SpMVs at 1e-5
    and a batched solve that matches the problems solved one by one."""
    probs = synth.batched_problems(4, scale=0.01)
    p0 = probs[0]
    D32 = oracle.dictionary(p0.grad_dirs, p0.atom_dirs, p0.bval, p0.lam)[0].astype(np.float32)
    nt = p0.n_theta
    phis = [oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
            for p in probs]
    idxs = [life.upload_problem(p, precision=life.LIFE_FP32, algo=life.LIFE_ALGO_TC) for p in probs]
    batch = life.life_batch_create(idxs, algo=life.LIFE_ALGO_TC)
    assert batch.info()["algo"] == life.LIFE_ALGO_TC
    rng = np.random.default_rng(8)
    ws = [rng.random(p.n_fasc).astype(np.float32) for p in probs]
    rs = [rng.standard_normal(nt * p.n_voxels).astype(np.float32) for p in probs]
    D = dev(D32)
    y, _ = life.life_dsc(batch.index, D, dev(np.concatenate(ws)))
    g, _ = life.life_wc(batch.index, D, dev(np.concatenate(rs)))
    torch.cuda.synchronize()
    life.life_check_device_status()
    y, g = y.cpu().numpy(), g.cpu().numpy()
    for k, p in enumerate(probs):
        yk = y[nt * batch.vox_off[k]:nt * batch.vox_off[k + 1]]
        gk = g[batch.fasc_off[k]:batch.fasc_off[k + 1]]
        assert rel(yk, oracle.dsc(phis[k], D32, ws[k], nt, p.n_voxels)) <= TOL_FP32
        assert rel(gk, oracle.wc(phis[k], D32, rs[k], nt, p.n_fasc)) <= TOL_FP32
    bs = [oracle.problem_signal(phis[k], D32, p.w_true, p.noise, nt, p.n_voxels) for k, p in enumerate(probs)]
    wb = [torch.ones(p.n_fasc, device="cuda") for p in probs]
    st = life.new_batch_states(len(probs))
    life.life_batch_solve(batch, D, [dev(b) for b in bs], wb, 300, st, life.new_batch_workspace(batch), tol=1e-4)
    torch.cuda.synchronize()
    life.life_check_device_status()
    sb = life.read_batch_states(st, len(probs))
    for k, p in enumerate(probs):
        w = torch.ones(p.n_fasc, device="cuda")
        s1, w1 = life.new_sbb_state(), life.new_sbb_workspace(idxs[k])
        life.life_sbbnnls_solve(idxs[k], D, dev(bs[k]), w, 300, s1, w1, tol=1e-4)
        torch.cuda.synchronize()
        ss = life.read_sbb_state(s1)
        # a batched run sums in another order (run sums split at other slot
        # boundaries, other atomic orders), so the two trajectories stop at
        # different points of the tolerance's neighbourhood of the optimum
        assert sb[k]["converged"] == ss["converged"] == 1
        assert abs(sb[k]["obj"] - ss["obj"]) <= 1e-3 * ss["obj"]
        assert rel(wb[k].cpu().numpy(), w.cpu().numpy()) <= 1e-2


def test_tc32_autotune(life):
    """The autotuner on an FP32 tensor-core index: it times brick edges and WC
    scatter groups as for BF16 storage, and the chosen layout keeps the FP32
    tolerance."""
    p = synth.config_problem("tiny")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    idx = life.upload_problem(p, precision=life.LIFE_FP32, algo=life.LIFE_ALGO_TC, autotune=True)
    info = idx.info()
    assert info["tuned"] == 1 and info["algo"] == life.LIFE_ALGO_TC and info["wc_groups"] in (1, 2, 4)
    run_check(life, idx, phi, D32, p.n_theta, p.n_atoms, p.n_voxels, p.n_fasc, seed=9)


def test_tc32_dsc_non_finite_weights(life):
    """As for BF16 storage: weights of order 1e6 with one +inf and one NaN; the
    finite outputs keep the FP32 bound, the non-finite ones match the oracle's
    (an infinite one may read NaN)."""
    p = synth.config_problem("tiny")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    idx = tc32_index(life, p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_atoms, p.n_voxels,
                     p.n_fasc, ijk=p.voxel_ijk)
    nt, nv, nf = p.n_theta, p.n_voxels, p.n_fasc
    rng = np.random.default_rng(42)
    w = (rng.random(nf) * 1e6).astype(np.float32)
    used = np.unique(phi.fasc)
    w[int(used[2])] = np.inf
    w[int(used[-3])] = np.nan
    y, _ = life.life_dsc(idx, dev(D32), dev(w))
    torch.cuda.synchronize()
    life.life_check_device_status()
    y = y.cpu().numpy()
    with np.errstate(invalid="ignore"):
        y_ref = oracle.dsc(phi, D32, w.astype(np.float64), nt, nv)
    np.testing.assert_array_equal(np.isfinite(y), np.isfinite(y_ref))
    assert np.isnan(y[np.isnan(y_ref)]).all()
    ok = np.isfinite(y_ref)
    assert 0 < (~ok).sum() < ok.size
    w0 = np.where(np.isfinite(w), w, 0.0).astype(np.float32)
    yb = dsc_bound(phi, D32, w0, nt, nv, p.n_atoms)
    assert (np.abs(y[ok] - y_ref[ok]) <= yb[ok] + 1e-30).all()
