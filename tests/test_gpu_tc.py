"""GPU parity of the tensor-core (BF16-storage) path against the FP64 oracle.

Tolerance: relative L2 error <= 3e-3 for the reduced-precision path (Φ values and D
stored in BF16; the tensor-core operands S / r tiles and D in FP16 under exact
power-of-two scales; accumulation FP32; reductions FP64).
Every call is followed by a device-status check, so a bounded wait that gave up
inside a kernel fails the test instead of passing silently.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_BF16 = 3e-3
U_BF16 = 2.0 ** -8   # unit roundoff of BF16 (8 significand bits, round to nearest)
U_F16 = 2.0 ** -11   # unit roundoff of FP16 (11 significand bits)
U_TC = 2 * U_BF16 + U_F16   # per result: two BF16 roundings (Phi value, D) and one FP16 (S or r)


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


def tc_index(life, a, v, f, x, nt, na, nv, nf, ijk=None):
    idx = life.index_from_arrays(a, v, f, x, nt, na, nv, nf, voxel_ijk=ijk, precision=life.LIFE_BF16,
                                 algo=life.LIFE_ALGO_TC)
    assert idx.info()["algo"] == life.LIFE_ALGO_TC
    return idx


def rounding_bounds(phi, D32, w, r, nt, nv, nf):
    """First-order bounds on |GPU - exact| per output element.  DSC rounds the Phi
    value and D to BF16 (stored precision) and S = sum val*w to FP16 (the MMA
    operand): |err| <= (2u + u16) sum|D||val w|.  WC rounds the value and D to BF16
    and r to FP16: |err| <= (2u + u16) sum_k |val| sum_t |D||r|.  The FP16 operand
    scales are exact powers of two; FP32 accumulation adds far less and is covered
    by the factor 1.25."""
    a = np.abs
    yb = oracle.dsc(oracle.Phi(phi.atom, phi.voxel, phi.fasc, a(phi.val)), a(D32), a(w), nt, nv)
    gb = oracle.wc(oracle.Phi(phi.atom, phi.voxel, phi.fasc, a(phi.val)), a(D32), a(r), nt, nf)
    return 1.25 * U_TC * yb, 1.25 * U_TC * gb


def run_check(life, idx, phi, D32, nt, nv, nf, seed=0, tol=TOL_BF16, elementwise=False):
    rng = np.random.default_rng(seed)
    w = rng.random(nf).astype(np.float32)
    w[rng.random(nf) < 0.3] = 0.0
    r = rng.standard_normal(nt * nv).astype(np.float32)
    b = rng.standard_normal(nt * nv).astype(np.float32)
    D = dev(D32)
    y, ss = life.life_dsc(idx, D, dev(w), sumsq=True)
    e, _ = life.life_dsc(idx, D, dev(w), b=dev(b))
    g, ssg = life.life_wc(idx, D, dev(r), sumsq=True)
    torch.cuda.synchronize()
    life.life_check_device_status()
    y_ref = oracle.dsc(phi, D32, w, nt, nv)
    g_ref = oracle.wc(phi, D32, r, nt, nf)
    errs = dict(y=rel(y.cpu().numpy(), y_ref), e=rel(e.cpu().numpy(), y_ref - b), g=rel(g.cpu().numpy(), g_ref),
                ss=abs(float(ss) - y_ref @ y_ref) / max(y_ref @ y_ref, 1e-30),
                ssg=abs(float(ssg) - g_ref @ g_ref) / max(g_ref @ g_ref, 1e-30))
    yb, gb = rounding_bounds(phi, D32, w, r, nt, nv, nf)
    assert (np.abs(y.cpu().numpy() - y_ref) <= yb + 1e-30).all()
    assert (np.abs(g.cpu().numpy() - g_ref) <= gb + 1e-30).all()
    if elementwise:   # degenerate shapes: too few terms for the statistical L2 bound
        return errs
    assert errs["y"] <= tol and errs["e"] <= tol and errs["g"] <= tol, errs
    assert errs["ss"] <= 2 * tol and errs["ssg"] <= 2 * tol, errs
    return errs


def test_tc_tiny_workload(life):
    p = synth.config_problem("tiny")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    idx = tc_index(life, p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_atoms, p.n_voxels,
                   p.n_fasc, ijk=p.voxel_ijk)
    info = idx.info()
    assert info["n_bricks"] == 8 and info["n_tiles"] == 32   # 16^3 grid in 8^3 bricks of 4 tiles
    print(run_check(life, idx, phi, D32, p.n_theta, p.n_voxels, p.n_fasc))


def raw_problem(nt, na, nv, nf, nnz, seed):
    rng = np.random.default_rng(seed)
    live_v = rng.permutation(nv)[: max(1, int(nv * 0.9))]
    a = rng.integers(0, na, nnz).astype(np.int32)
    v = live_v[rng.integers(0, len(live_v), nnz)].astype(np.int32)
    f = rng.integers(0, nf, nnz).astype(np.int32)
    x = rng.uniform(0.5, 1.0, nnz).astype(np.float32)
    return a, v, f, x


@pytest.mark.parametrize("shape", [(96, 360, 1000, 300, 30000), (16, 7, 130, 50, 2000), (33, 64, 257, 1031, 20011),
                                   (128, 512, 300, 400, 60000), (1, 1, 5, 3, 40), (64, 100, 3000, 20000, 150000)])
def test_tc_shapes(life, shape):
    nt, na, nv, nf, nnz = shape
    a, v, f, x = raw_problem(nt, na, nv, nf, nnz, seed=nnz)
    phi = oracle.canon(a, v, f, x, na, nv, nf)
    D32 = np.random.default_rng(1).standard_normal(nt * na).astype(np.float32)
    idx = tc_index(life, a, v, f, x, nt, na, nv, nf)
    run_check(life, idx, phi, D32, nt, nv, nf, elementwise=nt < 8)


def test_tc_giant_voxel_and_empty(life):
    nt, na, nv, nf = 96, 360, 700, 3000
    rng = np.random.default_rng(5)
    n = 80000
    v = np.where(rng.random(n) < 0.7, 333, rng.integers(0, 600, n)).astype(np.int32)   # voxels 600.. empty
    a = rng.integers(0, na, n).astype(np.int32)
    f = rng.integers(0, nf, n).astype(np.int32)
    x = rng.uniform(0.5, 1, n).astype(np.float32)
    phi = oracle.canon(a, v, f, x, na, nv, nf)
    D32 = rng.standard_normal(nt * na).astype(np.float32)
    idx = tc_index(life, a, v, f, x, nt, na, nv, nf)
    run_check(life, idx, phi, D32, nt, nv, nf)
    # an index with no entries at all
    idx0 = tc_index(life, a[:0], v[:0], f[:0], x[:0], nt, na, nv, nf)
    y, _ = life.life_dsc(idx0, dev(D32), torch.ones(nf, device="cuda"))
    g, _ = life.life_wc(idx0, dev(D32), torch.ones(nt * nv, device="cuda"))
    torch.cuda.synchronize()
    life.life_check_device_status()
    assert float(y.abs().max()) == 0.0 and float(g.abs().max()) == 0.0


def test_tc_matches_simt_bf16_values(life):
    """Same BF16-rounded Φ values on both paths: the remaining difference is the
    BF16 rounding of D and the FP16 rounding of the on-chip S / r tiles."""
    p = synth.config_problem("tiny")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    i_tc = tc_index(life, p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_atoms, p.n_voxels,
                    p.n_fasc, ijk=p.voxel_ijk)
    i_st = life.upload_problem(p, precision=life.LIFE_BF16, algo=life.LIFE_ALGO_SIMT)
    w = dev(p.w_true)
    y1, _ = life.life_dsc(i_tc, dev(D32), w)
    y2, _ = life.life_dsc(i_st, dev(D32), w)
    torch.cuda.synchronize()
    assert rel(y1.cpu().numpy(), y2.cpu().numpy()) <= TOL_BF16


@pytest.mark.parametrize("outlier", [False, True])
def test_tc_sbb_teacher_forced(life, outlier):
    """outlier: one voxel's signal 1e4 times larger, so the residual of one brick
    spans four more decades; both WCs of the step size their fixed-point tables
    from the per-tile maxima that the preceding DSC wrote, and must still agree.
    Four iterations there: from the fifth on, the projected gradient of this
    case cancels so strongly that BF16 storage alone (FP32 tables as well)
    moves <g~, g~> by several per cent."""
    p = synth.config_problem("tiny")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    b = oracle.problem_signal(phi, D32, p.w_true, p.noise, p.n_theta, p.n_voxels)
    if outlier:
        hot = int(phi.voxel[len(phi.voxel) // 3])
        b[hot * p.n_theta:(hot + 1) * p.n_theta] *= 1e4
    idx = tc_index(life, p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_atoms, p.n_voxels,
                   p.n_fasc, ijk=p.voxel_ijk)
    w = torch.ones(p.n_fasc, device="cuda")
    st, ws = life.new_sbb_state(), life.new_sbb_workspace(idx)
    ost = oracle.SbbState()
    worst = 0.0
    for it in range(4 if outlier else 6):
        w_in = w.double().cpu().numpy().copy()
        prev = life.read_sbb_state(st)
        ost.s.it, ost.s.alpha, ost.s.gg0 = prev["it"], prev["alpha"], prev["gg0"]
        life.life_sbbnnls_step(idx, dev(D32), dev(b), w, st, ws)
        torch.cuda.synchronize()
        oracle.sbb_step(phi, D32, b, w_in, p.n_theta, p.n_voxels, p.n_fasc, ost)
        gst = life.read_sbb_state(st)
        assert gst["eq"] == ost.eq
        for k in ("obj", "gg", "vv", "alpha"):
            worst = max(worst, abs(gst[k] - getattr(ost, k)) / abs(getattr(ost, k)))
    life.life_check_device_status()
    # g carries the BF16 error of WC plus the DSC error of e = Mw - b amplified by
    # |Mw| / |e|; <g~,g~> doubles the relative error: a few times 3e-3
    assert worst <= 3e-2, worst


def expected_tiles(phi, tile_vox, brick_tile_ptr, nv, n_sub):
    """The tile layout the restructuring must produce, rebuilt on the host from the
    oracle's merged Phi and the library's voxel -> (tile, row) assignment."""
    n_tiles = len(tile_vox) // 128
    vox_tile = np.full(nv, -1, np.int64)
    vox_row = np.full(nv, -1, np.int64)
    for t in range(n_tiles):
        for r in range(128):
            v = tile_vox[128 * t + r]
            if v >= 0:
                assert vox_tile[v] == -1, "voxel placed twice"
                vox_tile[v], vox_row[v] = t, r
    assert (vox_tile >= 0).all(), "voxel missing from the tiles"
    tile_brick = np.repeat(np.arange(len(brick_tile_ptr) - 1), np.diff(brick_tile_ptr))
    t = vox_tile[phi.voxel]
    row = vox_row[phi.voxel]
    a = phi.atom.astype(np.int64)
    f = phi.fasc.astype(np.int64)
    # inside a 128-atom chunk, cells in the order of their place in the S operand:
    # (row / 8, atom mod 128 / 8, row mod 8, atom mod 8)
    cell = ((a >> 7) << 14) | ((row >> 3) << 10) | (((a >> 3) & 15) << 6) | ((row & 7) << 3) | (a & 7)
    order = np.lexsort((f, cell, t))
    t, row, a, f, val = t[order], row[order], a[order], f[order], phi.val[order]
    va = (row | (a << 7)).astype(np.uint16)
    b = tile_brick[t]
    bfk = np.unique(b * (1 << 32) + f)
    bptr = np.searchsorted(bfk >> 32, np.arange(len(brick_tile_ptr)))
    local = np.searchsorted(bfk, b * (1 << 32) + f) - bptr[b]
    cont = np.zeros(len(t), bool)
    cont[1:] = (t[1:] == t[:-1]) & (a[1:] == a[:-1]) & (row[1:] == row[:-1])
    fl = (local | np.where(cont, 0x8000, 0)).astype(np.uint16)
    n_c = n_sub // 4
    seg = t * n_c + (a >> 7)
    chunk_ptr = np.searchsorted(seg, np.arange(n_tiles * n_c + 1))
    import torch as _t
    valb = _t.from_numpy(val).to(_t.bfloat16).float().numpy()
    return dict(va=va, fl=fl, val=valb, brick_fasc_ptr=bptr.astype(np.int32), brick_fasc=(bfk & 0xffffffff).astype(np.int32),
                chunk_ptr=chunk_ptr.astype(np.int32))


@pytest.mark.parametrize("use_ijk", [False, True])
def test_tc_layout_bit_exact(life, use_ijk):
    p = synth.config_problem("tiny")
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    idx = tc_index(life, p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_atoms, p.n_voxels,
                   p.n_fasc, ijk=p.voxel_ijk if use_ijk else None)
    info = idx.info()
    got = {k: v.cpu().numpy() for k, v in life.life_index_export_tiles(idx).items()}
    m = info["nnz"]
    exp = expected_tiles(phi, got["tile_vox"], got["brick_tile_ptr"], p.n_voxels, info["n_sub"])
    np.testing.assert_array_equal(got["chunk_ptr"], exp["chunk_ptr"])
    np.testing.assert_array_equal(got["va"][:m].view(np.uint16), exp["va"])
    np.testing.assert_array_equal(got["val"][:m], exp["val"])
    np.testing.assert_array_equal(got["brick_fasc_ptr"], exp["brick_fasc_ptr"])
    np.testing.assert_array_equal(got["brick_fasc"][:info["n_brick_fasc"]], exp["brick_fasc"])
    np.testing.assert_array_equal(got["fl"][:m].view(np.uint16), exp["fl"])
    assert sorted(got["brick_order"][:info["n_bricks"]]) == list(range(info["n_bricks"]))
    if use_ijk:   # every brick's voxels lie in one spatial cube of the stated edge
        B = info["brick_edge"]
        for bi in range(info["n_bricks"]):
            tv = got["tile_vox"][128 * got["brick_tile_ptr"][bi]:128 * got["brick_tile_ptr"][bi + 1]]
            ijk = p.voxel_ijk[tv[tv >= 0]] // B
            assert (ijk == ijk[0]).all()


def fixed_point_bound(phi, D32, r, tile_vox, brick_tile_ptr, nt, nv, nf):
    """Per-fascicle bound on the extra error of WC's fixed-point brick tables.

    Each entry's product val*Z is rounded to a multiple of the brick's unit
    2^(e-29), where bnd = cnt * vmax * d1 * rmax < 2^e is the brick's bound on any
    fascicle's sum (cnt: most entries of one fascicle in the brick, vmax: largest
    |val|, d1: largest column sum of |D| in BF16, rmax: largest |r| over the
    brick's voxels).  Half a unit is below 2^-29 * bnd, once per entry."""
    import torch as _t
    tile_brick = np.repeat(np.arange(len(brick_tile_ptr) - 1), np.diff(brick_tile_ptr))
    vox_brick = np.full(nv, -1, np.int64)
    rows = np.nonzero(tile_vox >= 0)[0]
    vox_brick[tile_vox[rows]] = tile_brick[rows // 128]
    nb = len(brick_tile_ptr) - 1
    eb = vox_brick[phi.voxel]
    valb = np.abs(_t.from_numpy(phi.val).to(_t.bfloat16).float().numpy()).astype(np.float64)
    Db = np.abs(_t.from_numpy(D32).to(_t.bfloat16).float().numpy()).astype(np.float64).reshape(-1, nt)
    d1 = Db.sum(axis=1).max()
    cnt = np.zeros(nb)
    key, c = np.unique(eb * (nf + 1) + phi.fasc, return_counts=True)
    np.maximum.at(cnt, key // (nf + 1), c)
    vmax = np.zeros(nb)
    np.maximum.at(vmax, eb, valb)
    rmax = np.zeros(nb)
    placed = vox_brick >= 0
    np.maximum.at(rmax, vox_brick[placed], np.abs(r.reshape(nv, nt)[placed]).max(axis=1).astype(np.float64))
    bnd = cnt * vmax * d1 * rmax
    return np.bincount(phi.fasc, weights=2.0 ** -29 * bnd[eb], minlength=nf)


def tiny_case(life):
    p = synth.config_problem("tiny")
    D32 = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)[0].astype(np.float32)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    idx = tc_index(life, p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_atoms, p.n_voxels,
                   p.n_fasc, ijk=p.voxel_ijk)
    return p, D32, phi, idx


def test_wc_fixed_point_outlier(life):
    """One voxel's residual 1e5 times the rest: that brick's fixed-point unit is
    set by the outlier, and every fascicle still lands within the BF16 rounding
    bound plus the fixed-point bound (a scale that overflowed the int32 tables or
    was too coarse would break it)."""
    p, D32, phi, idx = tiny_case(life)
    nt, nv, nf = p.n_theta, p.n_voxels, p.n_fasc
    rng = np.random.default_rng(11)
    r = rng.standard_normal(nt * nv).astype(np.float32)
    hot = int(phi.voxel[len(phi.voxel) // 2])
    r[hot * nt:(hot + 1) * nt] *= 1e5
    g, _ = life.life_wc(idx, dev(D32), dev(r))
    torch.cuda.synchronize()
    life.life_check_device_status()
    g = g.cpu().numpy()
    g_ref = oracle.wc(phi, D32, r, nt, nf)
    tiles = {k: v.cpu().numpy() for k, v in life.life_index_export_tiles(idx).items()}
    n_tiles = idx.info()["n_tiles"]
    fxb = fixed_point_bound(phi, D32, r, tiles["tile_vox"][:128 * n_tiles], tiles["brick_tile_ptr"], nt, nv, nf)
    _, gb = rounding_bounds(phi, D32, np.zeros(nf, np.float32), r, nt, nv, nf)
    assert (np.abs(g - g_ref) <= gb + fxb + 1e-30).all(), float((np.abs(g - g_ref) / (gb + fxb + 1e-30)).max())
    assert rel(g, g_ref) <= TOL_BF16


def test_wc_non_finite_residual(life):
    """A NaN in one voxel's residual and +inf in another's: the fascicles through
    them come out NaN / infinite exactly as in the FP64 oracle (their bricks keep
    FP32 tables), and every other fascicle stays within the rounding bound."""
    p, D32, phi, idx = tiny_case(life)
    nt, nv, nf = p.n_theta, p.n_voxels, p.n_fasc
    rng = np.random.default_rng(12)
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
    np.testing.assert_array_equal(np.isnan(g), np.isnan(g_ref))
    np.testing.assert_array_equal(np.isposinf(g), np.isposinf(g_ref))
    np.testing.assert_array_equal(np.isneginf(g), np.isneginf(g_ref))
    ok = np.isfinite(g_ref)
    assert 0 < (~ok).sum() < nf
    r0 = np.where(np.isfinite(r), r, 0.0).astype(np.float32)
    _, gb = rounding_bounds(phi, D32, np.zeros(nf, np.float32), r0, nt, nv, nf)
    assert (np.abs(g[ok] - g_ref[ok]) <= gb[ok] + 1e-30).all()


@pytest.mark.parametrize("scale", [1e-30, 1e-12, 1e12, 1e30])
def test_tc_operand_scales(life, scale):
    """The FP16 tensor-core operands carry exact power-of-two scales chosen per call
    (S, from max |w|) and per brick (the r tile, from its max |r|): weights and
    residuals far outside FP16's range give the same relative accuracy as at unit
    scale, and the results scale exactly with the inputs up to rounding."""
    p, D32, phi, idx = tiny_case(life)
    nt, nv, nf = p.n_theta, p.n_voxels, p.n_fasc
    rng = np.random.default_rng(31)
    w = (rng.random(nf) * scale).astype(np.float32)
    w[rng.random(nf) < 0.3] = 0.0
    r = (rng.standard_normal(nt * nv) * scale).astype(np.float32)
    D = dev(D32)
    y, _ = life.life_dsc(idx, D, dev(w))
    g, _ = life.life_wc(idx, D, dev(r))
    torch.cuda.synchronize()
    life.life_check_device_status()
    y, g = y.cpu().numpy(), g.cpu().numpy()
    y_ref = oracle.dsc(phi, D32, w, nt, nv)
    g_ref = oracle.wc(phi, D32, r, nt, nf)
    yb, gb = rounding_bounds(phi, D32, w, r, nt, nv, nf)
    assert np.isfinite(y).all() and np.isfinite(g).all()
    assert (np.abs(y - y_ref) <= yb + 1e-38).all(), float((np.abs(y - y_ref) / (yb + 1e-38)).max())
    # WC's fixed-point tables round each entry to a unit relative to its brick's bound
    tiles = {k: v.cpu().numpy() for k, v in life.life_index_export_tiles(idx).items()}
    fxb = fixed_point_bound(phi, D32, r, tiles["tile_vox"][:128 * idx.info()["n_tiles"]], tiles["brick_tile_ptr"],
                            nt, nv, nf)
    assert (np.abs(g - g_ref) <= gb + fxb + 1e-38).all()
    assert rel(y, y_ref) <= TOL_BF16 and rel(g, g_ref) <= TOL_BF16


def test_tc_dsc_non_finite_weights(life):
    """Weights of order 1e6 (run sums far beyond FP16's range unless scaled) with
    one +inf and one NaN: the FP16 scale of S comes from the finite weights, so
    every output the non-finite weights do not reach stays within the rounding
    bound, and the outputs they reach are non-finite exactly where the FP64
    oracle's are (NaN where it has NaN)."""
    p, D32, phi, idx = tiny_case(life)
    nt, nv, nf = p.n_theta, p.n_voxels, p.n_fasc
    rng = np.random.default_rng(41)
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
    yb, _ = rounding_bounds(phi, D32, w0, np.zeros(nt * nv, np.float32), nt, nv, nf)
    assert (np.abs(y[ok] - y_ref[ok]) <= yb[ok] + 1e-30).all()
