"""Host logic of the voxel-sharded SBB-NNLS solve on CPU: the exchange driver
(``paper_1905_06234_gb300.shard``) over gloo ranks and over shards held by one
process, with each shard's phases computed by the FP64 oracle.

The oracle phases below split ``oracle_sbb_step`` (Eq. 5-8, Algorithm 1) at the
exchange points exactly as the CUDA phases do: M w, the residual and M g~ are
shard-local rows; g, u = M^T M g~, <e,e> and <M g~, M g~> are sums over shards.
Run through the driver, the sharded iterations must reproduce the unsharded
oracle solve to FP64 rounding: a wrong split (a local sum treated as global or
the other way round, a missed exchange, the exchange at the wrong point) moves
w or the step sizes far beyond that.
"""
import math
import os
import socket

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1905_06234_gb300.shard import LocalSum, ProcessGroupSum, Shard, ShardedSBB, voxel_ranges

N_ITER = 12


def make_case():
    p = synth.make_problem("shard", seed=1905062349, n_theta=12, n_atoms=20, grid=(5, 5, 4), n_fasc=30,
                           steps=(6, 14))
    D, _ = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
    phi = oracle.canon(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_atoms, p.n_voxels, p.n_fasc)
    b = oracle.problem_signal(phi, D, p.w_true, p.noise, p.n_theta, p.n_voxels).astype(np.float64)
    return p, D, phi, b


class OracleState:
    def __init__(self):
        self.it, self.alpha, self.obj, self.gg, self.gg0, self.vv, self.uu = 0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0
        self.eq, self.converged = 0, 0


class OraclePhases:
    """The three phases of one shard's iteration, in FP64 with the oracle's SpMVs."""

    def phase(self, s, k, tol, eq7_on_even):
        x, st = s.extra, s.st
        phi, D, nt, nv, nf = x["phi"], s.D, x["nt"], x["nv"], x["nf"]
        g, u, scal, w = s.g.numpy(), s.u.numpy(), s.scal.numpy(), s.w.numpy()
        if k == 1:
            if st.converged:
                g[:] = 0.0
                return
            e = oracle.dsc(phi, D, w, nt, nv) - s.b
            scal[0] = float(e @ e)
            g[:] = oracle.wc(phi, D, e, nt, nf)
        elif k == 2:
            if st.converged:
                return
            gt = np.where((w == 0.0) & (g > 0.0), 0.0, g)
            gg = float(gt @ gt)
            st.obj, st.gg = 0.5 * scal[0], gg
            if st.it == 0:
                st.gg0 = gg
            if gg == 0.0 or math.sqrt(gg) <= tol * math.sqrt(st.gg0):
                st.converged, st.eq = 1, 0
                return
            even = st.it % 2 == 0
            st.eq = 7 if (even if eq7_on_even else not even) else 8
            v = oracle.dsc(phi, D, gt, nt, nv)
            scal[1] = float(v @ v)
            u[:] = oracle.wc(phi, D, v, nt, nf) if st.eq == 8 else 0.0
            x["gt"] = gt
        else:
            if st.converged:
                return
            vv = scal[1]
            uu = float(u @ u) if st.eq == 8 else 0.0
            alpha = st.alpha
            if st.eq == 7 and vv > 0.0:
                alpha = st.gg / vv
            if st.eq == 8 and uu > 0.0:
                alpha = vv / uu
            st.vv, st.uu, st.alpha = vv, uu, alpha
            w[:] = np.maximum(w - alpha * x["gt"], 0.0)
            st.it += 1


def oracle_shard(p, D, phi, b, v0, v1):
    sel = (phi.voxel >= v0) & (phi.voxel < v1)
    sphi = oracle.Phi(phi.atom[sel], phi.voxel[sel] - v0, phi.fasc[sel], phi.val[sel])
    nt, nf = p.n_theta, p.n_fasc
    return Shard(index=None, D=D, b=b[v0 * nt:v1 * nt], w=torch.ones(nf, dtype=torch.float64), st=OracleState(),
                 g=torch.zeros(nf, dtype=torch.float64), u=torch.zeros(nf, dtype=torch.float64),
                 scal=torch.zeros(2, dtype=torch.float64), extra=dict(phi=sphi, nt=nt, nv=v1 - v0, nf=nf))


def reference(p, D, phi, b, n_iter, tol=0.0):
    w = np.ones(p.n_fasc)
    st = oracle.sbb_solve(phi, D, b, w, p.n_theta, p.n_voxels, p.n_fasc, n_iter, tol=tol)
    return w, st


def check_against_reference(w, st, w_ref, st_ref):
    assert st.it == st_ref.it and st.eq == st_ref.eq and st.converged == st_ref.converged
    for k in ("obj", "gg", "gg0", "vv", "uu", "alpha"):
        a, r = getattr(st, k), getattr(st_ref, k)
        assert abs(a - r) <= 1e-9 * max(abs(r), 1e-300), (k, a, r)
    assert np.abs(w - w_ref).max() <= 1e-9 * max(np.abs(w_ref).max(), 1e-300)


@pytest.mark.parametrize("n_shards", [1, 3])
def test_local_shards_match_unsharded_oracle(n_shards):
    p, D, phi, b = make_case()
    shards = [oracle_shard(p, D, phi, b, v0, v1) for v0, v1 in voxel_ranges(p.n_voxels, n_shards)]
    ShardedSBB(shards, OraclePhases(), LocalSum()).solve(N_ITER)
    w_ref, st_ref = reference(p, D, phi, b, N_ITER)
    for s in shards:
        check_against_reference(s.w.numpy(), s.st, w_ref, st_ref)


def test_local_shards_stop_together():
    p, D, phi, b = make_case()
    shards = [oracle_shard(p, D, phi, b, v0, v1) for v0, v1 in voxel_ranges(p.n_voxels, 2)]
    ShardedSBB(shards, OraclePhases(), LocalSum(), tol=1e-3).solve(200)
    w_ref, st_ref = reference(p, D, phi, b, 200, tol=1e-3)
    assert st_ref.converged == 1 and st_ref.it < 200
    for s in shards:
        check_against_reference(s.w.numpy(), s.st, w_ref, st_ref)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        p, D, phi, b = make_case()
        v0, v1 = voxel_ranges(p.n_voxels, world)[rank]
        s = oracle_shard(p, D, phi, b, v0, v1)
        ShardedSBB([s], OraclePhases(), ProcessGroupSum()).solve(N_ITER)
        st = s.st
        np.save(os.path.join(out_dir, f"w{rank}.npy"), s.w.numpy())
        np.save(os.path.join(out_dir, f"st{rank}.npy"),
                np.array([st.it, st.eq, st.converged, st.obj, st.gg, st.gg0, st.vv, st.uu, st.alpha], np.float64))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_match_unsharded_oracle(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    p, D, phi, b = make_case()
    w_ref, st_ref = reference(p, D, phi, b, N_ITER)
    ws = [np.load(tmp_path / f"w{r}.npy") for r in range(world)]
    assert np.array_equal(ws[0], ws[1])   # the replicated state is identical on every rank
    for r in range(world):
        v = np.load(tmp_path / f"st{r}.npy")
        st = OracleState()
        st.it, st.eq, st.converged = int(v[0]), int(v[1]), int(v[2])
        st.obj, st.gg, st.gg0, st.vv, st.uu, st.alpha = v[3:]
        check_against_reference(ws[r], st, w_ref, st_ref)
