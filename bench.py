"""LiFE SBB-NNLS throughput on one or more GB300s (one process per GPU, replicas).

A step is one SBB-NNLS iteration (Eq. 5-8, Algorithm 1: DSC with the residual,
WC, the projected gradient, DSC of the projected gradient, WC on Eq. 8
iterations, the BB step and the projection) on the paper-scale synthetic
problem: Nθ = 96, Na = 360, a 96x96x72 grid with an ellipsoidal mask, Nf = 500k
persistent-walk fascicles of 20-300 steps.  ``value`` is whole-job SBB iterations
per second (every rank runs its own replica; max-over-ranks time).

Default run (no flags): 1 GPU, the fastest path beside the plain FP32 path,
20 timed steps after 5 warm-up steps.  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DSC+WC effective HBM GB/s (% of peak) and SBB-NNLS iters/s at Nf=500k, vs plain FP32"
UNIT = "iter/s"
PEAK_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


# DRAM bytes (read + write) of the launches of one timed tensor-core call, from
# ncu captures (dram__bytes_read.sum + dram__bytes_write.sum, one kernel per
# capture) on the paper-density workload at a third of the size: DSC with the
# fused residual = max|w| pass + DSC kernel; WC through the public call =
# per-tile max|r| pass + WC kernel; per path (BF16 storage, FP32 storage on the
# tensor cores).  Scaled to the timed workload by its entry count (the traffic
# grows with the entries and voxels alike).  The figures hold only for the kernel
# source that was captured; after any change to it the bench reports null.
TRAFFIC_CAPTURE = {
    "src": os.path.join("paper_1905_06234_gb300", "csrc", "spmv_tc.cu"),
    "sha256": "c2ce55ecc66241ca51bf6295504ca4d5f7318b4270cc02fecf8076e9626f776a",
    "nnz": 23816750,
    "bytes": {
        "bf16-tc": {"dsc": (607488 + 0) + (197645312 + 16574976), "wc": (39993600 + 0) + (201986816 + 118016)},
        "fp32-tc": {"dsc": (607488 + 0) + (248668160 + 20288256), "wc": (39993856 + 0) + (252520448 + 125696)},
    },
}


def kernel_traffic(path_name, kind, nnz):
    """Measured DRAM bytes of one launch (scaled to `nnz` entries if the workload differs), or None."""
    import hashlib
    per_path = TRAFFIC_CAPTURE["bytes"].get(path_name)
    if per_path is None:
        return None
    try:
        with open(os.path.join(ROOT, TRAFFIC_CAPTURE["src"]), "rb") as fh:
            sha = hashlib.sha256(fh.read()).hexdigest()
    except OSError:
        return None
    if sha != TRAFFIC_CAPTURE["sha256"]:
        return None
    return per_path[kind] * nnz / TRAFFIC_CAPTURE["nnz"]


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return PEAK_FALLBACK, "fallback"


# --------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ workload

def make_workload(name: str):
    import synth
    t0 = time.time()
    p = synth.config_problem(name)
    return p, time.time() - t0


def workload_desc(p):
    """The workload as both arms name it (the merged entry count is a separate key)."""
    mask = "ellipsoidal mask" if p.meta.get("mask") else "no mask"
    gx, gy, gz = p.grid
    return (f"paper-scale LiFE: Ntheta={p.n_theta}, Na={p.n_atoms}, {gx}x{gy}x{gz} grid with {mask} "
            f"(Nv={p.n_voxels}), Nf={p.n_fasc} persistent walks of {p.meta['steps'][0]}-{p.meta['steps'][1]} "
            f"steps, {p.n_raw} raw Phi entries")


# ------------------------------------------------------------ GPU arm

class GpuPath:
    """Index + device buffers for one precision/algorithm choice."""

    def __init__(self, life, p, D, b, precision, algo, autotune=False, sparse_dsc=False):
        import torch
        self.life = life
        t0 = time.time()
        self.idx = life.upload_problem(p, precision=precision, algo=algo, sparse_dsc=sparse_dsc)
        if autotune:
            life.life_index_autotune(self.idx)
        torch.cuda.synchronize()
        self.build_s = time.time() - t0
        self.info = self.idx.info()
        self.p, self.D, self.b = p, D, b
        self.w = torch.ones(p.n_fasc, dtype=torch.float32, device="cuda")
        self.st = life.new_sbb_state()
        self.ws = life.new_sbb_workspace(self.idx)

    def reset(self):
        self.w.fill_(1.0)
        self.life.life_sbb_state_init(self.st)

    def run_steps(self, k):
        self.life.life_sbbnnls_solve(self.idx, self.D, self.b, self.w, k, self.st, self.ws)

    def run_steps_each(self, k):
        """The same iterations as k single-step calls, so that every kernel is its
        own launch (a profiler does not see inside the solve's conditional graph)."""
        for _ in range(k):
            self.life.life_sbbnnls_step(self.idx, self.D, self.b, self.w, self.st, self.ws)


def time_steps(path, steps, warmup):
    import torch
    path.reset()
    path.run_steps(warmup)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    path.run_steps(steps)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def time_kernel(fn, reps=10):
    """Average device time of fn() over reps launches, CUDA events on the current stream."""
    import torch
    fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def spmv_bytes(path, kind, fused_b=False):
    """Algorithmic bytes of one SpMV call: the canonical compact Phi stream
    (u16 atom + i32 fascicle + value: 10 B/nonzero FP32, 8 B BF16) plus the CSR
    pointers, the dense vectors read and written, and D once."""
    p, info = path.p, path.info
    nnz = info["nnz"]
    per_nz = 8 if info["precision"] == 1 else 10
    sig = 4 * p.n_theta * p.n_voxels
    phi = per_nz * nnz + 4 * (p.n_voxels + 1)
    dbytes = 4 * p.n_theta * p.n_atoms
    if kind == "dsc":
        return phi + 4 * p.n_fasc + sig + (sig if fused_b else 0) + dbytes
    return phi + sig + 4 * p.n_fasc + dbytes


def kernel_calls(life, path):
    """The two SpMV calls whose launches the roofline times: DSC with the fused
    residual, and WC through the public call (on the tensor-core path that is
    the per-tile max|r| pass and the WC kernel)."""
    import torch
    p = path.p
    r = path.b
    g = torch.empty(p.n_fasc, dtype=torch.float32, device="cuda")
    e = torch.empty(p.n_theta * p.n_voxels, dtype=torch.float32, device="cuda")
    w = torch.rand(p.n_fasc, device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    return (lambda: life.life_dsc(path.idx, path.D, w, b=path.b, y=e)), (lambda: life.life_wc(path.idx, path.D, r, g=g))


def measure_kernels(life, path):
    dsc_call, wc_call = kernel_calls(life, path)
    t_dsc = time_kernel(dsc_call)
    t_wc = time_kernel(wc_call)
    b_dsc = spmv_bytes(path, "dsc", fused_b=True)
    b_wc = spmv_bytes(path, "wc")
    return dict(dsc_s=t_dsc, wc_s=t_wc, dsc_bytes=b_dsc, wc_bytes=b_wc)


def e2e_steps(life, path, steps, warmup):
    """Per step through the public API with host buffers: w (pinned host) -> device,
    one SBB iteration, w and the state -> host."""
    import torch
    p = path.p
    w_host = torch.ones(p.n_fasc, dtype=torch.float32).pin_memory()
    st_host = torch.empty(path.st.numel(), dtype=torch.uint8).pin_memory()
    s = torch.cuda.current_stream()
    path.reset()

    def one():
        path.w.copy_(w_host, non_blocking=True)
        life.life_sbbnnls_step(path.idx, path.D, path.b, path.w, path.st, path.ws)
        w_host.copy_(path.w, non_blocking=True)
        st_host.copy_(path.st, non_blocking=True)
        s.synchronize()

    for _ in range(warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    dt = time.perf_counter() - t0
    return steps / dt, 4 * p.n_fasc, 4 * p.n_fasc + path.st.numel()


def launches_per_step(path):
    # DSC + WC + project + scalars + DSC + WC + sumsq + scalars + update + the
    # solve loop's condition kernel, and on the tensor-core path the brick weight
    # gather before each of the two DSCs (the WCs take the per-tile max |r| from
    # the DSC before them, so the step launches no separate max pass)
    return 12 if path.info["algo"] == 2 else 10


def launches_per_solve(path, steps):
    """Kernels of one timed solve: the steps plus the loop-counter initialisation."""
    return launches_per_step(path) * steps + 1


def max_over_ranks(value, dist, device):
    """The largest value over all ranks (the slowest replica's time); the value
    itself without a process group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def job_throughput(steps, world, dt_max):
    """Whole-job iterations per second: every replica runs `steps` iterations
    and the job lasts as long as the slowest replica."""
    return world * steps / dt_max


def host_cpu():
    """The host CPU as lscpu names it (architecture, model, CPUs)."""
    import platform
    desc = {"arch": platform.machine(), "cpus": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Model name", "Vendor ID", "Core(s) per socket", "Core(s) per cluster", "Socket(s)"):
                desc[k.strip()] = v.strip()
    except Exception:
        pass
    return desc


def cpu_allcores_baseline(p, D32, b, reps=2):
    """The FP64 baseline as it stands on all host cores (the oracle's arithmetic
    with Phi grouped by voxel for DSC and by fascicle for WC, OpenMP), on the whole
    workload: one untimed and `reps` timed SBB iterations from w = 1."""
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    op = oracle.OmpProblem(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_voxels, p.n_fasc)
    group_s = time.perf_counter() - t0
    b64 = np.asarray(b, np.float64)
    w = np.ones(p.n_fasc)
    st = oracle.SbbState()
    work = np.empty(2 * p.n_theta * p.n_voxels + 2 * p.n_fasc, np.float64)
    op.sbb_step(D32, b64, w, st, work=work)
    t0 = time.perf_counter()
    for _ in range(reps):
        op.sbb_step(D32, b64, w, st, work=work)
    dt = time.perf_counter() - t0
    return dict(iter_s=dt / reps, reps=reps, cores=oracle.omp_threads(), group_s=group_s)


def full_solve(life, path, n_iter=500):
    """The workload's full solve: n_iter SBB-NNLS iterations from w = 1 as one
    graph launch (the graph is built by an untimed call first)."""
    import torch
    path.reset()
    path.run_steps(1)
    torch.cuda.synchronize()
    path.reset()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    path.run_steps(n_iter)
    e1.record(s)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    st = life.read_sbb_state(path.st)
    out = {"iters": int(st["it"]), "s": t, "iter_per_s": st["it"] / t, "obj": st["obj"],
           "rel_pg": (st["gg"] / st["gg0"]) ** 0.5 if st["gg0"] > 0 else None,
           "zero_weights": float((path.w == 0).float().mean())}
    if path.info.get("sparse_dsc"):
        out["live_entry_stream"] = life.life_index_sparse_stats(path.idx)
    return out


def sparse_dsc_sweep(life, live, full, fracs=(0.0, 0.5, 0.9, 0.97), reps=10):
    """DSC with the fused residual for weights with a given fraction of zeros: the
    index with the live-entry stream (first call untimed: it builds the stream for
    this support) against the same layout streaming every entry."""
    import torch
    p = live.p
    y = torch.empty(p.n_theta * p.n_voxels, dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(1)
    out = []
    for zf in fracs:
        w = torch.rand(p.n_fasc, device="cuda", generator=gen)
        w[torch.rand(p.n_fasc, device="cuda", generator=gen) < zf] = 0.0
        row = {"zero_frac": zf}
        for name, path in (("live", live), ("full", full)):
            row[name + "_ms"] = time_kernel(lambda: life.life_dsc(path.idx, path.D, w, b=path.b, y=y), reps) * 1e3
        st = life.life_index_sparse_stats(live.idx)
        row["live_entries"], row["entries"] = st["live_entries"], st["entries"]
        out.append(row)
    return out


def time_to_tolerance(life, lo, hi, tol, switches=(1e-3, 3e-4, 1e-4), max_iter=500, hi_tc=None):
    """Time to ‖g~‖ <= tol·‖g~_0‖ from w = 1: the plain path `hi` alone, the fast
    path `lo` alone, and `lo` until each switch tolerance followed by `hi` to tol
    from the same w and state (the state keeps ‖g~_0‖, so both phases test against
    the same reference); with `hi_tc` (FP32 storage on the tensor cores) also that
    path alone and as the second phase.  Graphs are built by untimed calls first."""
    import torch
    s = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def state(st):
        x = life.read_sbb_state(st)
        return {"iters": int(x["it"]), "converged": int(x["converged"]), "obj": x["obj"],
                "rel_pg": (x["gg"] / x["gg0"]) ** 0.5 if x["gg0"] > 0 else None}

    out = {"tol": tol, "max_iter": max_iter}
    alone = [("plain", hi), ("fast", lo)] + ([("fp32_tc", hi_tc)] if hi_tc is not None else [])
    for name, path in alone:
        path.reset()
        life.life_sbbnnls_solve(path.idx, path.D, path.b, path.w, 1, path.st, path.ws, tol=tol)
        torch.cuda.synchronize()
        path.reset()
        t = timed(lambda: life.life_sbbnnls_solve(path.idx, path.D, path.b, path.w, max_iter, path.st, path.ws,
                                                  tol=tol))
        out[name] = dict(state(path.st), s=t)

    seconds = [("fast_then_plain", hi)] + ([("fast_then_fp32_tc", hi_tc)] if hi_tc is not None else [])
    for key, second in seconds:
        out[key] = {}
        for tol_lo in switches:
            def mixed():
                life.life_sbbnnls_solve(lo.idx, lo.D, lo.b, lo.w, max_iter, lo.st, lo.ws, tol=tol_lo)
                ph1 = life.read_sbb_state(lo.st)["it"] if timing_phase1 else None
                life.life_sbb_state_resume(lo.st)
                life.life_sbbnnls_solve(second.idx, second.D, second.b, lo.w, max_iter, lo.st, second.ws, tol=tol)
                return ph1

            timing_phase1 = True
            lo.reset()
            it_fast = mixed()
            torch.cuda.synchronize()
            timing_phase1 = False
            lo.reset()
            t = timed(mixed)
            out[key][f"{tol_lo:g}"] = dict(state(lo.st), s=t, iters_fast=int(it_fast))
    done = {k: v for k, v in out["fast_then_plain"].items() if v["converged"]}
    if out["plain"]["converged"] and done:
        best = min(done, key=lambda k: done[k]["s"])
        out["best_switch"] = best
        out["speedup_at_tol"] = out["plain"]["s"] / done[best]["s"]
    # the fastest route to the tolerance among all forms, against the plain FP32 solve
    routes = {}
    if out.get("fp32_tc", {}).get("converged"):
        routes["fp32_tc"] = out["fp32_tc"]["s"]
    for key, _ in seconds:
        for sw, v in out[key].items():
            if v["converged"]:
                routes[f"{key}@{sw}"] = v["s"]
    if out["plain"]["converged"] and routes:
        best = min(routes, key=routes.get)
        out["best_route"] = best
        out["best_route_speedup"] = out["plain"]["s"] / routes[best]
    return out


def run_batched(life, D, max_iter=500, tol=1e-4, tol_switch=1e-3):
    """The batched workload: 16 independent problems of uneven size (Nf log-uniform
    in 1e4..2e5, cubic grids of edge 32..80, no mask) solved by SBB-NNLS to
    ‖g~‖/‖g~_0‖ <= tol, as one batched solve (one graph launch) and as 16
    sequential plain solves, for the FP32 CUDA-core, FP32 tensor-core and BF16
    tensor-core paths, and as BF16 batched iterations to tol_switch followed by
    FP32 batched iterations (CUDA cores or tensor cores) to tol from the same
    weights and states.  The tensor-core batches' tile layouts come from the
    autotuner."""
    import torch
    import synth
    t0 = time.time()
    probs = synth.batched_problems(16)
    gen_s = time.time() - t0
    dev = torch.device("cuda")
    out = {"problems": len(probs), "nnz_raw": int(sum(p.n_raw for p in probs)),
           "n_fasc": [int(p.n_fasc) for p in probs], "grid_edge": [int(p.grid[0]) for p in probs],
           "max_iter": max_iter, "tol": tol, "gen_s": gen_s}
    bs = None
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    batches, all_idxs = {}, []
    for name, prec, algo in (("fp32-simt", life.LIFE_FP32, life.LIFE_ALGO_SIMT),
                             ("fp32-tc", life.LIFE_FP32, life.LIFE_ALGO_TC),
                             ("bf16-tc", life.LIFE_BF16, life.LIFE_ALGO_TC)):
        idxs = [life.upload_problem(p, precision=prec, algo=algo) for p in probs]
        all_idxs += idxs
        if bs is None:  # b_p = M_p w_true + noise from the FP32 DSC
            bs = []
            for p, ix in zip(probs, idxs):
                b, _ = life.life_dsc(ix, D, torch.from_numpy(p.w_true).to(dev))
                bs.append(b + torch.from_numpy(p.noise).to(dev))
        t0 = time.time()
        batch = life.life_batch_create(idxs, autotune=(algo == life.LIFE_ALGO_TC))
        torch.cuda.synchronize()
        create_s = time.time() - t0
        batches[name] = batch
        ws = [torch.ones(p.n_fasc, device=dev) for p in probs]
        st = life.new_batch_states(len(probs))
        wsp = life.new_batch_workspace(batch)
        life.life_batch_solve(batch, D, bs, ws, max_iter, st, wsp, tol=tol)   # builds the graph
        torch.cuda.synchronize()
        for w in ws:
            w.fill_(1.0)
        st.copy_(life.new_batch_states(len(probs)))
        e0.record(s)
        life.life_batch_solve(batch, D, bs, ws, max_iter, st, wsp, tol=tol)
        e1.record(s)
        torch.cuda.synchronize()
        t_batch = e0.elapsed_time(e1) / 1e3
        bst = life.read_batch_states(st, len(probs))
        # sequential plain solves, each graph built once before timing
        seq = []
        for p, ix, b in zip(probs, idxs, bs):
            w = torch.ones(p.n_fasc, device=dev)
            st1, ws1 = life.new_sbb_state(), life.new_sbb_workspace(ix)
            life.life_sbbnnls_solve(ix, D, b, w, 1, st1, ws1, tol=tol)
            seq.append((ix, b, w, st1, ws1))
        torch.cuda.synchronize()
        for ix, b, w, st1, ws1 in seq:
            w.fill_(1.0)
            life.life_sbb_state_init(st1)
        e0.record(s)
        for ix, b, w, st1, ws1 in seq:
            life.life_sbbnnls_solve(ix, D, b, w, max_iter, st1, ws1, tol=tol)
        e1.record(s)
        torch.cuda.synchronize()
        t_seq = e0.elapsed_time(e1) / 1e3
        sst = [life.read_sbb_state(x[3]) for x in seq]
        its_b = [int(x["it"]) for x in bst]
        its_s = [int(x["it"]) for x in sst]
        obj_dev = max(abs(a["obj"] - b_["obj"]) / abs(b_["obj"]) for a, b_ in zip(bst, sst))
        out[name] = {"batched_ms": t_batch * 1e3, "sequential_ms": t_seq * 1e3, "speedup": t_seq / t_batch,
                     "batched_iter_per_s": sum(its_b) / t_batch, "sequential_iter_per_s": sum(its_s) / t_seq,
                     "iters": its_b, "iters_sequential": its_s,
                     "converged": int(sum(x["converged"] for x in bst)),
                     "final_obj": [x["obj"] for x in bst],
                     "max_rel_obj_diff_vs_sequential": obj_dev, "create_s": create_s, "batch": batch.info()}
        del seq
    # BF16 batched iterations to tol_switch, then FP32 batched iterations to tol (on
    # the CUDA cores or the tensor cores), from the same weights and states (both
    # graphs built by an untimed run)
    for hi_name in ("fp32-simt", "fp32-tc"):
        ws = [torch.ones(p.n_fasc, device=dev) for p in probs]
        st = life.new_batch_states(len(probs))
        wlo, whi = life.new_batch_workspace(batches["bf16-tc"]), life.new_batch_workspace(batches[hi_name])

        def mixed():
            life.life_batch_solve(batches["bf16-tc"], D, bs, ws, max_iter, st, wlo, tol=tol_switch)
            life.life_sbb_state_resume(st, len(probs))
            life.life_batch_solve(batches[hi_name], D, bs, ws, max_iter, st, whi, tol=tol)

        mixed()
        torch.cuda.synchronize()
        for w in ws:
            w.fill_(1.0)
        st.copy_(life.new_batch_states(len(probs)))
        e0.record(s)
        mixed()
        e1.record(s)
        torch.cuda.synchronize()
        t_mix = e0.elapsed_time(e1) / 1e3
        mst = life.read_batch_states(st, len(probs))
        out["bf16-tc+" + hi_name] = {"batched_ms": t_mix * 1e3, "tol_switch": tol_switch,
                                     "iters": [int(x["it"]) for x in mst],
                                     "converged": int(sum(x["converged"] for x in mst)),
                                     "final_obj": [x["obj"] for x in mst],
                                     "speedup_vs_fp32_sequential": out["fp32-simt"]["sequential_ms"] / (t_mix * 1e3),
                                     "speedup_vs_fp32_batched": out["fp32-simt"]["batched_ms"] / (t_mix * 1e3)}
    for b_ in batches.values():
        b_.close()
    for ix in all_idxs:
        ix.close()
    return out


def run_ours(args):
    import numpy as np
    import torch
    import paper_1905_06234_gb300 as life

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    life.load()
    peaks, peak_src = read_peaks()
    p, gen_s = make_workload(args.workload)
    dev = torch.device("cuda", local)
    g = torch.from_numpy(p.grad_dirs)
    u = torch.from_numpy(p.atom_dirs)
    D, _ = life.life_dictionary(g, u, p.bval, p.lam)
    # the measured signal b = M w_true + noise, computed on the device
    fp32 = GpuPath(life, p, D, torch.zeros(p.n_theta * p.n_voxels, device=dev), life.LIFE_FP32, life.LIFE_ALGO_SIMT)
    w_true = torch.from_numpy(p.w_true).to(dev)
    b, _ = life.life_dsc(fp32.idx, D, w_true)
    b += torch.from_numpy(p.noise).to(dev)
    fp32.b = b
    paths = {"fp32-simt": fp32}
    if args.precision in ("fp32", "both"):
        # FP32 storage on the tensor cores (split FP16 hi/lo operands)
        try:
            paths["fp32-tc"] = GpuPath(life, p, D, b, life.LIFE_FP32, life.LIFE_ALGO_TC, autotune=args.autotune)
        except life.LifeError as e:
            paths["fp32-tc"] = None
            if rank == 0:
                print(f"# fp32 tensor-core path unavailable: {e}", file=sys.stderr)
    if args.precision in ("bf16", "both"):
        try:
            paths["bf16-tc"] = GpuPath(life, p, D, b, life.LIFE_BF16, life.LIFE_ALGO_TC, autotune=args.autotune)
        except life.LifeError as e:
            paths["bf16-tc"] = None
            if rank == 0:
                print(f"# bf16 tensor-core path unavailable: {e}", file=sys.stderr)
    live_path = None
    if args.full_solve == "on" and paths.get("bf16-tc") is not None:
        # the same tensor-core index with the live-entry DSC stream (sparse-w-aware DSC)
        live_path = GpuPath(life, p, D, b, life.LIFE_BF16, life.LIFE_ALGO_TC, autotune=args.autotune,
                            sparse_dsc=True)
    if args.profile:
        # Profiling mode: between cudaProfilerStart/Stop (for ncu
        # --profile-from-start off) run only the SBB steps of each path (one call
        # per step), then one of each of the DSC and WC calls that the roofline times.
        for name, path in paths.items():
            if path is None:
                continue
            path.reset()
            path.run_steps(args.warmup)
            dsc_call, wc_call = kernel_calls(life, path)
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            path.run_steps_each(args.steps)
            dsc_call()
            wc_call()
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        if dist:
            dist.destroy_process_group()
        return
    results = {}
    for name, path in paths.items():
        if path is None:
            continue
        kern = measure_kernels(life, path)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        dt = time_steps(path, args.steps, args.warmup)
        ck = clocks.stop()
        dt = max_over_ranks(dt, dist, dev)
        results[name] = dict(path=path, dt=dt, kern=kern, clocks=ck)
    best_name = min(results, key=lambda k: results[k]["dt"])
    best = results[best_name]
    path = best["path"]
    e2e_n = max(3, args.steps // 2)
    e2e_val, h2d, d2h = e2e_steps(life, path, e2e_n, 2)
    e2e_val = job_throughput(e2e_n, world, max_over_ranks(e2e_n / e2e_val, dist, dev))
    st = life.read_sbb_state(path.st)
    solves, tol_run = None, None
    if args.full_solve == "on":
        solves = {k: full_solve(life, v) for k, v in paths.items() if v is not None}
        if live_path is not None:
            solves["bf16-tc-live"] = full_solve(life, live_path)
            solves["bf16-tc-live"]["dsc_vs_zero_weights"] = sparse_dsc_sweep(life, live_path, paths["bf16-tc"])
        if paths.get("bf16-tc") is not None:
            tol_run = time_to_tolerance(life, paths["bf16-tc"], paths["fp32-simt"], tol=1e-4,
                                        hi_tc=paths.get("fp32-tc"))
    batched = run_batched(life, D) if args.batched == "on" else None
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    kern = best["kern"]
    # dominant kernel of an iteration: 2 DSC + 1.5 WC per iteration on average (Sec. 2.2)
    share_dsc, share_wc = 2 * kern["dsc_s"], 1.5 * kern["wc_s"]
    dom = "dsc" if share_dsc >= share_wc else "wc"
    t_dom = kern[f"{dom}_s"]
    achieved = kern[f"{dom}_bytes"] / t_dom / 1e9
    peak = float(peaks.get("hbm_gbs", PEAK_FALLBACK["hbm_gbs"]))
    dsc_wc_gbs = (kern["dsc_bytes"] + kern["wc_bytes"]) / (kern["dsc_s"] + kern["wc_s"]) / 1e9
    cpu = cpu_allcores_baseline(p, D.cpu().numpy(), b.cpu().numpy())
    cpu_value = 1.0 / cpu["iter_s"]
    value = job_throughput(args.steps, world, best["dt"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": best["dt"] / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if best_name.startswith("bf16") else "f32", "data": "synthetic",
        "config": {"workload": workload_desc(p), "nnz_merged": path.info["nnz"], "path": best_name,
                   "l2": "inputs larger than L2 (Phi stream %.2f GB per SpMV)" % (path.info["stream_bytes"] / 1e9),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": f"{peak_src} hbm_gbs",
                     "traffic": kernel_traffic(best_name, dom, path.info["nnz"]),
                     "traffic_note": "ncu DRAM bytes of one timed call of this kernel (its launches), captured on the "
                                     "one-third-size paper-density case and scaled by the entry count"},
        "dsc_wc": {"gbs": dsc_wc_gbs, "frac_of_peak": dsc_wc_gbs / peak, "dsc_ms": kern["dsc_s"] * 1e3,
                   "wc_ms": kern["wc_s"] * 1e3},
        "paths": {k: {"iter_per_s": args.steps / v["dt"], "dsc_ms": v["kern"]["dsc_s"] * 1e3,
                      "wc_ms": v["kern"]["wc_s"] * 1e3,
                      "dsc_gbs": v["kern"]["dsc_bytes"] / v["kern"]["dsc_s"] / 1e9,
                      "wc_gbs": v["kern"]["wc_bytes"] / v["kern"]["wc_s"] / 1e9,
                      "dsc_frac": v["kern"]["dsc_bytes"] / v["kern"]["dsc_s"] / 1e9 / peak,
                      "wc_frac": v["kern"]["wc_bytes"] / v["kern"]["wc_s"] / 1e9 / peak,
                      "vs_fp32_simt": results["fp32-simt"]["dt"] / v["dt"],
                      "dsc_traffic": kernel_traffic(k, "dsc", v["path"].info["nnz"]),
                      "wc_traffic": kernel_traffic(k, "wc", v["path"].info["nnz"]),
                      "index_build_s": v["path"].build_s} for k, v in results.items()},
        "vs_plain_fp32": (args.steps / best["dt"]) / (args.steps / results["fp32-simt"]["dt"]),
        "cpu_baseline": {"value": cpu_value, "unit": UNIT, "cores": cpu["cores"], "kind": "oracle",
                         "host": host_cpu(),
                         "sample": "%d FP64 SBB iterations of the whole workload (all %d raw entries) after one "
                                   "untimed, on %d host threads (OpenMP: voxel-grouped DSC, fascicle-grouped WC); "
                                   "grouping the entries took %.1f s" % (cpu["reps"], p.n_raw, cpu["cores"],
                                                                         cpu["group_s"])},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_solve(path, args.steps) * world,
        "clocks": best["clocks"],
        "final_state": {"it": st["it"], "obj": st["obj"], "alpha": st["alpha"]},
        "tile_layout": {k: path.info[k] for k in ("brick_edge", "wc_groups", "tuned")},
        "full_solve": solves,
        "time_to_tolerance": tol_run,
        "batched": batched,
        "gen_s": gen_s,
    }
    print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args):
    """The FP64 baseline as it stands on the host cores (the oracle's arithmetic,
    OpenMP over voxel and fascicle groups): every step is one SBB iteration of the
    whole workload, so ms_per_step x steps is the time that ran."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle
    p, _ = make_workload(args.workload)
    D64, _ = oracle.dictionary(p.grad_dirs, p.atom_dirs, p.bval, p.lam)
    D32 = D64.astype(np.float32)
    t0 = time.perf_counter()
    op = oracle.OmpProblem(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_voxels, p.n_fasc)
    group_s = time.perf_counter() - t0
    b = (op.dsc(D32, p.w_true) + p.noise).astype(np.float32).astype(np.float64)
    w = np.ones(p.n_fasc)
    st = oracle.SbbState()
    work = np.empty(2 * p.n_theta * p.n_voxels + 2 * p.n_fasc, np.float64)
    for _ in range(args.warmup):
        op.sbb_step(D32, b, w, st, work=work)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        op.sbb_step(D32, b, w, st, work=work)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    cores = oracle.omp_threads()
    sample = ("whole workload (all %d raw entries), every step one FP64 SBB iteration on %d host threads "
              "(OpenMP: voxel-grouped DSC, fascicle-grouped WC); grouping the entries took %.1f s"
              % (p.n_raw, cores, group_s))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(p), "path": "oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "final_state": {"it": st.it, "obj": st.obj}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="paper", choices=["paper", "paper_small", "medium", "tiny"])
    ap.add_argument("--precision", default="both", choices=["fp32", "bf16", "both"])
    ap.add_argument("--autotune", action="store_true",
                    help="let the autotuner choose the BF16 tile layout of the main workload")
    ap.add_argument("--batched", default="on", choices=["on", "off"],
                    help="also time the batched workload (16 problems, batched vs sequential solves)")
    ap.add_argument("--full-solve", dest="full_solve", default="on", choices=["on", "off"],
                    help="also time the workload's full 500-iteration solve per path and the time to a "
                         "1e-4 projected-gradient tolerance")
    ap.add_argument("--profile", action="store_true",
                    help="run only warm-up + timed SBB steps inside cudaProfilerStart/Stop, print nothing")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
