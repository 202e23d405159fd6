"""ctypes binding of liblife.so (include/life.h).

Argument marshalling only: every computation runs in the CUDA library.  There is
no CPU fallback; if the library is missing or cannot load, every call raises.
Tensors are torch CUDA tensors; each call runs on torch's current stream.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

LIFE_OK, LIFE_EINVAL, LIFE_ERANGE, LIFE_ENOMEM, LIFE_ECUDA, LIFE_ETIMEOUT, LIFE_ENOTSUP = range(7)
LIFE_FP32, LIFE_BF16 = 0, 1
LIFE_ALGO_AUTO, LIFE_ALGO_SIMT, LIFE_ALGO_TC = 0, 1, 2
LIFE_LAYOUT_VOXEL, LIFE_LAYOUT_FIBER, LIFE_LAYOUT_ATOM = 0, 1, 2

_STATUS_NAMES = {0: "LIFE_OK", 1: "LIFE_EINVAL", 2: "LIFE_ERANGE", 3: "LIFE_ENOMEM", 4: "LIFE_ECUDA",
                 5: "LIFE_ETIMEOUT", 6: "LIFE_ENOTSUP"}

# Every symbol include/life.h declares (checked by the CPU test suite).
EXPORTS = [
    "life_build_index", "life_index_free", "life_index_get_info", "life_index_export",
    "life_index_export_voxel_streams", "life_index_export_tiles", "life_dsc", "life_wc",
    "life_dsc_grad_D", "life_dsc_grad_D_noalloc", "life_dictionary", "life_dot_f32", "life_sbb_workspace_bytes", "life_sbb_state_init",
    "life_sbbnnls_step", "life_sbbnnls_solve", "life_batch_create", "life_batch_free", "life_batch_get_info",
    "life_batch_offsets", "life_batch_index", "life_batch_workspace_bytes", "life_batch_solve",
    "life_index_autotune", "life_selftest_bounded_wait", "life_check_device_status", "life_last_error",
    "life_version", "life_prune", "life_voxel_rmse", "life_index_sparse_stats", "life_build_index_shard",
    "life_sbb_shard_phase", "life_sbb_state_resume",
]


class LifeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class life_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("algo", ctypes.c_int32), ("brick_dim", ctypes.c_int32),
                ("wc_groups", ctypes.c_int32), ("autotune", ctypes.c_int32), ("sparse_dsc", ctypes.c_int32),
                ("simt_kernels", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class life_index_info(ctypes.Structure):
    _fields_ = [("nnz_raw", ctypes.c_int64), ("nnz", ctypes.c_int64), ("n_theta", ctypes.c_int32),
                ("n_atoms", ctypes.c_int32), ("n_voxels", ctypes.c_int32), ("n_fasc", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("algo", ctypes.c_int32), ("n_tiles", ctypes.c_int64),
                ("n_bricks", ctypes.c_int64), ("device_bytes", ctypes.c_int64), ("stream_bytes", ctypes.c_int64),
                ("n_brick_fasc", ctypes.c_int64), ("n_sub", ctypes.c_int32), ("brick_edge", ctypes.c_int32),
                ("wc_groups", ctypes.c_int32), ("tuned", ctypes.c_int32), ("simt_runs", ctypes.c_int32),
                ("sparse_dsc", ctypes.c_int32)]


class life_batch_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("algo", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("n_voxels", ctypes.c_int32), ("n_fasc", ctypes.c_int32), ("brick_edge", ctypes.c_int32),
                ("wc_groups", ctypes.c_int32), ("tc_grid", ctypes.c_int32), ("simt_grid", ctypes.c_int32),
                ("tuned", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class life_sbb_state(ctypes.Structure):
    _fields_ = [("it", ctypes.c_int64), ("alpha", ctypes.c_double), ("obj", ctypes.c_double),
                ("gg", ctypes.c_double), ("gg0", ctypes.c_double), ("vv", ctypes.c_double),
                ("uu", ctypes.c_double), ("eq", ctypes.c_int32), ("converged", ctypes.c_int32)]


SBB_STATE_BYTES = ctypes.sizeof(life_sbb_state)

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads liblife.so (optionally compiling it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and (not os.path.exists(path) or _build.needs_build()):
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"liblife.so not built ({path}); run __graft_entry__.build() or "
                          "python -m paper_1905_06234_gb300.build")
    L = ctypes.CDLL(path)
    P, i64, i32, dbl, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int
    L.life_build_index.argtypes = [P, P, P, P, i64, i32, i32, i32, i32, P, ctypes.POINTER(life_opts), P,
                                   ctypes.POINTER(P)]
    L.life_index_free.argtypes = [P]
    L.life_index_get_info.argtypes = [P, ctypes.POINTER(life_index_info)]
    L.life_index_export.argtypes = [P, i32, P, P, P, P, P]
    L.life_index_export_voxel_streams.argtypes = [P, P, P, P, P, P]
    L.life_index_export_tiles.argtypes = [P, P, P, P, P, P, P, P, P, P, P]
    L.life_dsc.argtypes = [P, P, P, P, P, P, P]
    L.life_wc.argtypes = [P, P, P, P, P, P]
    L.life_dsc_grad_D.argtypes = [P, P, P, P, P]
    L.life_dsc_grad_D_noalloc.argtypes = [P, P, P, P, P]
    L.life_dictionary.argtypes = [i32, i32, P, P, dbl, dbl, P, P, P]
    L.life_dot_f32.argtypes = [i64, P, P, P, P]
    L.life_sbb_workspace_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    L.life_sbb_state_init.argtypes = [P, P]
    L.life_sbb_state_resume.argtypes = [P, i32, P]
    L.life_sbbnnls_step.argtypes = [P, P, P, P, P, P, dbl, i32, P]
    L.life_sbbnnls_solve.argtypes = [P, P, P, P, i64, dbl, i32, P, P, P]
    L.life_batch_create.argtypes = [i32, P, ctypes.POINTER(life_opts), P, ctypes.POINTER(P)]
    L.life_batch_free.argtypes = [P]
    L.life_batch_get_info.argtypes = [P, ctypes.POINTER(life_batch_info)]
    L.life_batch_offsets.argtypes = [P, P, P]
    L.life_batch_index.argtypes = [P, ctypes.POINTER(P)]
    L.life_batch_workspace_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    L.life_batch_solve.argtypes = [P, P, P, P, i64, dbl, i32, P, P, P]
    L.life_index_autotune.argtypes = [P, P]
    L.life_selftest_bounded_wait.argtypes = [i64, P]
    L.life_check_device_status.argtypes = [P]
    L.life_index_sparse_stats.argtypes = [P, P, P]
    L.life_build_index_shard.argtypes = [P, P, P, P, i64, i32, i32, i32, i32, P, i32, i32,
                                         ctypes.POINTER(life_opts), P, ctypes.POINTER(P)]
    L.life_sbb_shard_phase.argtypes = [P, P, P, P, P, P, P, P, P, dbl, i32, i32, P]
    L.life_prune.argtypes = [i32, P, ctypes.c_float, P, P, P, P, P]
    L.life_voxel_rmse.argtypes = [i32, i32, P, P, P, P]
    L.life_last_error.restype = ctypes.c_char_p
    L.life_version.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("life_last_error", "life_version"):
            getattr(L, name).restype = st
    _lib = L
    return L


def _check(status):
    if status != LIFE_OK:
        msg = _lib.life_last_error().decode(errors="replace")
        raise LifeError(status, msg)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("liblife takes CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("liblife takes contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t, dtype, numel, name):
    if t is None:
        raise ValueError(f"{name} is required")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t


class LifeIndex:
    """Owner of a life_index handle (freed on close() or garbage collection)."""

    def __init__(self, handle, lib):
        self._h = handle
        self._lib = lib
        i = self.info()
        self.nnz = i["nnz"]
        self.n_theta, self.n_atoms = i["n_theta"], i["n_atoms"]
        self.n_voxels, self.n_fasc = i["n_voxels"], i["n_fasc"]
        self.precision, self.algo = i["precision"], i["algo"]

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("index already freed")
        return self._h

    def info(self) -> dict:
        out = life_index_info()
        _check(self._lib.life_index_get_info(self.handle, ctypes.byref(out)))
        return {k: getattr(out, k) for k, _ in life_index_info._fields_}

    def close(self):
        if self._h is not None:
            self._lib.life_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------------ the ABI

def life_build_index(atom, voxel, fasc, val, n_theta, n_atoms, n_voxels, n_fasc, voxel_ijk=None,
                     precision=LIFE_FP32, algo=LIFE_ALGO_AUTO, brick_dim=0, wc_groups=0, autotune=False,
                     sparse_dsc=False, simt_kernels=0) -> LifeIndex:
    L = load()
    n = int(atom.numel())
    for t, dt, nm in ((atom, torch.int32, "atom"), (voxel, torch.int32, "voxel"), (fasc, torch.int32, "fasc"),
                      (val, torch.float32, "val")):
        _need(t, dt, n, nm)
    if voxel_ijk is not None:
        _need(voxel_ijk, torch.int32, 3 * n_voxels, "voxel_ijk")
    opts = life_opts(precision=int(precision), algo=int(algo), brick_dim=int(brick_dim), wc_groups=int(wc_groups),
                     autotune=1 if autotune else 0, sparse_dsc=1 if sparse_dsc else 0,
                     simt_kernels=int(simt_kernels))
    h = ctypes.c_void_p()
    _check(L.life_build_index(_ptr(atom), _ptr(voxel), _ptr(fasc), _ptr(val), n, int(n_theta), int(n_atoms),
                              int(n_voxels), int(n_fasc), _ptr(voxel_ijk), ctypes.byref(opts), _stream(),
                              ctypes.byref(h)))
    return LifeIndex(h, L)


def life_index_export(index: LifeIndex, layout=LIFE_LAYOUT_VOXEL):
    dev = torch.device("cuda")
    m = index.nnz
    a, v, f = (torch.empty(m, dtype=torch.int32, device=dev) for _ in range(3))
    x = torch.empty(m, dtype=torch.float32, device=dev)
    _check(load().life_index_export(index.handle, int(layout), _ptr(a), _ptr(v), _ptr(f), _ptr(x), _stream()))
    return a, v, f, x


def life_index_export_voxel_streams(index: LifeIndex):
    """(vox_ptr, atom, fasc, val) exactly as the CUDA-core kernels stream them."""
    dev = torch.device("cuda")
    m = index.nnz
    ptr = torch.empty(index.n_voxels + 1, dtype=torch.int32, device=dev)
    a, f = (torch.empty(m, dtype=torch.int32, device=dev) for _ in range(2))
    x = torch.empty(m, dtype=torch.float32, device=dev)
    _check(load().life_index_export_voxel_streams(index.handle, _ptr(ptr), _ptr(a), _ptr(f), _ptr(x), _stream()))
    return ptr, a, f, x


def life_index_export_tiles(index: LifeIndex) -> dict:
    """The tensor-core layout arrays (see include/life.h), as device tensors."""
    i = index.info()
    dev = torch.device("cuda")
    nt, nb, m = i["n_tiles"], i["n_bricks"], i["nnz"]
    out = dict(tile_vox=torch.empty(nt * 128, dtype=torch.int32, device=dev),
               chunk_ptr=torch.empty(nt * (i["n_sub"] // 4) + 1, dtype=torch.int32, device=dev),
               brick_tile_ptr=torch.empty(nb + 1, dtype=torch.int32, device=dev),
               brick_fasc_ptr=torch.empty(nb + 1, dtype=torch.int32, device=dev),
               brick_fasc=torch.empty(max(i["n_brick_fasc"], 1), dtype=torch.int32, device=dev),
               brick_order=torch.empty(max(nb, 1), dtype=torch.int32, device=dev),
               va=torch.empty(max(m, 1), dtype=torch.int16, device=dev),
               fl=torch.empty(max(m, 1), dtype=torch.int16, device=dev),
               val=torch.empty(max(m, 1), dtype=torch.float32, device=dev))
    _check(load().life_index_export_tiles(index.handle, *[_ptr(out[k]) for k in (
        "tile_vox", "chunk_ptr", "brick_tile_ptr", "brick_fasc_ptr", "brick_fasc", "brick_order", "va", "fl", "val")],
        _stream()))
    return out


def life_dsc(index: LifeIndex, D, w, b=None, y=None, want_y=True, sumsq=False):
    """y = M w (− b).  Returns (y or None, sumsq tensor or None)."""
    nt, nv = index.n_theta, index.n_voxels
    _need(D, torch.float32, nt * index.n_atoms, "D")
    _need(w, torch.float32, index.n_fasc, "w")
    if b is not None:
        _need(b, torch.float32, nt * nv, "b")
    if want_y and y is None:
        y = torch.empty(nt * nv, dtype=torch.float32, device=w.device)
    if y is not None:
        _need(y, torch.float32, nt * nv, "y")
    ss = torch.empty(1, dtype=torch.float64, device=w.device) if sumsq else None
    _check(load().life_dsc(index.handle, _ptr(D), _ptr(w), _ptr(b), _ptr(y), _ptr(ss), _stream()))
    return y, ss


def life_wc(index: LifeIndex, D, r, g=None, sumsq=False):
    """g = M^T r.  Returns (g, sumsq tensor or None)."""
    _need(D, torch.float32, index.n_theta * index.n_atoms, "D")
    _need(r, torch.float32, index.n_theta * index.n_voxels, "r")
    if g is None:
        g = torch.empty(index.n_fasc, dtype=torch.float32, device=r.device)
    _need(g, torch.float32, index.n_fasc, "g")
    ss = torch.empty(1, dtype=torch.float64, device=r.device) if sumsq else None
    _check(load().life_wc(index.handle, _ptr(D), _ptr(r), _ptr(g), _ptr(ss), _stream()))
    return g, ss


def life_dsc_grad_D(index: LifeIndex, gy, w, gD=None):
    _need(gy, torch.float32, index.n_theta * index.n_voxels, "gy")
    _need(w, torch.float32, index.n_fasc, "w")
    if gD is None:
        gD = torch.empty(index.n_theta * index.n_atoms, dtype=torch.float32, device=w.device)
    _check(load().life_dsc_grad_D(index.handle, _ptr(gy), _ptr(w), _ptr(gD), _stream()))
    return gD


def life_dsc_grad_D_noalloc(index: LifeIndex, gy, w, gD):
    """dL/dD into the caller's gD with no device allocation (see include/life.h)."""
    _need(gy, torch.float32, index.n_theta * index.n_voxels, "gy")
    _need(w, torch.float32, index.n_fasc, "w")
    _need(gD, torch.float32, index.n_theta * index.n_atoms, "gD")
    _check(load().life_dsc_grad_D_noalloc(index.handle, _ptr(gy), _ptr(w), _ptr(gD), _stream()))
    return gD


def life_dictionary(grad_dirs, atom_dirs, bval, lam, with_derivative=True):
    """(D, dD/dλ) as float32 column-major [θ + Nθ·a]."""
    g = grad_dirs.to(device="cuda", dtype=torch.float64).contiguous()
    u = atom_dirs.to(device="cuda", dtype=torch.float64).contiguous()
    nt, na = g.shape[0], u.shape[0]
    D = torch.empty(nt * na, dtype=torch.float32, device="cuda")
    dD = torch.empty(nt * na, dtype=torch.float32, device="cuda") if with_derivative else None
    _check(load().life_dictionary(nt, na, _ptr(g), _ptr(u), float(bval), float(lam), _ptr(D), _ptr(dD), _stream()))
    return D, dD


def life_dot_f32(x, y):
    out = torch.empty(1, dtype=torch.float64, device=x.device)
    _check(load().life_dot_f32(int(x.numel()), _ptr(x), _ptr(y), _ptr(out), _stream()))
    return out


def life_sbb_workspace_bytes(index: LifeIndex) -> int:
    n = ctypes.c_size_t()
    _check(load().life_sbb_workspace_bytes(index.handle, ctypes.byref(n)))
    return int(n.value)


def new_sbb_state(device="cuda"):
    """A device buffer for one life_sbb_state, initialised (it = 0, alpha = 1)."""
    st = torch.empty(SBB_STATE_BYTES, dtype=torch.uint8, device=device)
    life_sbb_state_init(st)
    return st


def new_sbb_workspace(index: LifeIndex):
    nbytes = life_sbb_workspace_bytes(index)
    return torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")


def _aligned(ws):
    p = ws.data_ptr()
    off = (-p) % 256
    return ctypes.c_void_p(p + off)


def life_sbb_state_init(st):
    _check(load().life_sbb_state_init(_ptr(st), _stream()))


def life_sbb_state_resume(st, n: int = 1):
    """Clears the stop flag of n device states (see include/life.h)."""
    _need(st, torch.uint8, n * SBB_STATE_BYTES, "st")
    _check(load().life_sbb_state_resume(_ptr(st), int(n), _stream()))


def read_sbb_state(st) -> dict:
    raw = bytes(st.cpu().numpy().tobytes())
    s = life_sbb_state.from_buffer_copy(raw)
    return {k: getattr(s, k) for k, _ in life_sbb_state._fields_}


def life_sbbnnls_step(index: LifeIndex, D, b, w, st, workspace, tol=0.0, eq7_on_even=True):
    _check(load().life_sbbnnls_step(index.handle, _ptr(D), _ptr(b), _ptr(w), _ptr(st), _aligned(workspace),
                                    float(tol), 1 if eq7_on_even else 0, _stream()))


def life_sbbnnls_solve(index: LifeIndex, D, b, w, max_iter, st, workspace, tol=0.0, eq7_on_even=True):
    _check(load().life_sbbnnls_solve(index.handle, _ptr(D), _ptr(b), _ptr(w), int(max_iter), float(tol),
                                     1 if eq7_on_even else 0, _ptr(st), _aligned(workspace), _stream()))


def life_index_sparse_stats(index: LifeIndex) -> dict:
    """Counters of the live-entry DSC stream (see include/life.h)."""
    out = (ctypes.c_int64 * 6)()
    _check(load().life_index_sparse_stats(index.handle, out, _stream()))
    keys = ("calls", "compact_calls", "rebuilds", "live_entries", "entries", "live_slots")
    return dict(zip(keys, (int(x) for x in out)))


def life_check_device_status():
    _check(load().life_check_device_status(_stream()))


def life_version() -> str:
    return load().life_version().decode()


def life_index_autotune(index: LifeIndex):
    """Re-tunes the tile layout of a tensor-core index on this GPU (no-op otherwise)."""
    _check(load().life_index_autotune(index.handle, _stream()))
    return index.info()


# ----------------------------------------------------------------- batches

class LifeBatch:
    """Owner of a life_batch handle: several problems solved together."""

    def __init__(self, handle, lib):
        self._h = handle
        self._lib = lib
        i = self.info()
        self.n = i["n"]
        vo = (ctypes.c_int32 * (self.n + 1))()
        fo = (ctypes.c_int32 * (self.n + 1))()
        _check(lib.life_batch_offsets(handle, vo, fo))
        self.vox_off = list(vo)
        self.fasc_off = list(fo)
        ih = ctypes.c_void_p()
        _check(lib.life_batch_index(handle, ctypes.byref(ih)))
        self.index = _BorrowedIndex(ih, lib, self)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("batch already freed")
        return self._h

    def info(self) -> dict:
        out = life_batch_info()
        _check(self._lib.life_batch_get_info(self.handle, ctypes.byref(out)))
        return {k: getattr(out, k) for k, _ in life_batch_info._fields_ if k != "reserved"}

    def close(self):
        if self._h is not None:
            self._lib.life_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _BorrowedIndex(LifeIndex):
    """The combined index of a batch (owned by the batch, never freed here)."""

    def __init__(self, handle, lib, owner):
        self._owner = owner
        super().__init__(handle, lib)

    @property
    def handle(self):
        if self._owner._h is None:
            raise ValueError("batch already freed")
        return self._h

    def close(self):
        """Nothing to free: the batch owns the combined index."""


def life_batch_create(indices, algo=LIFE_ALGO_AUTO, brick_dim=0, wc_groups=0,
                      autotune=False) -> LifeBatch:
    L = load()
    n = len(indices)
    arr = (ctypes.c_void_p * n)(*[ix.handle for ix in indices])
    opts = life_opts(algo=int(algo), brick_dim=int(brick_dim), wc_groups=int(wc_groups),
                     autotune=1 if autotune else 0)
    h = ctypes.c_void_p()
    _check(L.life_batch_create(n, arr, ctypes.byref(opts), _stream(), ctypes.byref(h)))
    return LifeBatch(h, L)


def new_batch_workspace(batch: LifeBatch):
    n = ctypes.c_size_t()
    _check(load().life_batch_workspace_bytes(batch.handle, ctypes.byref(n)))
    return torch.empty(n.value + 256, dtype=torch.uint8, device="cuda")


def new_batch_states(n: int):
    """n device SBB states, initialised (it = 0, alpha = 1)."""
    st = torch.zeros(n * SBB_STATE_BYTES, dtype=torch.uint8, device="cuda")
    for p in range(n):
        _check(load().life_sbb_state_init(ctypes.c_void_p(st.data_ptr() + p * SBB_STATE_BYTES), _stream()))
    return st


def read_batch_states(st, n: int) -> list:
    raw = st.cpu().numpy().tobytes()
    out = []
    for p in range(n):
        s = life_sbb_state.from_buffer_copy(raw[p * SBB_STATE_BYTES:(p + 1) * SBB_STATE_BYTES])
        out.append({k: getattr(s, k) for k, _ in life_sbb_state._fields_})
    return out


def life_batch_solve(batch: LifeBatch, D, bs, ws, max_iter, st, workspace, tol=0.0, eq7_on_even=True):
    """Solves every problem of the batch in one graph launch; ws[p] updated in place."""
    n = batch.n
    if len(bs) != n or len(ws) != n:
        raise ValueError(f"need {n} signals and {n} weight vectors")
    nt = batch.index.n_theta
    _need(D, torch.float32, nt * batch.index.n_atoms, "D")
    for p in range(n):
        _need(bs[p], torch.float32, nt * (batch.vox_off[p + 1] - batch.vox_off[p]), f"b[{p}]")
        _need(ws[p], torch.float32, batch.fasc_off[p + 1] - batch.fasc_off[p], f"w[{p}]")
    _need(st, torch.uint8, n * SBB_STATE_BYTES, "st")
    bp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in bs])
    wp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in ws])
    _check(load().life_batch_solve(batch.handle, _ptr(D), bp, wp, int(max_iter), float(tol),
                                   1 if eq7_on_even else 0, _ptr(st), _aligned(workspace), _stream()))


def life_selftest_bounded_wait(limit_ns: int):
    """Runs a wait that cannot complete, bounded to limit_ns (see include/life.h)."""
    _check(load().life_selftest_bounded_wait(int(limit_ns), _stream()))


# ------------------------------------------------------ connectome evaluation

def life_prune(w, threshold=0.0):
    """(keep uint8 [Nf], kept int32 ids in increasing order, w_pruned) for w > threshold."""
    _need(w, torch.float32, w.numel(), "w")
    nf = int(w.numel())
    keep = torch.empty(nf, dtype=torch.uint8, device=w.device)
    kept = torch.empty(max(nf, 1), dtype=torch.int32, device=w.device)
    n_kept = torch.empty(1, dtype=torch.int64, device=w.device)
    w_pruned = torch.empty(nf, dtype=torch.float32, device=w.device)
    _check(load().life_prune(nf, _ptr(w), float(threshold), _ptr(keep), _ptr(kept), _ptr(n_kept), _ptr(w_pruned),
                             _stream()))
    return keep, kept[:int(n_kept.item())], w_pruned


def life_voxel_rmse(e, n_theta: int, n_voxels: int):
    """(rmse float32 [Nv], Σ e² as a float64 device tensor) of a residual e = M w − b."""
    _need(e, torch.float32, n_theta * n_voxels, "e")
    rmse = torch.empty(n_voxels, dtype=torch.float32, device=e.device)
    ss = torch.empty(1, dtype=torch.float64, device=e.device)
    _check(load().life_voxel_rmse(int(n_theta), int(n_voxels), _ptr(e), _ptr(rmse), _ptr(ss), _stream()))
    return rmse, ss


def evaluate_connectome(index: LifeIndex, D, w, b, threshold=0.0):
    """LiFE's evaluation of a fitted connectome: the pruned model (fascicles with
    w > threshold) and its per-voxel prediction error.  Returns a dict with the
    kept fascicle ids, the pruned weights, the residual of the pruned model
    e = M w_pruned − b, its per-voxel RMSE and the global RMSE."""
    keep, kept, w_pruned = life_prune(w, threshold)
    e, _ = life_dsc(index, D, w_pruned, b=b)
    rmse, ss = life_voxel_rmse(e, index.n_theta, index.n_voxels)
    n = index.n_theta * index.n_voxels
    return dict(keep=keep, kept=kept, w_pruned=w_pruned, e=e, rmse=rmse,
                global_rmse=float((ss / max(n, 1)).sqrt().item()))


# ------------------------------------------------------- voxel-sharded solve

def life_build_index_shard(atom, voxel, fasc, val, n_theta, n_atoms, n_voxels, n_fasc, v_begin, v_end,
                           voxel_ijk=None, precision=LIFE_FP32, algo=LIFE_ALGO_AUTO, brick_dim=0) -> LifeIndex:
    """Index over voxels [v_begin, v_end) of a problem given as device COO arrays."""
    L = load()
    n = int(atom.numel())
    for t, dt, nm in ((atom, torch.int32, "atom"), (voxel, torch.int32, "voxel"), (fasc, torch.int32, "fasc"),
                      (val, torch.float32, "val")):
        _need(t, dt, n, nm)
    if voxel_ijk is not None:
        _need(voxel_ijk, torch.int32, 3 * n_voxels, "voxel_ijk")
    opts = life_opts(precision=int(precision), algo=int(algo), brick_dim=int(brick_dim))
    h = ctypes.c_void_p()
    _check(L.life_build_index_shard(_ptr(atom), _ptr(voxel), _ptr(fasc), _ptr(val), n, int(n_theta), int(n_atoms),
                                    int(n_voxels), int(n_fasc), _ptr(voxel_ijk), int(v_begin), int(v_end),
                                    ctypes.byref(opts), _stream(), ctypes.byref(h)))
    return LifeIndex(h, L)


def life_sbb_shard_phase(index: LifeIndex, D, b, w, g, u, scal, st, workspace, phase, tol=0.0, eq7_on_even=True):
    """Phase 1, 2 or 3 of a sharded SBB-NNLS iteration (see include/life.h)."""
    _need(g, torch.float32, index.n_fasc, "g")
    _need(u, torch.float32, index.n_fasc, "u")
    _need(scal, torch.float64, 2, "scal")
    _check(load().life_sbb_shard_phase(index.handle, _ptr(D), _ptr(b), _ptr(w), _ptr(g), _ptr(u), _ptr(scal),
                                       _ptr(st), _aligned(workspace), float(tol), 1 if eq7_on_even else 0, int(phase),
                                       _stream()))
