"""Moves a host-side LiFE problem (numpy COO arrays) to the device and builds its index."""
from __future__ import annotations

import numpy as np
import torch

from ._native import LIFE_ALGO_AUTO, LIFE_FP32, life_build_index


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def index_from_arrays(atom, voxel, fasc, val, n_theta, n_atoms, n_voxels, n_fasc, voxel_ijk=None,
                      precision=LIFE_FP32, algo=LIFE_ALGO_AUTO, brick_dim=0, sparse_dsc=False,
                      simt_kernels=0, autotune=False):
    """Builds a life index from host COO arrays (copied to the device first)."""
    ijk = None if voxel_ijk is None else _dev(np.asarray(voxel_ijk).reshape(-1), torch.int32)
    return life_build_index(_dev(atom, torch.int32), _dev(voxel, torch.int32), _dev(fasc, torch.int32),
                            _dev(val, torch.float32), n_theta, n_atoms, n_voxels, n_fasc, voxel_ijk=ijk,
                            precision=precision, algo=algo, brick_dim=brick_dim, sparse_dsc=sparse_dsc,
                            simt_kernels=simt_kernels, autotune=autotune)


def upload_problem(p, precision=LIFE_FP32, algo=LIFE_ALGO_AUTO, use_coords=True, brick_dim=0, sparse_dsc=False,
                   simt_kernels=0, autotune=False):
    """Index for a synthetic problem object with coo_* arrays and voxel_ijk."""
    return index_from_arrays(p.coo_atom, p.coo_voxel, p.coo_fasc, p.coo_val, p.n_theta, p.n_atoms, p.n_voxels,
                             p.n_fasc, voxel_ijk=p.voxel_ijk if use_coords else None, precision=precision,
                             algo=algo, brick_dim=brick_dim, sparse_dsc=sparse_dsc,
                             simt_kernels=simt_kernels, autotune=autotune)
