"""GB300 (sm_103a) LiFE hot path: DSC (y = M w), WC (g = M^T r) and SBB-NNLS.

The computation lives in the C-ABI CUDA library ``lib/liblife.so`` (declared in
``include/life.h``); this package is its thin Python binding plus an autograd
wrapper.  Build the library with ``python -m paper_1905_06234_gb300.build``.
"""
from ._native import (  # noqa: F401
    EXPORTS, LIFE_ALGO_AUTO, LIFE_ALGO_SIMT, LIFE_ALGO_TC, LIFE_BF16, LIFE_FP32, LIFE_LAYOUT_ATOM,
    LIFE_LAYOUT_FIBER, LIFE_LAYOUT_VOXEL, LifeError, LifeIndex, life_build_index, life_check_device_status,
    life_dictionary, life_dot_f32, life_dsc, life_dsc_grad_D, life_dsc_grad_D_noalloc, life_index_export, life_index_export_tiles, life_index_export_voxel_streams, life_sbb_state_init,
    life_sbb_workspace_bytes, life_sbbnnls_solve, life_sbbnnls_step, life_version, life_wc, load, new_sbb_state,
    new_sbb_workspace, read_sbb_state, LifeBatch, life_batch_create, life_batch_solve, life_index_autotune,
    new_batch_states, new_batch_workspace, read_batch_states, life_selftest_bounded_wait,
    life_prune, life_voxel_rmse, evaluate_connectome, life_index_sparse_stats,
    life_build_index_shard, life_sbb_shard_phase, life_sbb_state_resume,
)
from .autograd import LifeDSC, LifeDictionary, dictionary, dsc  # noqa: F401
from .problem import index_from_arrays, upload_problem  # noqa: F401
