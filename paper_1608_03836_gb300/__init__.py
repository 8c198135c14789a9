"""GB300-native weight-adjusted DG (WADG) right-hand side for curved tetrahedral meshes.

Chan, Hewett & Warburton, "Weight-adjusted discontinuous Galerkin methods:
curvilinear meshes" (arXiv:1608.03836).  The hot path (strong-weak volume and
surface terms, weight-adjusted mass inverse, LSRK(5,4) update) runs in the
hand-written CUDA kernels of libwadg.so behind the C ABI of include/wadg.h;
this package only marshals arguments.  Importing it loads the library and
raises ImportError when it has not been built: there is no CPU fallback.
"""
from ._lib import WadgError, load, LIB_PATH  # noqa: F401

load()

from .api import (  # noqa: E402,F401
    WADG_FP32,
    WADG_FP64,
    WADG_FP32_3XBF16,
    WADG_FP32_TF32,
    wadg_device_status,
    wadg_selftest_bounded_wait,
    BatchHandle,
    MeshHandle,
    wadg_batch_autotune,
    wadg_batch_create,
    wadg_batch_destroy,
    wadg_batch_info,
    wadg_batch_last_error,
    wadg_batch_set_grid,
    wadg_batch_set_rule,
    wadg_batch_solve,
    wadg_batch_step,
    wadg_energy,
    wadg_energy_noalloc,
    wadg_l2_error,
    wadg_last_error,
    wadg_mesh_create,
    wadg_mesh_destroy,
    wadg_project,
    wadg_reference_rules,
    wadg_receivers_adjoint,
    wadg_rhs,
    wadg_rhs_adjoint,
    wadg_set_operators,
    wadg_set_receivers,
    wadg_set_sources,
    wadg_solve,
    wadg_status_string,
    wadg_step,
    wadg_step_host,
    wadg_set_formulation,
    wadg_set_conservation,
    wadg_set_compensation,
    wadg_compensation_carry,
    wadg_set_planar_split,
    wadg_planar_info,
    FORMULATIONS,
    wadg_segment_adjoint,
    wadg_step_adjoint,
    wadg_step_record,
    wadg_version,
    wadg_volume_points,
)
