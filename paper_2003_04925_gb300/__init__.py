"""GB300 (sm_103a) implementation of the perfectly parallel sCOLA method
(Leclercq et al., arXiv:2003.04925): per-tile particle-mesh COLA evolution of
independent sCOLA boxes with Dirichlet boundary conditions.

The compute path is the CUDA library ``libscola.so`` (C ABI in
``include/scola.h``); ``binding`` marshals arguments to it, and ``Scola``
below adds device-memory management with PyTorch tensors.  Importing the
package fails loudly if the library has not been built.
"""
from .binding import (  # noqa: F401
    EXPORTED, KERNEL_CLASSES, SCOLA_BATCH_ALL, SCOLA_BATCH_PER_TILE, SCOLA_DEPOSIT_ATOMIC,
    SCOLA_DEPOSIT_AUTO, SCOLA_DEPOSIT_SORTED, SCOLA_STEPPING_MODIFIED, SCOLA_STEPPING_STANDARD, SCOLA_DST_AUTO, SCOLA_DST_SIMT,
    SCOLA_STUDY_NONE, SCOLA_STUDY_TRUE_DENSITY, SCOLA_STUDY_TRUE_POTENTIAL,
    SCOLA_DST_TC_3XTF32, SCOLA_DST_TC_4XTF32, SCOLA_DST_TC_3PASS, SCOLA_DST_RADIX, ScolaError, ScolaParams, make_params,
    scola_backward, scola_backward_density, scola_checkpoint_interval, scola_box_density_noalloc, scola_box_mass, scola_box_offsets, scola_box_particle_count, scola_box_particle_ids,
    scola_create, scola_density_adjoint, scola_destroy, scola_device_status, scola_final_density, scola_forward,
    scola_forward_host, scola_generate_white_noise, scola_get_stats, scola_kernel_times, scola_last_error, scola_lpt_fields,
    scola_mesh_cell_count, scola_padded_cell_count, scola_pm_force, scola_power_spectrum, scola_selftest_conversions, scola_selftest_wait_timeout,
    scola_set_checkpoint_interval, scola_set_checkpointing, scola_set_profiling, scola_shard_ranges, scola_setup_boxes, scola_status_string,
    scola_tcola, scola_tcola_kernel_times, TCOLA_STAGES, scola_tiling_info, scola_time_table, scola_uses_tensor_cores,
)
from .simulation import Scola, ScolaDensity, ScolaState  # noqa: F401
