"""GB300-native (sm_103a) Lienard-Wiechert hot path of PyCharge (arXiv 2107.12437).

The computation lives in libpycharge_gb300.so (C ABI: include/pycharge_gb300.h); `capi` is its
thin ctypes binding.  Names follow the header: pc_fields, pc_fields_plane, pc_dipoles_run,
pc_ke_fit, pc_dipoles_adjoint and pc_dipoles_rates_adjoint (with the autograd wrappers final_energy and
fitted_rates).
"""
from .capi import (  # noqa: F401
    PC_COULOMB,
    PC_F64,
    PC_MIXED,
    PC_RADIATION,
    PC_TOTAL,
    PC_TRAJ_ACCELERATING,
    PC_TRAJ_CIRCULAR,
    PC_TRAJ_OSCILLATING,
    PC_TRAJ_STATIONARY,
    Context,
    PcError,
    charges_to_device,
    dipoles_to_device,
    final_energy,
    fitted_rates,
    lo_config_to_device,
    load,
    pc_alu_peaks,
    pc_autotune_plane,
    pc_dipoles_adjoint,
    pc_dipoles_adjoint_moving,
    pc_dipoles_fields_adjoint,
    pc_dipoles_rates_adjoint,
    pc_dipoles_run,
    pc_dipoles_run_moving,
    pc_dipoles_state_size,
    pc_fields,
    pc_fields_noalloc,
    pc_fields_param,
    pc_set_plane_tiling,
    pc_fields_plane,
    pc_fields_plane_to_host,
    pc_fields_to_host,
    pc_ke_fit,
)
