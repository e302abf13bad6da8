"""Seeded synthetic inputs for the transmission hot path.

This package only builds inputs: grids, synthetic Kohn-Sham potentials, absorbing
boundary (CAP) profiles, Monkhorst-Pack k-meshes, energy grids and sampled column
lists. It holds none of the transport method's arithmetic (no Hamiltonian, no solver,
no trace), so both the CPU oracle and the CUDA path can take their inputs from here
without sharing any of the computation they are compared on.
"""

from .configs import (  # noqa: F401
    Grid,
    Instance,
    fcc_sites,
    gaussian_potential,
    quadratic_cap,
    gaussian_cap,
    monkhorst_pack,
    sommerfeld_fermi,
    free_electron_slab,
    cu_bulk,
    cu_bulk_ideal,
    inversion_symmetrize,
    rh_point_contact,
    uneven_batch,
    small_instance,
    left_cap_columns,
    sample_columns,
    random_complex,
    config_seed,
)
