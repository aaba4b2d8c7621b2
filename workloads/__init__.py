"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package generates inputs only: atom positions, atom types, box sides,
thermal velocities, random symmetric test matrices and the fixed model
constants of the water-like tight-binding recipe.  It holds none of the
method's arithmetic (no Hamiltonian, no density matrix, no charges, no
forces), so that the CPU oracle and the CUDA path can both consume the same
inputs while sharing no code that computes a result.
"""

from .water import (  # noqa: F401
    TYPE_O, TYPE_H, ModelParams, XLParams, WaterSystem,
    atom_counts, box_from_density, water_system, thermal_velocities,
    random_gapped_matrix, batch_sizes, serving_trajectories,
    water_24_atoms, water_2048_atoms, water_16384_atoms_morton, molecular_water, molecular_liquid,
    gapped_params, gapped_vapour, nonorth_params, isolated_clusters,
)
