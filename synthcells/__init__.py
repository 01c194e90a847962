"""Seeded synthetic inputs shared by the oracle and the CUDA path.

Holds no arithmetic of the J/K method: only geometry, basis draws and
Gaussian matrices.  See ``cells.py``.
"""
from .cells import (BOHR_PER_ANGSTROM, Cell, Shell, config, density_from_overlap, density_perturbation,
                    diamond_cell, large_cell, ncart, nuclear_charges, serving_requests, small_random_cell, tiny_cell,
                    water_cell)
from .rng import MASTER_SEED, Stream, stream

__all__ = [
    "BOHR_PER_ANGSTROM", "Cell", "Shell", "config", "density_from_overlap", "density_perturbation", "diamond_cell",
    "large_cell", "ncart", "nuclear_charges", "serving_requests", "small_random_cell", "tiny_cell", "water_cell", "MASTER_SEED",
    "Stream", "stream",
]
