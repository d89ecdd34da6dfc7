"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only draws random numbers and lays them out; it contains none of
the method's arithmetic (no integrals, no energies, no amplitudes).
"""
from .gen import (CONFIGS, System, make_system, make_displacements,
                  make_displacement_nontotsym, pack_dense, unpack_dense,
                  as_c1, irrep_split, chol_split, random_system)

__all__ = ["CONFIGS", "System", "make_system", "make_displacements",
           "make_displacement_nontotsym", "pack_dense", "unpack_dense",
           "as_c1", "irrep_split", "chol_split", "random_system"]
