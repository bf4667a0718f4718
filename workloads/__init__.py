"""Seeded synthetic workloads shared by the CUDA path's tests and the oracle's.

This package only builds inputs (initial fields and parameter sets).  It holds
none of the split-step method's arithmetic and imports neither the oracle nor
the CUDA library.
"""
from .rng import SplitMix64
from .ics import (KernelParams, Lump, Workload, coords, gaussian_lumps, centred_gaussian_2d,
                  head_on_collision_3d, nbody_3d, scan_instance_2d, random_small, SCAN_SIZES,
                  optical_beams_2d, random_fields)

__all__ = ["SplitMix64", "KernelParams", "Lump", "Workload", "coords", "gaussian_lumps",
           "centred_gaussian_2d", "head_on_collision_3d", "nbody_3d", "scan_instance_2d",
           "random_small", "SCAN_SIZES", "optical_beams_2d", "random_fields"]
