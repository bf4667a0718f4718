"""FP64 CPU oracle of the split-step Schroedinger-Newton solver.

Test infrastructure only: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the CUDA library or its binding.
"""
from .sn_oracle import (dft_naive, fft_radix2, fftn, wavenumbers, k_squared, cell_volume,
                        green_multiplier, kinetic, potential, nonlinear, strang_step, evolve,
                        kernel_kwargs, observables, rel_l2, KIND_NMC, KIND_POISSON)

__all__ = ["dft_naive", "fft_radix2", "fftn", "wavenumbers", "k_squared", "cell_volume",
           "green_multiplier", "kinetic", "potential", "nonlinear", "strang_step", "evolve",
           "kernel_kwargs", "observables", "rel_l2", "KIND_NMC", "KIND_POISSON"]
