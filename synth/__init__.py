"""Seeded synthetic inputs shared by the CUDA library's tests/bench and the oracle.

This package holds no arithmetic of the PM step itself: it only generates
particle initial conditions (Philox-keyed Gaussian random field + Zel'dovich
displacement) and names the workloads.
"""
from .philox import philox4x32, mode_gaussians
from .ics import (Cosmology, InitialConditions, einstein_de_sitter, lcdm_bbks,
                  zeldovich, sigma_delta_1d, white_noise_modes, linear_delta_k)
from .workloads import (WORKLOADS, Request, Workload, ensemble_c4, make_ics, rescaled_ics, serving_c5,
                        uniform_schedule)

__all__ = ["philox4x32", "mode_gaussians", "Cosmology", "InitialConditions",
           "einstein_de_sitter", "lcdm_bbks", "zeldovich", "sigma_delta_1d",
           "white_noise_modes", "linear_delta_k", "WORKLOADS", "Workload",
           "make_ics", "uniform_schedule", "ensemble_c4", "Request", "serving_c5",
           "rescaled_ics"]
