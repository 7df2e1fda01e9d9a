"""Brute-force pairwise force (test pin for the PM force only).

Newtonian attraction in the code units of mesh.py: lap Phi = (3/2) Omega_m
rho gives F = -(3 Omega_m / (8 pi)) m_j (x_i - x_j) / |x_i - x_j|^3 per pair,
nearest periodic image only.  The paper disables its PP force (Section 3);
this is not part of the method.
"""
import numpy as np


def pp_force(pos, n, mass, omega_m):
    pos = np.asarray(pos, dtype=np.float64)
    npart = pos.shape[1]
    out = np.zeros_like(pos)
    g = 3.0 * omega_m / (8.0 * np.pi) * mass
    for i in range(npart):
        d = pos - pos[:, i:i + 1]
        d -= n * np.round(d / n)
        r2 = np.sum(d * d, axis=0)
        r2[i] = np.inf
        out[:, i] = g * np.sum(d / r2 ** 1.5, axis=1)
    return out
