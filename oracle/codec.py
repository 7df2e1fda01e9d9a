"""Fixed-point position codes and arctan velocity codes (Sections 2.1, 2.2).

Oracle: plain FP64 restatement of Eqs. chi, x, nu, v.
"""
import numpy as np


# ---------------------------------------------------------------- positions (Eqs. chi, x)
def pos_decode(cell, chi, n_chi):
    """Eq. x: coordinate in coarse-cell units of a particle in coarse cell
    `cell` (0-based, i.e. n_c - 1) with code `chi`:
        x = cell + 2^(-8n) (chi + 2^(8n-1) + 1/2).
    """
    nb = 2 ** (8 * n_chi)
    return np.asarray(cell, dtype=np.float64) + (np.asarray(chi, dtype=np.float64) + nb / 2 + 0.5) / nb


def pos_encode(x, n_chi):
    """Eq. chi with [ ] read as the floor: returns (cell, chi) of a coordinate x
    in coarse-cell units,
        cell = floor(x),  chi = floor(2^(8n) (x - floor(x))) - 2^(8n-1).
    x - floor(x) and the power-of-two scaling are exact in FP64 for FP32 x.
    """
    x = np.asarray(x, dtype=np.float64)
    nb = 2 ** (8 * n_chi)
    cell = np.floor(x)
    frac = x - cell
    b = np.floor(frac * nb)
    return cell.astype(np.int64), (b - nb // 2).astype(np.int64)


def chi_dtype(n_chi):
    return np.int8 if n_chi == 1 else np.int16


# ---------------------------------------------------------------- velocities (Eqs. nu, v)
def nu_max(n_nu):
    """Largest code magnitude: |nu| <= 2^(8n-1) - 1 (M/2 = 127.5 for n = 1 maps
    to +-infinity, so it is never reached by a finite velocity)."""
    return 2 ** (8 * n_nu - 1) - 1


def vel_scale(sigma):
    """sqrt(pi / (2 sigma^2)) of Eq. nu, with sigma the per-dimension scale."""
    return np.sqrt(np.pi / (2.0 * sigma * sigma))


def vel_encode(dv, sigma, n_nu):
    """Eq. nu:  nu = nint( (2^(8n)-1)/pi * atan(dv * sqrt(pi/(2 sigma^2))) ).

    `dv` = v - v_c.  The nearest integer rounds halves away from zero; the
    result is clamped to +-(2^(8n-1)-1).
    """
    m = 2 ** (8 * n_nu) - 1
    x = (m / np.pi) * np.arctan(np.asarray(dv, dtype=np.float64) * vel_scale(sigma))
    nu = np.sign(x) * np.floor(np.abs(x) + 0.5)
    lim = nu_max(n_nu)
    return np.clip(nu, -lim, lim).astype(np.int64)


def vel_decode_offset(nu, sigma, n_nu):
    """Eq. v without v_c: tan(pi nu / (2^(8n)-1)) * sqrt(2 sigma^2 / pi)."""
    m = 2 ** (8 * n_nu) - 1
    return np.tan(np.pi * np.asarray(nu, dtype=np.float64) / m) * np.sqrt(2.0 * sigma * sigma / np.pi)


def vel_decode(nu, vc, sigma, n_nu):
    """Eq. v: v = v_c + tan(pi nu / (2^(8n)-1)) sqrt(2 sigma^2 / pi)."""
    return np.asarray(vc, dtype=np.float64) + vel_decode_offset(nu, sigma, n_nu)


def nu_dtype(n_nu):
    return np.int8 if n_nu == 1 else np.int16


# ---------------------------------------------------------------- codec scale snapping
def snap_sigma(sigma, floor=2.0 ** -30):
    """Snap a positive scale to the nearest 2^(m/16) in log2 (ties up).

    Reading of Section 2.2's nonlinear update: the measured scale only sets the
    codec's bin widths, so it is quantised to 1/16 octave; FP64 reduction-order
    noise then cannot change the codes.  Values below `floor` become `floor`.
    """
    s = max(float(sigma), floor)
    m = np.floor(16.0 * np.log2(s) + 0.5)
    return float(np.exp2(m / 16.0))
