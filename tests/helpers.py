"""Shared test helpers: homogeneous test flows and small utilities (test code only)."""
from __future__ import annotations

import numpy as np

from paper_1006_0532_gb300 import synth

STATE_KEYS = ("x", "y", "u", "v", "w", "om", "psi")


def base_params(**kw) -> dict:
    p = dict(synth.TABLE4)
    p.update(nu=1e-4, c0_mode=1, C0=2.0, tm_mode=1, Cphi=2.0, Cs=0.02, Ct=0.7,
             src_x=0.5, src_y=0.5, src_r=0.02, bins=(4, 4, 4), min_per_bin=2, minnpel=0,
             interp_mode=0, source_on=1, seed=7, instance=0)
    p.update(kw)
    return p


def homogeneous_fields(grid, k, Omega, nu, CT=6.0, p_iso=None, U=(0.0, 0.0, 0.0),
                       dP=(0.0, 0.0), grad=None, lap=(0.0, 0.0, 0.0), omega_w=1.0):
    """Spatially constant fields with isotropic <u_i u_j> = 2k/3 and wp = p_iso * I.

    p_iso=None selects wp_ii = eps/2, which makes G_ij = 0 (Eq. 11).
    """
    eps = Omega * (k + nu * CT * CT * Omega)
    p = 0.5 * eps if p_iso is None else p_iso
    wp = np.eye(3) * p
    uu = (2.0 * k / 3.0,) * 3 + (0.0, 0.0, 0.0)
    return synth.uniform_fields(grid.nn, U=U, dP=dP, grad=grad, lap=lap, wp=wp, uu=uu,
                                omega=Omega, omega_w=omega_w), eps


def rel_err(a, b, scale):
    return np.abs(a - b) / np.maximum(np.abs(b), scale)


def period_diff(a, b, L):
    d = a - b
    if L > 0:
        d = (d + 0.5 * L) % L - 0.5 * L
    return d
