"""Degree-3 real spherical-harmonic colour, the 3DGS baseline representation
that the SG colour of Sec. 3.2 replaces (the comparison of Sec. 4 and Table 1).

TEST INFRASTRUCTURE ONLY (see sg_oracle.py).

The 16 basis functions are built from their definition, not from a table of
constants:

    Y_l^0 = K_l^0 P_l^0(z)
    Y_l^m = sqrt(2) K_l^m cos(m phi) P_l^m(z)          m > 0
    Y_l^m = sqrt(2) K_l^|m| sin(|m| phi) P_l^|m|(z)    m < 0
    K_l^m = sqrt((2l + 1) / (4 pi) * (l - m)! / (l + m)!)

with P_l^m the associated Legendre function including the Condon-Shortley
phase (-1)^m, z = cos(theta) and phi the azimuth of the unit direction
(x, y, z). On the unit sphere

    P_l^m(z) {cos, sin}(m phi) = (-1)^m (d^m P_l / dz^m)(z) {Re, Im}((x + i y)^m),

which is a polynomial in (x, y, z): it is evaluated that way, in float64
torch ops, so that autograd differentiates it everywhere (also at the poles).
Coefficient order: l = 0..3, m = -l..l (index l^2 + l + m).

The colour reading (the 3DGS convention the paper compares against):
c = max(0, 0.5 + sum_k Y_k(v) f_k) per channel, v the unit direction from the
camera centre to the Gaussian.
"""
from __future__ import annotations

import math

import numpy as np
import torch
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly

DEGREE = 3
N_COEFFS = (DEGREE + 1) ** 2


def _legendre_derivative_coeffs(l: int, m: int) -> np.ndarray:
    """Power-series coefficients of d^m P_l / dz^m."""
    c = np.zeros(l + 1)
    c[l] = 1.0
    return nppoly.polyder(npleg.leg2poly(c), m) if m > 0 else npleg.leg2poly(c)


def _norm(l: int, m: int) -> float:
    return math.sqrt((2 * l + 1) / (4.0 * math.pi) * math.factorial(l - m) / math.factorial(l + m))


def basis(v: torch.Tensor) -> torch.Tensor:
    """All 16 real SH basis values. v [..., 3] unit (float64) -> [..., 16]."""
    x, y, z = v.unbind(-1)
    # {Re, Im}((x + i y)^m) for m = 0..3
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for _ in range(DEGREE):
        r, i = re[-1], im[-1]
        re.append(r * x - i * y)
        im.append(r * y + i * x)
    out = []
    for l in range(DEGREE + 1):
        for m in range(-l, l + 1):
            a = abs(m)
            coeffs = _legendre_derivative_coeffs(l, a)
            dP = torch.zeros_like(z)
            for p, cp in enumerate(coeffs):   # power series in z
                if cp != 0.0:
                    dP = dP + float(cp) * z ** p
            cs = (-1.0) ** a
            if m == 0:
                out.append(_norm(l, 0) * dP)
            elif m > 0:
                out.append(math.sqrt(2.0) * _norm(l, a) * cs * dP * re[a])
            else:
                out.append(math.sqrt(2.0) * _norm(l, a) * cs * dP * im[a])
    return torch.stack(out, -1)


def sh3_color(sh: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    """Colour before the clamp: 0.5 + sum_k Y_k(v) f[ch, k].

    sh [N, 3, 16] float64 (per Gaussian, channel, coefficient), v [N, 3] unit.
    Returns [N, 3].
    """
    Y = basis(v)                                   # [N, 16]
    return 0.5 + (sh * Y[:, None, :]).sum(-1)
