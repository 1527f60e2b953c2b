"""Real spherical harmonics up to degree 3, float64 (torch or numpy arrays).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper adopts the base 3DGS colour model unchanged (Supp. "Implementation
Details"): view-dependent colour c(d) = max(0, sum_lm k_lm Y_lm(d) + 1/2) with
real orthonormal spherical harmonics of the unit view direction d. The basis
below uses the sign convention of that base method, which is the real basis
Y_l,-m = sqrt(2) Im Y_l^m, Y_l0 = Y_l^0, Y_l,m = sqrt(2) Re Y_l^m (m > 0) built
from the complex harmonics with the Condon-Shortley phase; coefficients are
ordered l = 0..3, m = -l..l. Normalisation constants are written as closed
forms.
"""
from __future__ import annotations

import math

PI = math.pi
C0 = 1.0 / (2.0 * math.sqrt(PI))
C1 = math.sqrt(3.0 / (4.0 * PI))
C2 = [0.5 * math.sqrt(15.0 / PI), -0.5 * math.sqrt(15.0 / PI), 0.25 * math.sqrt(5.0 / PI),
      -0.5 * math.sqrt(15.0 / PI), 0.25 * math.sqrt(15.0 / PI)]
C3 = [-0.25 * math.sqrt(35.0 / (2.0 * PI)), 0.5 * math.sqrt(105.0 / PI),
      -0.25 * math.sqrt(21.0 / (2.0 * PI)), 0.25 * math.sqrt(7.0 / PI),
      -0.25 * math.sqrt(21.0 / (2.0 * PI)), 0.25 * math.sqrt(105.0 / PI),
      -0.25 * math.sqrt(35.0 / (2.0 * PI))]


def basis(x, y, z, degree: int):
    """List of (degree+1)^2 arrays Y_k(x, y, z) for a unit direction."""
    out = [C0 + 0.0 * x]
    if degree >= 1:
        out += [-C1 * y, C1 * z, -C1 * x]
    if degree >= 2:
        xx, yy, zz = x * x, y * y, z * z
        out += [C2[0] * x * y, C2[1] * y * z, C2[2] * (2.0 * zz - xx - yy),
                C2[3] * x * z, C2[4] * (xx - yy)]
    if degree >= 3:
        xx, yy, zz = x * x, y * y, z * z
        out += [C3[0] * y * (3.0 * xx - yy), C3[1] * x * y * z,
                C3[2] * y * (4.0 * zz - xx - yy), C3[3] * z * (2.0 * zz - 3.0 * xx - 3.0 * yy),
                C3[4] * x * (4.0 * zz - xx - yy), C3[5] * z * (xx - yy),
                C3[6] * x * (xx - 3.0 * yy)]
    return out
