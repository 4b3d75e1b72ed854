"""Discrete Dirac delta functions used for grid transfer.

Test infrastructure only (see the package docstring).

* M4'  (Monaghan 1985), used for vortex regularization and interpolation
  (Sec. 2.1, Eq. vortexregularization; Fig. 1b, solid line).  The paper names
  the function without printing it; the standard piecewise cubic is used:
      1 - 5/2 r^2 + 3/2 |r|^3          for |r| <= 1
      1/2 (2 - |r|)^2 (1 - |r|)         for 1 < |r| <= 2
      0                                 otherwise.
* Smoothed three-point function (Yang et al. 2009), used for surface
  regularization R_s and interpolation E_s (Sec. 2.2.1; Fig. 1b, dashed line).
  Also not printed in the paper; the published closed form is used, support
  |r| < 2.  Both are pinned in the tests by their defining moment properties.
"""
import numpy as np


def m4prime(r):
    """M4' kernel, elementwise on an array of (signed) offsets in grid units."""
    a = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(a)
    inner = a <= 1.0
    outer = (a > 1.0) & (a <= 2.0)
    out[inner] = 1.0 - 2.5 * a[inner] ** 2 + 1.5 * a[inner] ** 3
    out[outer] = 0.5 * (2.0 - a[outer]) ** 2 * (1.0 - a[outer])
    return out


def yang3(r):
    """Smoothed three-point delta of Yang et al. (2009), elementwise."""
    a = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(a)
    s3 = np.sqrt(3.0)
    inner = a <= 1.0
    ai = a[inner]
    out[inner] = (17.0 / 48.0 + s3 * np.pi / 108.0 + ai / 4.0 - ai ** 2 / 4.0
                  + (1.0 - 2.0 * ai) / 16.0 * np.sqrt(np.maximum(-12.0 * ai ** 2 + 12.0 * ai + 1.0, 0.0))
                  - s3 / 12.0 * np.arcsin(s3 / 2.0 * (2.0 * ai - 1.0)))
    outer = (a > 1.0) & (a < 2.0)
    ao = a[outer]
    out[outer] = (55.0 / 48.0 - s3 * np.pi / 108.0 - 13.0 * ao / 12.0 + ao ** 2 / 4.0
                  + (2.0 * ao - 3.0) / 48.0 * np.sqrt(np.maximum(-12.0 * ao ** 2 + 36.0 * ao - 23.0, 0.0))
                  + s3 / 36.0 * np.arcsin(s3 / 2.0 * (2.0 * ao - 3.0)))
    return out
