"""Real orthonormal spherical harmonics for the anisotropic scattering source
(Eqs. (3)-(8) of Tano & Ragusa).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper expands the scattering kernel in Legendre polynomials and uses the
addition theorem P_n(Omega . Omega') = 4 pi / (2n + 1) sum_m Y_nm(Omega) Y*_nm(Omega')
to write the source with flux moments.  Any orthonormal basis of the degree-n
harmonics satisfies the theorem; the real one used here is
  Y_n0 = Y_n^0,   Y_nm = sqrt(2) (-1)^m Re Y_n^m,   Y_n,-m = sqrt(2) (-1)^m Im Y_n^m  (m > 0)
built from scipy's complex harmonics Y_n^m(theta, phi) (theta the polar angle from
the z axis, phi the azimuth in the x-y plane).  Moment k = n^2 + n + m.  yhat
returns them scaled by sqrt(4 pi), so that Yh_00 = 1 and moment 0 is the scalar
flux.
"""
import numpy as np
from scipy.special import sph_harm_y


def yhat(omega, L):
    """sqrt(4 pi) Y_k(Omega_d) for directions omega [ndir, 3], k < (L + 1)^2: [ndir, K]."""
    om = np.atleast_2d(np.asarray(omega, dtype=np.float64))
    theta = np.arccos(np.clip(om[:, 2], -1.0, 1.0))
    phi = np.arctan2(om[:, 1], om[:, 0])
    K = (L + 1) ** 2
    out = np.empty((om.shape[0], K))
    for n in range(L + 1):
        for m in range(-n, n + 1):
            k = n * n + n + m
            if m == 0:
                v = sph_harm_y(n, 0, theta, phi).real
            elif m > 0:
                v = np.sqrt(2.0) * (-1) ** m * sph_harm_y(n, m, theta, phi).real
            else:
                v = np.sqrt(2.0) * (-1) ** m * sph_harm_y(n, -m, theta, phi).imag
            out[:, k] = np.sqrt(4.0 * np.pi) * v
    return out


def order_of(k):
    return int(np.floor(np.sqrt(k) + 1e-12))
