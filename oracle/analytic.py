"""Host-side closed forms of the paper used to set up cases for the oracle.

TEST INFRASTRUCTURE ONLY (part of the oracle).  Each function cites the
passage it restates; the tests pin them against the numbers the paper prints
(Sec. 2.4 and Table A1) and against limits that the formulas must satisfy.
"""
import numpy as np

from .oracle import bessel_j01

CS2 = 1.0 / 3.0  # Sec. 2.1: c_s = 1/sqrt(3)


def tau_from_physical(nu, dx, dt):
    """Eq. (Viscosity) in lattice units: nu dt/dx^2 = c_s^2 (tau - 1/2)."""
    return 0.5 + nu * dt / (dx * dx) / CS2


def viscosity(tau):
    """Eq. (Viscosity): lattice kinematic viscosity nu = c_s^2 (tau - 1/2)."""
    return CS2 * (tau - 0.5)


def womersley_number(radius, omega, rho, mu):
    """Sec. 2.2: alpha = R sqrt(omega rho / mu)."""
    return radius * np.sqrt(omega * rho / mu)


def tube_law_coefficient(radius, young, thickness, poisson):
    """Sec. 2.4: dE = (1 - sigma^2) R^2 / (Y h) (p - P0); returns the factor multiplying (p - P0)."""
    return (1.0 - poisson ** 2) * radius ** 2 / (young * thickness)


def kappa_lattice(r0, eh_over_r0, poisson=0.5):
    """The Sec. 2.4 coefficient written with the stiffness parameter Eh/r0:
    (1 - sigma^2) R^2/(E h) = (1 - sigma^2) r0 / (E h / r0)."""
    return (1.0 - poisson ** 2) * r0 / eh_over_r0


def f_ratio(alpha, dr_over_R, M):
    """Sec. 2.3, the ratio F = (1 - M) / (1 - M J0(Lambda (1 - dr/R)) / J0(Lambda)),
    Lambda = i^(3/2) alpha (the garbled "d dr" of the printed second form read as dr)."""
    lam = alpha * np.exp(1j * 3.0 * np.pi / 4.0)
    j0L, _ = bessel_j01(lam)
    j0r, _ = bessel_j01(lam * (1.0 - dr_over_R))
    return (1.0 - M) / (1.0 - M * j0r / j0L)
