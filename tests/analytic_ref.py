"""Textbook closed-form flows used as pins for the oracle (test helpers).

These are written from the classical solutions, not from the oracle, and use
library routines (numpy, scipy.special) where a special function is needed.
"""
import numpy as np


def duct_velocity(x, y, a, b, G, mu, terms=201):
    """Fully developed laminar flow in a rectangular duct -a<x<a, -b<y<b driven by
    G = -dp/dz (series solution, e.g. White, Viscous Fluid Flow, Sec. 3-3):

        u = 16 a^2 G/(mu pi^3) sum_{n odd} (-1)^((n-1)/2) / n^3
            [1 - cosh(n pi y/(2a)) / cosh(n pi b/(2a))] cos(n pi x/(2a)).
    """
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    u = np.zeros(np.broadcast(x, y).shape)
    for n in range(1, 2 * terms, 2):
        k = n * np.pi / (2.0 * a)
        # cosh ratio written with exponentials that do not overflow
        ratio = np.exp(k * (np.abs(y) - b)) * (1 + np.exp(-2 * k * np.abs(y))) / (1 + np.exp(-2 * k * b))
        u += (-1) ** ((n - 1) // 2) / n ** 3 * (1.0 - ratio) * np.cos(k * x)
    return 16.0 * a * a * G / (mu * np.pi ** 3) * u


def womersley_rigid(xi, alpha, u_mean, u_amp, theta):
    """Axial velocity in a rigid tube for the flow rate
    Q(t) = pi R^2 (u_mean + u_amp sin(theta)) (Womersley 1955; the Sec. 2.2
    expression with M = 1 and c -> infinity, written for a prescribed flow rate):

        u = u_mean 2 (1 - xi^2) + u_amp Im[ s(xi) e^(i theta) ],
        s(xi) = (1 - J0(L xi)/J0(L)) / (1 - 2 J1(L)/(L J0(L))),  L = i^(3/2) alpha.
    """
    from scipy.special import jv
    lam = alpha * np.exp(1j * 3 * np.pi / 4)
    s = (1 - jv(0, lam * xi) / jv(0, lam)) / (1 - 2 * jv(1, lam) / (lam * jv(0, lam)))
    return u_mean * 2 * (1 - xi ** 2) + u_amp * np.imag(s * np.exp(1j * theta))


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
