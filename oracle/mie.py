"""Mie series for a homogeneous sphere, optionally coated by a conductive sheet.

Textbook Lorenz-Mie theory (Bohren & Huffman, ch. 4), time convention
exp(-i w t) as in that book.  The sheet of surface conductivity sigma at r = a
changes the tangential-H condition to r x (H_out - H_in) = sigma E_tan (the
jump condition of Eq. 4 of the paper).  Solving the two interface conditions
per multipole order with Riccati-Bessel functions psi_n(x) = x j_n(x),
xi_n(x) = x h1_n(x) gives

    a_n = (psi - g psi') / (xi - g xi'),   g = m psi_n(mx)/psi_n'(mx) + i s,
    b_n = (psi' - f psi) / (xi' - f xi),   f = m psi_n'(mx)/psi_n(mx) - i s,

(unprimed psi, xi at x; s = sigma Z_out, dimensionless), which reduce to the
usual coefficients at s = 0 and to the perfectly conducting sphere
(a_n = psi'/xi', b_n = psi/xi) as s -> infinity.  Magnitudes of S1, S2 are
independent of the time convention, so they compare directly with the
exp(+jwt) boundary-element far field.
"""

from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def coefficients(m, x, s=0.0, nmax=None):
    if nmax is None:
        nmax = int(np.ceil(x + 4.05 * x ** (1 / 3) + 2))
    n = np.arange(1, nmax + 1)
    mx = m * x

    def psi(z):
        return z * spherical_jn(n, z), spherical_jn(n, z) + z * spherical_jn(n, z, derivative=True)

    def xi(z):
        h = spherical_jn(n, z) + 1j * spherical_yn(n, z)
        dh = spherical_jn(n, z, derivative=True) + 1j * spherical_yn(n, z, derivative=True)
        return z * h, h + z * dh

    px, dpx = psi(x)
    xx, dxx = xi(x)
    pm, dpm = psi(mx)
    g = m * pm / dpm + 1j * s
    f = m * dpm / pm - 1j * s
    a = (px - g * dpx) / (xx - g * dxx)
    b = (dpx - f * px) / (dxx - f * xx)
    return n, a, b


def amplitudes(m, x, theta, s=0.0):
    """S1(theta), S2(theta) (Bohren & Huffman Eq. 4.74)."""
    n, a, b = coefficients(m, x, s)
    mu = np.cos(np.asarray(theta, dtype=np.float64))
    nmax = len(n)
    pi = np.zeros((nmax + 1,) + mu.shape)
    tau = np.zeros((nmax + 1,) + mu.shape)
    pi[1] = 1.0
    tau[1] = mu
    for k in range(2, nmax + 1):
        pi[k] = (2 * k - 1) / (k - 1) * mu * pi[k - 1] - k / (k - 1) * pi[k - 2]
        tau[k] = k * mu * pi[k] - (k + 1) * pi[k - 1]
    c = (2 * n + 1) / (n * (n + 1))
    S1 = np.einsum("n,n...->...", c * a, pi[1:]) + np.einsum("n,n...->...", c * b, tau[1:])
    S2 = np.einsum("n,n...->...", c * a, tau[1:]) + np.einsum("n,n...->...", c * b, pi[1:])
    return S1, S2


def efficiencies(m, x, s=0.0):
    n, a, b = coefficients(m, x, s)
    qsca = 2.0 / x**2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    qext = 2.0 / x**2 * np.sum((2 * n + 1) * np.real(a + b))
    return qsca, qext
