"""Scattering of a plane wave by a disk of constant contrast: the Mie (Bessel/Hankel) series.

Textbook closed form, used as an independent physical pin of the discrete
Lippmann-Schwinger solution (scattered field u of eq. Lippmann-Schwinger).
Inside the disk the total field is sum a_n J_n(k1 r) e^{i n phi}, outside it is
u_I + sum b_n H_n(w r) e^{i n phi}, k1 = w sqrt(1 + m0); a_n, b_n follow from the
continuity of the field and of its radial derivative at r = a.
"""
import math

import numpy as np
import scipy.special as sp


def mie_scattered(X, Z, omega, m0, a, theta, center=(0.5, 0.5), nterms=60):
    k1 = omega * math.sqrt(1.0 + m0)
    dx, dz = X - center[0], Z - center[1]
    r = np.hypot(dx, dz)
    ph = np.arctan2(dz, dx)
    u = np.zeros(X.shape, dtype=np.complex128)
    u_inc = np.exp(1j * omega * (X * math.cos(theta) + Z * math.sin(theta)))
    pre = np.exp(1j * omega * (center[0] * math.cos(theta) + center[1] * math.sin(theta)))
    out = r > a
    for nn in range(-nterms, nterms + 1):
        c = pre * (1j ** nn) * np.exp(-1j * nn * theta)   # plane-wave (Jacobi-Anger) coefficient
        J0, J0p = sp.jv(nn, omega * a), sp.jvp(nn, omega * a)
        J1, J1p = sp.jv(nn, k1 * a), sp.jvp(nn, k1 * a)
        H, Hp = sp.hankel1(nn, omega * a), sp.h1vp(nn, omega * a)
        b = c * (omega * J0p * J1 - k1 * J1p * J0) / (k1 * J1p * H - omega * Hp * J1)
        an = (c * J0 + b * H) / J1
        e = np.exp(1j * nn * ph)
        u[out] += b * sp.hankel1(nn, omega * r[out]) * e[out]
        u[~out] += an * sp.jv(nn, k1 * r[~out]) * e[~out]
    u[~out] -= u_inc[~out]
    return u
