"""Oracle: Green's function, quadrature weights and the Lippmann-Schwinger apply.

Test infrastructure only (see oracle/__init__.py).  FP64 throughout.

Paper passages followed
  * Sec. 1, eq. Greens_function: G(x) = -(i/4) H_0^(1)(w |x|).
  * Sec. 1, eq. Lippmann-Schwinger: u + w^2 G*(m u) = -w^2 G*(m u_I).
  * Sec. 2: uniform grid x_{i,j} = (h i, h j); trapezoidal rule with only the
    diagonal weight modified (order h^4 log h); H = I + w^2 G D and
    f = -w^2 G D u_I (eq. discrete_Lipmann-Schwinger); G embedded in a
    Toeplitz matrix and applied by FFT.

Reading of the diagonal weight (the paper gives no constant).  G has the
singular expansion G(r) = (1/2pi) J_0(w r) log r + S(r) with S smooth and
S(0) = -i/4 + (log(w/2) + gamma)/(2 pi).  The generalised Euler-Maclaurin
expansion of the punctured lattice sum h^2 sum_{d != 0} phi(hd) log|hd| has the
leading defect h^2 (log h + Z'(0)/2) phi(0), where Z(s) = sum_{d != 0} |d|^{-2s}
is the square-lattice Epstein zeta function, Z(s) = 4 zeta(s) beta(s), so
Z'(0) = -log(2 pi) - 2 log(Gamma(1/4)^2 / (2 pi sqrt 2)).  Putting that defect
and h^2 S(0) on the diagonal gives
    G_w(0) = h^2 [ -i/4 + (log(w h / 2) + gamma + Z'(0)/2) / (2 pi) ],
the only single-weight correction whose rule converges at order h^4 (log h):
the tests check that order against adaptive quadrature of the exact integral.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special as sp

EULER_GAMMA = 0.57721566490153286061


def green(r, omega):
    """G(r) = -(i/4) H_0^(1)(omega r), r > 0 (Sec. 1, eq. Greens_function)."""
    return -0.25j * sp.hankel1(0, omega * np.asarray(r, dtype=np.float64))


def epstein_zeta_prime_0() -> float:
    """Z'(0) for the square lattice, Z(s) = 4 zeta(s) beta(s) (Dirichlet beta).

    zeta(0) = -1/2, zeta'(0) = -log(2 pi)/2, beta(0) = 1/2,
    beta'(0) = log(Gamma(1/4)^2 / (2 pi sqrt 2)).
    """
    beta_p0 = math.log(math.gamma(0.25) ** 2 / (2.0 * math.pi * math.sqrt(2.0)))
    return -math.log(2.0 * math.pi) - 2.0 * beta_p0


def diagonal_weight(h: float, omega: float) -> complex:
    """Corrected diagonal weight G_w(0) (Sec. 2; reading in the module docstring)."""
    c = math.log(omega * h / 2.0) + EULER_GAMMA + 0.5 * epstein_zeta_prime_0()
    return h * h * complex(c / (2.0 * math.pi), -0.25)


def kernel_weights(K: int, h: float, omega: float) -> np.ndarray:
    """Quadrature weights G_w(d) for offsets d = (dx, dz) in [-K, K]^2 (Sec. 2).

    Returns an array W of shape (2K+1, 2K+1) with W[dz+K, dx+K] = G_w(dx, dz):
    h^2 G(h |d|) off the diagonal (trapezoidal rule) and diagonal_weight at d = 0.
    """
    d = np.arange(-K, K + 1, dtype=np.float64)
    DZ, DX = np.meshgrid(d, d, indexing="ij")
    r = h * np.sqrt(DX * DX + DZ * DZ)
    W = np.empty(r.shape, dtype=np.complex128)
    nz = r > 0
    W[nz] = h * h * green(r[nz], omega)
    W[K, K] = diagonal_weight(h, omega)
    return W


def toeplitz_embedding(n: int, h: float, omega: float, P: int | None = None) -> np.ndarray:
    """Circulant embedding of the n x n (per axis) Toeplitz matrix G (Sec. 2).

    Gpad[b, a] = G_w(a~, b~) with a~ = a for a < n and a~ = a - P for a > P - n;
    other entries are zero.  P >= 2n - 1 (default 2n) makes the circular
    convolution on the P x P torus equal the linear one on the n x n grid.
    """
    P = 2 * n if P is None else P
    if P < 2 * n - 1:
        raise ValueError("P must be >= 2n-1")
    W = kernel_weights(n - 1, h, omega)
    Gpad = np.zeros((P, P), dtype=np.complex128)
    idx = np.arange(-(n - 1), n) % P
    Gpad[np.ix_(idx, idx)] = W
    return Gpad


def apply_G(v: np.ndarray, h: float, omega: float) -> np.ndarray:
    """(G v)_k = sum_p G_w(k - p) v_p on the n x n grid, by zero-padded FFT (Sec. 2)."""
    n = v.shape[0]
    P = 2 * n
    Gpad = toeplitz_embedding(n, h, omega, P)
    V = np.zeros((P, P), dtype=np.complex128)
    V[:n, :n] = v
    return np.fft.ifft2(np.fft.fft2(Gpad) * np.fft.fft2(V))[:n, :n]


def apply_G_direct(v: np.ndarray, h: float, omega: float) -> np.ndarray:
    """Same sum as apply_G, evaluated directly in O(N^2) (brute force, small n only)."""
    n = v.shape[0]
    W = kernel_weights(n - 1, h, omega)
    out = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        for i in range(n):
            # W[(j - p_z) + n - 1, (i - p_x) + n - 1] over all p
            out[j, i] = np.sum(W[j:j + n, i:i + n][::-1, ::-1] * v)
    return out


def apply_H(u: np.ndarray, m: np.ndarray, h: float, omega: float) -> np.ndarray:
    """H u = u + w^2 G (m u)  (Sec. 2, H = I + w^2 G D; eq. Lippmann-Schwinger)."""
    return u + omega * omega * apply_G(m * u, h, omega)


def incident_plane_wave(n: int, omega: float, theta: float) -> np.ndarray:
    """u_I(x) = exp(i w (x cos(theta) + z sin(theta))) at the nodes (Sec. 1, eq. Helmholtz_incoming)."""
    h = 1.0 / n
    c = h * np.arange(1, n + 1, dtype=np.float64)
    Z, X = np.meshgrid(c, c, indexing="ij")
    return np.exp(1j * omega * (X * math.cos(theta) + Z * math.sin(theta)))


def rhs(m: np.ndarray, h: float, omega: float, u_inc: np.ndarray) -> np.ndarray:
    """f = -w^2 G D u_I (Sec. 2)."""
    return -omega * omega * apply_G(m * u_inc, h, omega)


def spectrum(n: int, h: float, omega: float, P: int | None = None) -> np.ndarray:
    """Ghat = (w^2 / P^2) FFT2(Gpad): the spectral factor of the LS apply (Sec. 2).

    With it, H u = u + IFFT2_unnormalised(Ghat * FFT2(pad(m u)))[:n, :n].
    """
    P = 2 * n if P is None else P
    return (omega * omega / (P * P)) * np.fft.fft2(toeplitz_embedding(n, h, omega, P))


def dense_G(n: int, h: float, omega: float) -> np.ndarray:
    """Dense N x N matrix G with G[k, p] = G_w(k - p), k, p in x-fastest order (tiny n only)."""
    W = kernel_weights(n - 1, h, omega)
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    kz = jj.ravel()
    kx = ii.ravel()
    return W[(kz[:, None] - kz[None, :]) + n - 1, (kx[:, None] - kx[None, :]) + n - 1]


def apply_H_points(u: np.ndarray, m: np.ndarray, h: float, omega: float, points) -> np.ndarray:
    """(H u)_k at selected nodes k = (j, i) by the direct quadrature sum (Sec. 2), O(N) each."""
    n = u.shape[0]
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    mu = m * u
    out = []
    for (j, i) in points:
        r = h * np.sqrt((ii - i) ** 2.0 + (jj - j) ** 2.0)
        W = np.empty(r.shape, dtype=np.complex128)
        nz = r > 0
        W[nz] = h * h * green(r[nz], omega)
        W[~nz] = diagonal_weight(h, omega)
        out.append(u[j, i] + omega * omega * np.sum(W * mu))
    return np.array(out)


class Convolution:
    """apply_G / apply_H / rhs with the FFT of the Toeplitz embedding computed once (Sec. 2).

    Same arithmetic as the functions above (zero-padded P = 2n circulant
    embedding, numpy FFT), for large grids where re-evaluating the kernel
    weights on every call would dominate.
    """

    def __init__(self, n: int, h: float, omega: float):
        self.n, self.h, self.omega, self.P = n, h, omega, 2 * n
        self.Gf = np.fft.fft2(toeplitz_embedding(n, h, omega, self.P))

    def G(self, v: np.ndarray) -> np.ndarray:
        V = np.zeros((self.P, self.P), dtype=np.complex128)
        V[:self.n, :self.n] = v
        return np.fft.ifft2(self.Gf * np.fft.fft2(V))[:self.n, :self.n]

    def H(self, u: np.ndarray, m: np.ndarray) -> np.ndarray:
        return u + self.omega * self.omega * self.G(m * u)

    def rhs(self, m: np.ndarray, u_inc: np.ndarray) -> np.ndarray:
        return -self.omega * self.omega * self.G(m * u_inc)
