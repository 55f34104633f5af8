"""Pseudo-spectral solver of the periodic KS equation, Eq. KS_eq,
    rho_T = -rho rho_X - rho_XX - rho_XXXX  on [0, L),
by exponential time differencing with fourth-order Runge-Kutta stages
(ETDRK4, Cox & Matthews 2002), with the phi-functions evaluated by contour
integrals as proposed by Kassam & Trefethen (SIAM J. Sci. Comput. 26, 2005).

TEST INFRASTRUCTURE ONLY: an independent reference for the LB oracle on
small periodic lattices.  Written here from the published method.
"""
from __future__ import annotations

import numpy as np


class ETDRK4:
    def __init__(self, n: int, L: float, h: float, contour_points: int = 64, dealias: bool = True):
        self.n, self.L, self.h = n, L, h
        k = np.fft.rfftfreq(n, d=L / (2.0 * np.pi * n))  # physical wavenumbers 2 pi m / L
        self.k = k
        lin = k ** 2 - k ** 4  # linear symbol of -d2 - d4
        self.E = np.exp(h * lin)
        self.E2 = np.exp(h * lin / 2.0)
        # phi-type coefficients by the mean over a circle of radius 1 around each h*lin
        roots = np.exp(1j * np.pi * (np.arange(1, contour_points + 1) - 0.5) / contour_points)
        z = h * lin[:, None] + roots[None, :]
        ez = np.exp(z)
        self.Qc = h * np.real(np.mean((np.exp(z / 2.0) - 1.0) / z, axis=1))
        self.f1 = h * np.real(np.mean((-4.0 - z + ez * (4.0 - 3.0 * z + z ** 2)) / z ** 3, axis=1))
        self.f2 = h * np.real(np.mean((2.0 + z + ez * (z - 2.0)) / z ** 3, axis=1))
        self.f3 = h * np.real(np.mean((-4.0 - 3.0 * z - z ** 2 + ez * (4.0 - z)) / z ** 3, axis=1))
        g = -0.5j * k  # -(1/2) d/dX of rho^2
        if dealias:
            g = g * (np.arange(k.size) < (n // 3))  # 2/3 rule
        g[-1] = 0.0 if n % 2 == 0 else g[-1]  # no Nyquist derivative
        self.g = g

    def _nonlin(self, v):
        u = np.fft.irfft(v, n=self.n)
        return self.g * np.fft.rfft(u * u)

    def step(self, v):
        Nv = self._nonlin(v)
        a = self.E2 * v + self.Qc * Nv
        Na = self._nonlin(a)
        b = self.E2 * v + self.Qc * Na
        Nb = self._nonlin(b)
        c = self.E2 * a + self.Qc * (2.0 * Nb - Nv)
        Nc = self._nonlin(c)
        return self.E * v + Nv * self.f1 + 2.0 * (Na + Nb) * self.f2 + Nc * self.f3

    def run(self, u0: np.ndarray, T: float) -> np.ndarray:
        nsteps = int(round(T / self.h))
        if abs(nsteps * self.h - T) > 1e-9 * max(1.0, T):
            raise ValueError("T must be a multiple of h")
        v = np.fft.rfft(np.asarray(u0, dtype=np.float64))
        for _ in range(nsteps):
            v = self.step(v)
        return np.fft.irfft(v, n=self.n)


def solve(u0_fn, L: float, T: float, n: int = 256, h: float = 1e-3) -> tuple[np.ndarray, object]:
    """Solve from u0_fn(X) sampled on n points; returns (solution on the grid,
    callable that evaluates the band-limited solution at arbitrary X)."""
    X = np.arange(n) * (L / n)
    u = ETDRK4(n, L, h).run(u0_fn(X), T)
    uh = np.fft.rfft(u) / n

    def at(Xq):
        Xq = np.asarray(Xq, dtype=np.float64)
        m = np.arange(uh.size)
        w = np.where((m == 0) | ((n % 2 == 0) & (m == n // 2)), 1.0, 2.0)
        ph = np.exp(2j * np.pi * np.outer(Xq, m) / L)
        return np.real(ph @ (w * uh))

    return u, at
