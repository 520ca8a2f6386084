"""Closed-form velocity fields used as initial and Dirichlet data (input data only).

* Beltrami (Ethier-Steinman family) unsteady Navier-Stokes solution on [0,1]^3 with
  parameters a, d and viscosity nu; its exactness (divergence-free, zero momentum
  residual with the pressure below) is checked symbolically by the test-suite.
* A seeded solenoidal field v0 = curl(b Psi) with a wall bump b that vanishes with its
  gradient on the unit-cube boundary (no-slip compatible), Psi a sum of 64 Fourier modes.
* The Arnold-Beltrami-Childress flow of the paper's convergence test (Sec. 3.2, Eq. CT_1),
  2 pi-periodic in every direction; its exactness is checked symbolically by the test-suite.
"""
from dataclasses import dataclass

import numpy as np

from .mesh import splitmix64_doubles


@dataclass(frozen=True)
class BeltramiParams:
    a: float = np.pi / 4
    d: float = np.pi / 2
    nu: float = 0.1


def beltrami_velocity(x, t, prm: BeltramiParams):
    """Velocity (..., 3) at points x (..., 3) and time t (scalar or broadcastable)."""
    a, d, nu = prm.a, prm.d, prm.nu
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    f = np.exp(-nu * d * d * np.asarray(t, dtype=np.float64))
    u = -a * (np.exp(a * X) * np.sin(a * Y + d * Z) + np.exp(a * Z) * np.cos(a * X + d * Y)) * f
    v = -a * (np.exp(a * Y) * np.sin(a * Z + d * X) + np.exp(a * X) * np.cos(a * Y + d * Z)) * f
    w = -a * (np.exp(a * Z) * np.sin(a * X + d * Y) + np.exp(a * Y) * np.cos(a * Z + d * X)) * f
    return np.stack([u, v, w], axis=-1)


def beltrami_pressure(x, t, prm: BeltramiParams):
    """Kinematic pressure (up to a time-dependent constant) of the Beltrami solution."""
    a, d, nu = prm.a, prm.d, prm.nu
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    f2 = np.exp(-2.0 * nu * d * d * np.asarray(t, dtype=np.float64))
    s = (np.exp(2 * a * X) + np.exp(2 * a * Y) + np.exp(2 * a * Z)
         + 2 * np.sin(a * X + d * Y) * np.cos(a * Z + d * X) * np.exp(a * (Y + Z))
         + 2 * np.sin(a * Y + d * Z) * np.cos(a * X + d * Y) * np.exp(a * (Z + X))
         + 2 * np.sin(a * Z + d * X) * np.cos(a * Y + d * Z) * np.exp(a * (X + Y)))
    return -0.5 * a * a * s * f2


def abc_velocity(x, t, nu):
    """ABC flow (Eq. CT_1): u = sin z + cos y, v = sin x + cos z, w = sin y + cos x, times
    exp(-nu t).  Velocity (..., 3) at points x (..., 3)."""
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    f = np.exp(-nu * np.asarray(t, dtype=np.float64))
    return np.stack([(np.sin(Z) + np.cos(Y)) * f, (np.sin(X) + np.cos(Z)) * f, (np.sin(Y) + np.cos(X)) * f], axis=-1)


def abc_pressure(x, t, nu):
    """Kinematic pressure of the ABC flow (Eq. CT_1), up to a constant:
    -(cos x sin y + sin x cos z + sin z cos y) exp(-2 nu t)."""
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    f = np.exp(-2.0 * nu * np.asarray(t, dtype=np.float64))
    return -(np.cos(X) * np.sin(Y) + np.sin(X) * np.cos(Z) + np.sin(Z) * np.cos(Y)) * f


class SolenoidalModes:
    """v0 = curl(b Psi), Psi = sum_m |k_m|^-3 a_m sin(2 pi k_m . x + phi_m), b = B^2,
    B = 64 x(1-x) y(1-y) z(1-z); modes drawn from splitmix64(seed); scaled so that the
    maximum speed over the 33^3 lattice of [0,1]^3 equals `vmax`."""

    def __init__(self, seed: int = 1, modes: int = 64, kmax: int = 4, vmax: float = 0.1):
        ks, amps, phis = [], [], []
        u = splitmix64_doubles(seed, 64 * modes * 8)
        c = 0
        while len(ks) < modes:
            k = np.floor(u[c:c + 3] * (2 * kmax + 1)).astype(np.int64) - kmax
            av = 2.0 * u[c + 3:c + 6] - 1.0
            ph = 2.0 * np.pi * u[c + 6]
            c += 7
            if not k.any() or np.linalg.norm(av) < 1e-3:
                continue
            ks.append(k.astype(np.float64))
            amps.append(av / np.linalg.norm(av) * np.linalg.norm(k) ** -3.0)
            phis.append(ph)
        self.k = np.array(ks)
        self.a = np.array(amps)
        self.phi = np.array(phis)
        self.scale = 1.0
        g = np.linspace(0.0, 1.0, 33)
        P = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
        self.scale = vmax / np.max(np.linalg.norm(self(P), axis=-1))

    def __call__(self, x, t=0.0):
        x = np.asarray(x, dtype=np.float64)
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        B = 64.0 * X * (1 - X) * Y * (1 - Y) * Z * (1 - Z)
        dB = 64.0 * np.stack([(1 - 2 * X) * Y * (1 - Y) * Z * (1 - Z),
                              X * (1 - X) * (1 - 2 * Y) * Z * (1 - Z),
                              X * (1 - X) * Y * (1 - Y) * (1 - 2 * Z)], axis=-1)
        b = B * B
        db = 2.0 * B[..., None] * dB
        th = 2.0 * np.pi * (x @ self.k.T) + self.phi            # (..., M)
        psi = np.sin(th) @ self.a                               # (..., 3)
        curl_psi = np.cos(th) @ (2.0 * np.pi * np.cross(self.k, self.a))
        v = np.cross(db, psi) + b[..., None] * curl_psi
        return self.scale * v
