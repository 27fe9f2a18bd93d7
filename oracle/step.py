"""Oracle time step of the penalized pseudo-spectral Navier--Stokes solver.

Test infrastructure only (see ``oracle/__init__``).

Equation (Sec. 4.1, Eq. penalized Navier--Stokes, sponge term left out):

    d_t u + omega x u = -grad Pi + nu lap u - (chi / C_eta) (u - u_s),   div u = 0

on the periodic box [0, L)^2 x [0, Lz) with n x n x nz points x_j = j dx,
dx = L/n = Lz/nz (Lz = L, nz = n unless given: the paper's revolving-wing
box of Sec. 4.2 is 4 x 4 x 2 with N x N x N/2 points). With the total
pressure eliminated by the Leray projection P, the spectral form is

    d_t u_hat = -nu |k|^2 u_hat + P N_hat,
    N_hat     = F[ u x omega - (chi/eta)(u - u_s) ]   (omega x u moves to the
                                                       right as +u x omega)

Readings of points the paper leaves open:

* Dealiasing: the 2/3 rule on every axis -- a mode (m_x, m_y, m_z) is kept
  iff 3|m_x| < n, 3|m_y| < n and 3|m_z| < nz (integer tests). It is applied
  to the initial field, to omega_hat and to the whole N_hat (penalization
  included).
* Time scheme: the paper's "Adams--Bashforth" (Sec. 4.1, time-stepping
  paragraph) taken as fixed-step integrating-factor AB2 on v = e^{nu|k|^2 t} u_hat:
      u^{n+1} = E u^n + (dt/2) (3 E N^n - E^2 N^{n-1}),  E = exp(-nu |k|^2 dt),
  and the first step as integrating-factor Euler u^1 = E (u^0 + dt N^0).
* Mean mode k = 0: MEAN_FIXED (default) sets N_hat(0) = 0, so the mean
  velocity stays at its initial value; MEAN_FREE keeps N_hat(0).
* C_eta of the paper is ``eta`` here.
* Sponge term (optional, off unless ``set_sponge``): the paper writes it as
  -(1/C_sp) curl (chi_sp omega) / lap and calls it a vorticity damping term;
  read literally that sign amplifies (for chi_sp = 1 it is +u/C_sp), so the
  damping reading is taken: -(1/C_sp) curl^{-1}(chi_sp omega), spectrally
      S_hat = -(1/C_sp) i k x s_hat / |k|^2,  s_hat = F[chi_sp omega] (2/3 rule),
  which is -u/C_sp for chi_sp = 1 (solenoidal, so the projection keeps it).
* Force on the solid from the penalization term, fluid density 1:
      F = (dx^3 / eta) sum_j chi_j (u_j - u_s,j)
      M = (dx^3 / eta) sum_j (x_j - x0) x chi_j (u_j - u_s,j)
  evaluated from u^n inside step n (Sec. 4.2.2 defines lift as the z
  component of the aerodynamic force).
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import fft as offt

MEAN_FIXED = 0
MEAN_FREE = 1


@dataclass
class Params:
    n: int
    L: float
    nu: float
    eta: float
    dt: float
    x0: tuple = (0.0, 0.0, 0.0)
    mean_mode: int = MEAN_FIXED
    nz: int = 0        # points along z (0: n)
    Lz: float = 0.0    # box length along z (0: L nz / n, the same spacing)

    def __post_init__(self):
        if self.nz == 0:
            self.nz = self.n
        if self.Lz == 0.0:
            self.Lz = self.L * self.nz / self.n
        if abs(self.Lz / self.nz - self.L / self.n) > 1e-12 * self.L / self.n:
            raise ValueError("the grid spacing must be the same on all axes")


def mode_numbers(n):
    """Signed mode numbers m of the FFT index order: 0..n/2-1, -n/2..-1."""
    q = np.arange(n)
    return np.where(q < n // 2, q, q - n)


def wavevectors(p):
    """(kx, ky, kz) broadcastable over the half spectrum [kx][ky][kz<=nz/2]."""
    n = p.n
    s = 2.0 * math.pi / p.L
    mx = mode_numbers(n)
    mz = np.arange(p.nz // 2 + 1)
    kx = (s * mx)[:, None, None]
    ky = (s * mx)[None, :, None]
    kz = (2.0 * math.pi / p.Lz * mz)[None, None, :]
    return kx, ky, kz


def dealias_mask(n, nz=None):
    """Boolean keep-mask of the 2/3 rule on the half spectrum (nz z points,
    default n)."""
    nz = n if nz is None else nz
    mx = np.abs(mode_numbers(n))
    mz = np.arange(nz // 2 + 1)
    kx = 3 * mx < n
    kz = 3 * mz < nz
    return kx[:, None, None] & kx[None, :, None] & kz[None, None, :]


def curl_hat(p, uh):
    """omega_hat = i k x u_hat (component-wise cross product)."""
    kx, ky, kz = wavevectors(p)
    ux, uy, uz = uh
    return np.stack([1j * (ky * uz - kz * uy),
                     1j * (kz * ux - kx * uz),
                     1j * (kx * uy - ky * ux)])


def project(p, Nh):
    """Leray projection N - k (k.N)/|k|^2; the k = 0 mode per ``mean_mode``."""
    kx, ky, kz = wavevectors(p)
    k2 = kx * kx + ky * ky + kz * kz
    k2_safe = np.where(k2 == 0.0, 1.0, k2)
    kdotN = kx * Nh[0] + ky * Nh[1] + kz * Nh[2]
    out = np.stack([Nh[0] - kx * kdotN / k2_safe,
                    Nh[1] - ky * kdotN / k2_safe,
                    Nh[2] - kz * kdotN / k2_safe])
    if p.mean_mode == MEAN_FIXED:
        out[:, 0, 0, 0] = 0.0
    else:
        out[:, 0, 0, 0] = Nh[:, 0, 0, 0]
    return out


def sponge_hat(p, sh, c_sp):
    """-(1/C_sp) i k x s_hat / |k|^2 (zero at k = 0)."""
    kx, ky, kz = wavevectors(p)
    k2 = kx * kx + ky * ky + kz * kz
    k2_safe = np.where(k2 == 0.0, 1.0, k2)
    sx, sy, sz = sh
    out = np.stack([1j * (ky * sz - kz * sy), 1j * (kz * sx - kx * sz), 1j * (kx * sy - ky * sx)])
    out = -out / (c_sp * k2_safe)
    out[:, 0, 0, 0] = 0.0
    return out


def integrating_factor(p):
    """E = exp(-nu |k|^2 dt) on the half spectrum."""
    kx, ky, kz = wavevectors(p)
    return np.exp(-p.nu * (kx * kx + ky * ky + kz * kz) * p.dt)


def grid_coords(p):
    """Physical coordinates x_j = j dx of the three axes, broadcastable."""
    x = np.arange(p.n) * (p.L / p.n)
    z = np.arange(p.nz) * (p.Lz / p.nz)
    return x[:, None, None], x[None, :, None], z[None, None, :]


def to_spectral(u):
    """Forward transform of the three components of a real field."""
    return np.stack([offt.rfft3(c) for c in u])


def to_physical(uh, nz):
    """Inverse transform of the three components of a half spectrum (nz
    points along z)."""
    return np.stack([offt.irfft3(c, nz) for c in uh])


def nonlinear_physical(u, w, chi, us, eta):
    """n = u x omega - (chi/eta)(u - u_s), pointwise."""
    cross = np.stack([u[1] * w[2] - u[2] * w[1],
                      u[2] * w[0] - u[0] * w[2],
                      u[0] * w[1] - u[1] * w[0]])
    return cross - (chi / eta)[None] * (u - us)


def penalization_force(p, u, chi, us):
    """Force and moment of the penalization term, exactly rounded sums."""
    dx3 = (p.L / p.n) ** 3
    pen = chi[None] * (u - us)
    X, Y, Z = grid_coords(p)
    shape = (p.n, p.n, p.nz)
    rx = np.broadcast_to(X - p.x0[0], shape)
    ry = np.broadcast_to(Y - p.x0[1], shape)
    rz = np.broadcast_to(Z - p.x0[2], shape)
    mom = [ry * pen[2] - rz * pen[1],
           rz * pen[0] - rx * pen[2],
           rx * pen[1] - ry * pen[0]]
    F = np.array([math.fsum(pen[c].ravel()) for c in range(3)]) * dx3 / p.eta
    M = np.array([math.fsum(np.asarray(mom[c]).ravel()) for c in range(3)]) * dx3 / p.eta
    return F, M


class Solver:
    """State (u_hat^n, N_hat^{n-1}, step count) and the step of the module doc."""

    def __init__(self, p):
        self.p = p
        n, nz = p.n, p.nz
        self.keep = dealias_mask(n, nz)
        self.E = integrating_factor(p)
        self.uh = np.zeros((3, n, n, nz // 2 + 1), dtype=np.complex128)
        self.Nprev = np.zeros_like(self.uh)
        self.nstep = 0
        self.chi = np.zeros((n, n, nz))
        self.us = np.zeros((3, n, n, nz))
        self.F = np.zeros(3)
        self.M = np.zeros(3)
        self.chi_sp = None
        self.c_sp = 0.0

    def set_velocity(self, u):
        """Transform, truncate and project u; the mean is kept; AB2 restarts."""
        uh = to_spectral(np.asarray(u, dtype=np.float64)) * self.keep
        kx, ky, kz = wavevectors(self.p)
        k2 = kx * kx + ky * ky + kz * kz
        k2_safe = np.where(k2 == 0.0, 1.0, k2)
        kdotu = kx * uh[0] + ky * uh[1] + kz * uh[2]
        mean = uh[:, 0, 0, 0].copy()
        uh = np.stack([uh[0] - kx * kdotu / k2_safe,
                       uh[1] - ky * kdotu / k2_safe,
                       uh[2] - kz * kdotu / k2_safe])
        uh[:, 0, 0, 0] = mean
        self.uh = uh
        self.Nprev = np.zeros_like(uh)
        self.nstep = 0

    def set_mask(self, chi, us):
        self.chi = np.asarray(chi, dtype=np.float64)
        self.us = np.asarray(us, dtype=np.float64)

    def set_sponge(self, chi_sp, c_sp):
        """Sponge mask (n^3) and constant C_sp; chi_sp None turns it off."""
        self.chi_sp = None if chi_sp is None else np.asarray(chi_sp, dtype=np.float64)
        self.c_sp = float(c_sp)

    def velocity(self):
        return to_physical(self.uh, self.p.nz)

    def rhs_hat(self):
        """Projected, truncated N_hat of the current state; sets F, M."""
        p = self.p
        wh = curl_hat(p, self.uh) * self.keep
        u = to_physical(self.uh, p.nz)
        w = to_physical(wh, p.nz)
        self.F, self.M = penalization_force(p, u, self.chi, self.us)
        nl = nonlinear_physical(u, w, self.chi, self.us, p.eta)
        Nh = to_spectral(nl) * self.keep
        if self.chi_sp is not None:
            Nh = Nh + sponge_hat(p, to_spectral(self.chi_sp[None] * w) * self.keep, self.c_sp)
        return project(p, Nh)

    def step(self, nsteps=1):
        for _ in range(nsteps):
            Nh = self.rhs_hat()
            E = self.E
            dt = self.p.dt
            if self.nstep == 0:
                new = E * (self.uh + dt * Nh)
            else:
                new = E * self.uh + 0.5 * dt * (3.0 * E * Nh - E * E * self.Nprev)
            self.uh = new
            self.Nprev = Nh
            self.nstep += 1

    def energy(self):
        """(1/2) integral |u|^2 dV via Parseval on the half spectrum."""
        n, nz = self.p.n, self.p.nz
        w = np.full(nz // 2 + 1, 2.0)
        w[0] = 1.0
        if nz % 2 == 0:
            w[nz // 2] = 1.0
        s = np.sum(np.abs(self.uh) ** 2 * w[None, None, None, :])
        return 0.5 * s * self.p.L ** 2 * self.p.Lz / (float(n) ** 2 * nz) ** 2

    def max_divergence(self):
        """max |k . c_k| over the half spectrum, c_k = DFT(u)_k / n^3 the
        Fourier coefficients (so the value does not scale with n)."""
        kx, ky, kz = wavevectors(self.p)
        d = kx * self.uh[0] + ky * self.uh[1] + kz * self.uh[2]
        return float(np.max(np.abs(d))) / (float(self.p.n) ** 2 * self.p.nz)
