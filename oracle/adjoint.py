"""Oracle discrete adjoint of the penalized pseudo-spectral step.

Test infrastructure only (see ``oracle/__init__``). The paper has no adjoint;
this is the exact transpose of the operations of ``oracle.step`` in their
order, for the objective

    J = sum_n w_n (a . F^n + b . M^n)

(time-averaged penalization force and moment; F^n, M^n from u^n inside step
n). Inner products: physical arrays sum_j x_j y_j; half-spectrum arrays
Re sum w_kz conj(x) y with w = 1 on the kz = 0 plane and 2 elsewhere, which is
the full-spectrum sum for Hermitian data. With the oracle's transforms
(rfft3 = DFT, irfft3 = inverse DFT with 1/N, N = n n nz the grid points)
the adjoints are
    rfft3*  = N irfft3,   irfft3* = rfft3 / N,
and truncation, projection, integrating factor and i k x are self-adjoint
mode by mode.

``rasterise_vjp`` is the transpose of the mask/u_s construction of
``oracle.mask`` with the closest triangle of each point held fixed: the
distance derivative by the envelope theorem (d delta / d X_v =
-beta_v (p - q) / delta) and the barycentric weights differentiated on their
active face (vertex, edge or interior).
"""
import math

import numpy as np

from . import fft as offt
from . import mask as OM
from . import step as S


def forward(p, u0, masks, weights, a, b):
    """Run len(masks) steps from u0 with per-step (chi, us); return J, the
    per-step states u_hat^n (before step n) and forces."""
    s = S.Solver(p)
    s.set_velocity(u0)
    states, J = [], 0.0
    for n, (chi, us) in enumerate(masks):
        states.append(s.uh.copy())
        s.set_mask(chi, us)
        s.step(1)
        J += weights[n] * (np.dot(a, s.F) + np.dot(b, s.M))
    return J, states


def adjoint(p, states, masks, weights, a, b):
    """Reverse sweep. Returns per-step (dJ/dchi^n, dJ/dus^n) lists."""
    n, nz = p.n, p.nz
    n3 = float(n) * n * nz          # points of the grid: rfft3* = n3 irfft3
    keep = S.dealias_mask(n, nz)
    E = S.integrating_factor(p)
    dt = p.dt
    dx3 = (p.L / n) ** 3
    X, Y, Z = S.grid_coords(p)
    shape = (n, n, nz)
    r = [np.broadcast_to(X - p.x0[0], shape), np.broadcast_to(Y - p.x0[1], shape),
         np.broadcast_to(Z - p.x0[2], shape)]
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    # dJ/dp_j = a + b x r_j  (p = chi (u - us))
    bxr = np.stack([b[1] * r[2] - b[2] * r[1], b[2] * r[0] - b[0] * r[2], b[0] * r[1] - b[1] * r[0]])
    gp = a[:, None, None, None] + bxr

    lam = np.zeros((3, n, n, nz // 2 + 1), dtype=np.complex128)
    mu = np.zeros_like(lam)
    K = len(states)
    gchi = [None] * K
    gus = [None] * K
    for k in range(K - 1, -1, -1):
        uh = states[k]
        chi, us = masks[k]
        c = chi / p.eta
        # the update u^{k+1} = E u^k + a1 G - a2 H (k >= 1), E (u^k + dt G) (k = 0)
        a1 = (1.5 * dt * E) if k > 0 else (dt * E)
        Gbar = a1 * lam + mu
        lam_new = E * lam
        mu_new = -(0.5 * dt * E * E) * lam if k > 0 else np.zeros_like(lam)
        # G = P keep rfft3(nl)  ->  nl_bar = n^3 irfft3(keep P Gbar)
        nlb = n3 * S.to_physical(S.project(p, Gbar) * keep, nz)
        # recompute the forward quantities of step k
        u = S.to_physical(uh, nz)
        w = S.to_physical(S.curl_hat(p, uh) * keep, nz)
        # nl = u x w - c (u - us)
        ub = np.stack([w[1] * nlb[2] - w[2] * nlb[1],
                       w[2] * nlb[0] - w[0] * nlb[2],
                       w[0] * nlb[1] - w[1] * nlb[0]]) - c[None] * nlb
        wb = np.stack([nlb[1] * u[2] - nlb[2] * u[1],
                       nlb[2] * u[0] - nlb[0] * u[2],
                       nlb[0] * u[1] - nlb[1] * u[0]])
        diff = u - us
        gc = -np.sum(nlb * diff, axis=0) / p.eta
        gs = c[None] * nlb
        # the force/moment term of J
        fw = weights[k] * dx3 / p.eta
        ub = ub + fw * chi[None] * gp
        gs = gs - fw * chi[None] * gp
        gc = gc + fw * np.sum(gp * diff, axis=0)
        # u = irfft3(uh), w = irfft3(keep curl(uh))  ->  lambda += ...
        Ub = S.to_spectral(ub) / n3
        Wb = S.to_spectral(wb) / n3 * keep
        lam = lam_new + keep * (Ub + S.curl_hat(p, Wb))
        mu = mu_new
        gchi[k] = gc
        gus[k] = gs
    return gchi, gus


def _prof_deriv(delta, tw, h, profile):
    if profile == OM.PROFILE_TANH:
        t = np.tanh((delta - tw) / h)
        return -0.5 * (1.0 - t * t) / h
    ramp = (delta > tw - h) & (delta < tw + h)
    return np.where(ramp, -0.5 * math.pi / (2.0 * h) * np.sin(math.pi * (delta - tw + h) / (2.0 * h)), 0.0)


def rasterise_vjp(n, L, xw, vw, tri, frame, tw, h, chi_bar, us_bar, profile=OM.PROFILE_COS, nz=None):
    """dJ/dxw (n_nodes x 3, wing frame) given dJ/dchi, dJ/dus on the grid
    (n x n x nz, nz = n unless given), for the mask of
    ``oracle.mask.rasterise`` with its argmin held fixed."""
    chi, us, arg, best = OM.rasterise(n, L, xw, vw, tri, frame, tw, h, profile, nz=nz)
    dx = L / n
    R = np.asarray(frame["R"], dtype=np.float64).reshape(3, 3)
    xg = OM.global_nodes(xw, frame)
    vw = np.asarray(vw, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    gX = np.zeros_like(xg)
    pts = np.argwhere(arg >= 0)
    for (i, j, k) in pts:
        t = arg[i, j, k]
        P = np.array([i, j, k], dtype=np.float64) * dx
        ids = tri[t]
        A, B, C = xg[ids[0]], xg[ids[1]], xg[ids[2]]
        d, beta = OM.closest_point_on_triangle(P[None], A, B, C)
        d = d[0]
        beta = beta[0]
        q = beta[0] * A + beta[1] * B + beta[2] * C
        cb = chi_bar[i, j, k]
        # distance path
        if d > 0:
            gd = cb * _prof_deriv(d, tw, h, profile)
            for v in range(3):
                gX[ids[v]] += gd * (-beta[v] * (P - q) / d)
        # u_s path through the barycentric weights
        ub = us_bar[:, i, j, k]
        if profile == OM.PROFILE_COS and not chi[i, j, k] > 0:
            continue
        g = np.array([ub @ (R @ vw[ids[v]]) for v in range(3)])   # dJ/dbeta_v
        act = beta > 1e-12
        na = int(act.sum())
        if na == 1:
            continue
        if na == 2:
            vv = np.nonzero(act)[0]
            iu, iv = vv[0], vv[1]
            U, V = xg[ids[iu]], xg[ids[iv]]
            e = V - U
            dd = e @ e
            nn = (P - U) @ e
            gt = g[iv] - g[iu]
            dtdU = (-(e + (P - U)) * dd + 2 * nn * e) / dd ** 2
            dtdV = ((P - U) * dd - 2 * nn * e) / dd ** 2
            gX[ids[iu]] += gt * dtdU
            gX[ids[iv]] += gt * dtdV
            continue
        e0, e1, dv = B - A, C - A, P - A
        s_, t_ = beta[1], beta[2]
        M = np.array([[e0 @ e0, e0 @ e1], [e0 @ e1, e1 @ e1]])
        gam = np.array([g[1] - g[0], g[2] - g[0]])
        z = np.linalg.solve(M, gam)
        cdd = z[0] * e0 + z[1] * e1
        ce0 = z[0] * dv - (z[0] * (2 * s_ * e0 + t_ * e1) + z[1] * (s_ * e1))
        ce1 = z[1] * dv - (z[0] * (t_ * e0) + z[1] * (s_ * e0 + 2 * t_ * e1))
        gX[ids[0]] += -cdd - ce0 - ce1
        gX[ids[1]] += ce0
        gX[ids[2]] += ce1
    return gX @ R          # dJ/dxw = R^T dJ/dX, row-wise
