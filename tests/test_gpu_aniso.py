"""The paper's revolving-wing box (Sec. 4.2: 4 x 4 x 2 with N x N x N/2
points, the same spacing on every axis) on the GPU, through the C ABI,
against the anisotropic oracle (z wavenumbers 2 pi m/Lz, the 2/3 rule with
nz along z, volume L^2 Lz) and, at the bench sizes, against closed forms at
sampled points."""
import math

import numpy as np
import pytest
import torch

from oracle import adjoint as OA
from oracle import mask as OM
from oracle import pressure as OP
from oracle import step as S
from paper_2002_08642_gb300 import binding as B
from paper_2002_08642_gb300 import build as pbuild
from paper_2002_08642_gb300 import inputs
from paper_2002_08642_gb300.solver import Solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def random_mask(n, nz, seed):
    """Dense mask: a solid block (chi = 1), a ramp of random values, zeros
    elsewhere; random u_s."""
    rng = np.random.default_rng(seed)
    chi = np.zeros((n, n, nz))
    a, b = n // 4, n // 2
    chi[a:b, a:b + 2, nz // 4:nz // 2 + 1] = 1.0
    chi[b:b + 3] = rng.uniform(0, 1, (3, n, nz))
    us = rng.standard_normal((3, n, n, nz)) * 0.1
    return chi, us


def pair(n, nz, L, nu, eta, dt, prec, x0=None):
    Lz = L * nz / n
    x0 = (0.5 * L, 0.5 * L, 0.5 * Lz) if x0 is None else x0
    o = S.Solver(S.Params(n=n, L=L, nu=nu, eta=eta, dt=dt, x0=x0, nz=nz))
    g = Solver(n, L, nu, eta, dt, precision=prec, x0=x0, nz=nz)
    return o, g


def test_supported_grids():
    for n, nz, ok in ((32, 16, True), (768, 384, True), (48, 24, True), (24, 12, False), (32, 8, False),
                      (32, 32, True)):
        p = B.PsParams()
        p.n, p.nz, p.precision, p.L, p.nu, p.eta, p.dt, p.tw, p.h = n, nz, B.PS_FP32, 4.0, 1e-3, 1e-3, 1e-3, 0.1, 0.1
        if ok:
            assert B.ps_workspace_size(p) > 0
        else:
            with pytest.raises(B.PsError) as e:
                B.ps_workspace_size(p)
            assert e.value.status == B.PS_EUNSUPPORTED


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 3e-6)])
@pytest.mark.parametrize("n", [32, 48])
def test_aniso_transform_roundtrip(n, prec, tol):
    nz, L = n // 2, 4.0
    o, g = pair(n, nz, L, 0.01, 1.0, 1e-3, prec)
    u = inputs.random_field(n, L, seed=n, nz=nz) + 0.3 * np.random.default_rng(n).standard_normal((3, n, n, nz))
    o.set_velocity(u)
    g.set_velocity(dev(u, torch.float64 if prec == "fp64" else torch.float32))
    assert rel(g.velocity().double().cpu().numpy(), o.velocity()) < tol
    e, d = g.diagnostics()
    assert abs(e - o.energy()) < (1e-13 if prec == "fp64" else 1e-6) * o.energy()


@pytest.mark.parametrize("n", [32, 48])
def test_aniso_fp64_step_matches_oracle(n):
    nz, L, nu, eta, dt = n // 2, 4.0, 0.02, 0.05, 2e-3
    x0 = (1.9, 2.1, 1.05)
    o, g = pair(n, nz, L, nu, eta, dt, "fp64", x0)
    u = inputs.random_field(n, L, seed=3 * n, rms=0.5, nz=nz)
    chi, us = random_mask(n, nz, n)
    o.set_velocity(u)
    o.set_mask(chi, us)
    g.set_velocity(dev(u, torch.float64))
    g.set_mask(dev(chi, torch.float64), dev(us, torch.float64))
    for k in range(4):   # Euler start, then AB2
        o.step(1)
        g.step(1)
        assert rel(g.velocity().cpu().numpy(), o.velocity()) < 1e-12 * (k + 1), k
        F, M = g.forces()
        assert np.allclose(F, o.F, rtol=1e-12, atol=1e-12 * np.abs(o.F).max())
        assert np.allclose(M, o.M, rtol=1e-12, atol=1e-12 * np.abs(o.M).max())
    e, d = g.diagnostics()
    assert abs(e - o.energy()) < 1e-13 * o.energy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_aniso_rasterised_wing_and_steps(prec):
    """The revolving wing about (2, 2, 1) in the 4 x 4 x 2 box: the GPU mask
    against the oracle rasteriser on the n x n x n/2 grid, then two steps."""
    n, nz, L, nu, eta, dt = 32, 16, 4.0, 1.527e-4, 1e-2, 5e-4
    dx = L / n
    dtype = torch.float64 if prec == "fp64" else torch.float32
    xw0, tri = inputs.elliptic_wing_mesh(300)
    xw, vw, fr = inputs.revolving_wing(0.3, xw0, inputs.flapping_amplitudes(xw0), centre=(2.0, 2.0, 1.0))
    chi_o, us_o, _, _ = OM.rasterise(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx, nz=nz)
    assert (chi_o > 0).sum() > 100
    o, g = pair(n, nz, L, nu, eta, dt, prec, x0=(2.0, 2.0, 1.0))
    g.set_mask_from_nodes(dev(xw, torch.float64), dev(vw, torch.float64), dev(tri, torch.int32), fr)
    chi, us = g.mask()
    chi, us = chi.double().cpu().numpy(), us.double().cpu().numpy()
    assert np.abs(chi - chi_o).max() < (1e-12 if prec == "fp64" else 2e-6)
    band = chi_o > 0.01
    du = np.abs(us - us_o).max(axis=0)[band]
    # u_s wherever the closest triangle is the same (all but near-ties)
    assert np.mean(du < (1e-12 if prec == "fp64" else 1e-6)) > 0.97
    u = inputs.random_field(n, L, seed=5, rms=0.3, nz=nz)
    o.set_velocity(u)
    o.set_mask(chi_o, us_o)
    g.set_velocity(dev(u, dtype))
    g.set_mask(dev(chi_o, dtype), dev(us_o, dtype))   # the oracle's mask: the step alone
    o.step(2)
    g.step(2)
    assert rel(g.velocity().double().cpu().numpy(), o.velocity()) < (2e-12 if prec == "fp64" else 2e-6)
    F, M = g.forces()
    assert np.allclose(F, o.F, rtol=1e-11 if prec == "fp64" else 1e-4, atol=1e-6 * np.abs(o.F).max())


def test_aniso_fp32_100_steps_vs_oracle():
    """The static plate, tanh mask, eta = 1e-3, nu = 1/1800, dt = 5e-4, on
    the 48 x 48 x 24 grid of the 4 x 4 x 2 box: FP32 after 100 steps."""
    n, nz, L, nu, eta, dt = 48, 24, 4.0, 1.0 / 1800, 1e-3, 5e-4
    dx = L / n
    xw, vw, tri, fr = inputs.plate(centre=(2.0, 2.0, 1.0))
    chi, us, _, _ = OM.rasterise(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx, OM.PROFILE_TANH, nz=nz)
    o, g = pair(n, nz, L, nu, eta, dt, "fp32")
    u = inputs.random_field(n, L, seed=1234, nz=nz)
    o.set_velocity(u)
    o.set_mask(chi, us)
    g.set_velocity(dev(u, torch.float32))
    g.set_mask(dev(chi, torch.float32), dev(us, torch.float32))
    ferr = []
    for _ in range(100):
        o.step(1)
        g.step(1)
        F, _ = g.forces()
        ferr.append(np.linalg.norm(np.array(F) - o.F) / np.linalg.norm(o.F))
    err = rel(g.velocity().double().cpu().numpy(), o.velocity())
    print("aniso fp32 rel L2 after 100 steps %.3e, max force rel err %.3e" % (err, max(ferr)))
    assert err < 2e-5
    assert max(ferr) < 1e-4


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_aniso_pressure_matches_oracle(prec, tol):
    n, nz, L, nu, eta, dt = 32, 16, 4.0, 1.527e-4, 1e-2, 5e-4
    dx = L / n
    dtype = torch.float64 if prec == "fp64" else torch.float32
    xw0, tri = inputs.elliptic_wing_mesh(300)
    xw, vw, fr = inputs.revolving_wing(0.3, xw0, inputs.flapping_amplitudes(xw0), centre=(2.0, 2.0, 1.0))
    chi, us, _, _ = OM.rasterise(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx, nz=nz)
    u = inputs.random_field(n, L, seed=7, rms=0.3, nz=nz)
    o, g = pair(n, nz, L, nu, eta, dt, prec, x0=(2.0, 2.0, 1.0))
    o.set_velocity(u)
    o.set_mask(chi, us)
    o.step(2)
    g.set_velocity(dev(u, dtype))
    g.set_mask(dev(chi, dtype), dev(us, dtype))
    g.step(2)
    got = g.pressure().double().cpu().numpy()
    want = OP.static_pressure(o.p, o.uh, chi, us)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < tol
    # node pressures and loads against the oracle's interpolation of the same field
    pn, fn = g.pressure_loads(g.pressure(), dev(xw, torch.float64), dev(tri, torch.int32), fr)
    xg = OM.global_nodes(xw, fr)
    pn_o = OP.interpolate(got, L, xg)
    assert np.abs(pn.cpu().numpy() - pn_o).max() < 1e-12 * np.abs(pn_o).max()
    fn_o = OP.node_loads(pn_o, xg, tri)
    assert np.abs(fn.cpu().numpy() - fn_o).max() < 1e-12 * np.abs(fn_o).max()


def test_aniso_adjoint_matches_oracle():
    n, nz, K = 32, 16, 3
    L = 4.0
    p = S.Params(n=n, L=L, nu=0.02, eta=0.05, dt=2e-3, x0=(1.9, 2.1, 1.05), nz=nz)
    rng = np.random.default_rng(2)
    u0 = inputs.random_field(n, L, seed=9, rms=0.5, nz=nz)
    masks = []
    for _ in range(K):
        chi = np.zeros((n, n, nz))
        chi[8:18, 9:19, 4:11] = rng.uniform(0.2, 1.0, (10, 10, 7))
        masks.append((chi, rng.standard_normal((3, n, n, nz)) * 0.1))
    w = np.full(K, 1.0 / K)
    a = np.array([0.3, -0.2, 1.0])
    b = np.array([0.1, 0.4, -0.3])
    J, states = OA.forward(p, u0, masks, w, a, b)
    gchi_o, gus_o = OA.adjoint(p, states, masks, w, a, b)
    g = Solver(n, L, p.nu, p.eta, p.dt, precision="fp64", x0=p.x0, with_adjoint=True, nz=nz)
    g.set_velocity(dev(u0, torch.float64))
    md = [(dev(c, torch.float64), dev(s, torch.float64)) for c, s in masks]
    bufs, Jg = [], 0.0
    for k in range(K):
        buf = g.state_buffer()
        g.save_state(buf)
        bufs.append(buf)
        g.set_mask(*md[k])
        g.step(1)
        F, M = g.forces()
        Jg += w[k] * (np.dot(a, F) + np.dot(b, M))
    assert abs(Jg - J) < 1e-12 * abs(J)
    gchi = torch.empty((n, n, nz), dtype=torch.float64, device="cuda")
    gus = torch.empty((3, n, n, nz), dtype=torch.float64, device="cuda")
    g.adjoint_reset()
    for k in range(K - 1, -1, -1):
        g.restore_state(bufs[k])
        g.set_mask(*md[k])
        g.adjoint_step(w[k] * a, w[k] * b, k == 0, gchi, gus)
        assert rel(gchi.cpu().numpy(), gchi_o[k]) < 1e-10, k
        assert rel(gus.cpu().numpy(), gus_o[k]) < 1e-10, k


# ------------------------------------------------------------ bench sizes
NSAMPLE = 8192


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("n", [128, 256, 768])
def test_aniso_first_step_closed_form(n, prec):
    """u0 = (sin y, sin 2z, sin x) on [0, 2 pi)^2 x [0, pi) (k_z = 2 m):
    omega = -(2 cos 2z, cos x, cos y) and P[u x omega] = -(sin 2z cos y,
    2 sin x cos 2z, sin y cos x); with chi = c, u_s = beta u0 one
    integrating-factor Euler step gives, per component, e^{-nu |k|^2 dt}
    (1 - dt (c/eta)(1 - beta)) u0 + dt e^{-nu |k'|^2 dt} P[u x omega] with
    |k|^2 = 1, 4, 1 and |k'|^2 = 5, 5, 2."""
    nz, L, nu, dt, eta, c, beta = n // 2, 2 * math.pi, 0.05, 0.01, 0.1, 0.4, 0.3
    dtype = torch.float64 if prec == "fp64" else torch.float32
    x = torch.arange(n, dtype=torch.float64, device="cuda") * (L / n)
    z = torch.arange(nz, dtype=torch.float64, device="cuda") * (L / n)
    u0 = torch.empty((3, n, n, nz), dtype=dtype, device="cuda")
    u0[0] = torch.sin(x)[None, :, None].expand(n, n, nz)
    u0[1] = torch.sin(2 * z)[None, None, :].expand(n, n, nz)
    u0[2] = torch.sin(x)[:, None, None].expand(n, n, nz)
    g = Solver(n, L, nu, eta, dt, precision=prec, nz=nz)
    g.set_velocity(u0)
    g.set_mask(torch.full((n, n, nz), c, dtype=dtype, device="cuda"), u0 * beta)
    del u0
    g.step(1)
    F, _ = g.forces()
    u1 = g.velocity()
    gen = torch.Generator(device="cpu").manual_seed(n)
    ix, iy = [torch.randint(0, n, (NSAMPLE,), generator=gen) for _ in range(2)]
    iz = torch.randint(0, nz, (NSAMPLE,), generator=gen)
    got = torch.stack([u1[k, ix.cuda(), iy.cuda(), iz.cuda()] for k in range(3)]).double().cpu().numpy()
    del u1
    g.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    X, Y, Z = [t.numpy() * (L / n) for t in (ix, iy, iz)]
    lam = dt * (c / eta) * (1 - beta)
    E = lambda k2: math.exp(-nu * k2 * dt)
    ref = np.stack([E(1) * (1 - lam) * np.sin(Y) - dt * E(5) * np.sin(2 * Z) * np.cos(Y),
                    E(4) * (1 - lam) * np.sin(2 * Z) - dt * E(5) * 2 * np.sin(X) * np.cos(2 * Z),
                    E(1) * (1 - lam) * np.sin(X) - dt * E(2) * np.sin(Y) * np.cos(X)])
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < (1e-13 if prec == "fp64" else 2e-6), err
    dx = L / n
    assert np.abs(np.array(F)).max() < (1e-11 if prec == "fp64" else 1e-5) * dx ** 3 / eta * c * n * n * nz
