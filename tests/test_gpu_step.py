"""GPU parity of the step, its transforms and diagnostics against the FP64
oracle, through the C ABI (libps.so via the ctypes binding).

Tolerances: FP64 path <= 1e-12 relative L2 per step (same state in);
FP32 path <= 2e-5 relative L2 after 100 steps; forces reported alongside.
"""
import math

import numpy as np
import pytest
import torch

from oracle import step as S
from oracle import mask as OM
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


def random_mask(n, seed):
    """Dense mask with a solid block (chi = 1), a ramp and zeros; random u_s."""
    rng = np.random.default_rng(seed)
    chi = np.zeros((n, n, n))
    a, b = n // 4, n // 2
    chi[a:b, a:b + 2, a + 1:b] = 1.0
    chi[b:b + 3] = rng.uniform(0, 1, (3, n, n))
    us = rng.standard_normal((3, n, n, n)) * 0.1
    return chi, us


def pair(n, L, nu, eta, dt, prec, x0=None, mean="fixed"):
    x0 = (0.5 * L, 0.5 * L, 0.5 * L) if x0 is None else x0
    o = S.Solver(S.Params(n=n, L=L, nu=nu, eta=eta, dt=dt, x0=x0,
                          mean_mode=S.MEAN_FREE if mean == "free" else S.MEAN_FIXED))
    g = Solver(n, L, nu, eta, dt, precision=prec, x0=x0, mean_mode=mean)
    return o, g


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 3e-6)])
@pytest.mark.parametrize("n", [12, 24, 32, 48, 64, 96])
def test_transform_roundtrip(n, prec, tol):
    """set_velocity (r2c, 2/3 truncation, projection) then get_velocity (c2r)."""
    L = 4.0
    o, g = pair(n, L, 0.01, 1.0, 1e-3, prec)
    u = inputs.random_field(n, L, seed=n) + 0.3 * np.random.default_rng(n).standard_normal((3, n, n, n))
    o.set_velocity(u)
    dt = torch.float64 if prec == "fp64" else torch.float32
    g.set_velocity(dev(u, dt))
    got = g.velocity().double().cpu().numpy()
    assert rel(got, o.velocity()) < tol


@pytest.mark.parametrize("n", [12, 24, 48, 64])
def test_fp64_step_matches_oracle(n):
    L, nu, eta, dt = 4.0, 0.02, 0.05, 2e-3
    x0 = (1.9, 2.1, 2.05)
    o, g = pair(n, L, nu, eta, dt, "fp64", x0)
    u = inputs.random_field(n, L, seed=3 * n, rms=0.5)
    chi, us = random_mask(n, n)
    o.set_velocity(u)
    o.set_mask(chi, us)
    g.set_velocity(dev(u, torch.float64))
    g.set_mask(dev(chi, torch.float64), dev(us, torch.float64))
    for k in range(4):   # Euler start, then AB2
        o.step(1)
        g.step(1)
        got = g.velocity().cpu().numpy()
        assert rel(got, o.velocity()) < 1e-12 * (k + 1), k
        F, M = g.forces()
        assert np.allclose(F, o.F, rtol=1e-12, atol=1e-12 * np.abs(o.F).max())
        assert np.allclose(M, o.M, rtol=1e-12, atol=1e-12 * np.abs(o.M).max())


def test_taylor_green_config_fp64():
    """32^3, L = 2 pi, chi = 0, nu = 0.01, dt = 1e-3, 20 steps."""
    n, L, nu, dt = 32, 2 * math.pi, 0.01, 1e-3
    o, g = pair(n, L, nu, 1.0, dt, "fp64")
    u0 = inputs.taylor_green_3d(n, L)
    o.set_velocity(u0)
    g.set_velocity(dev(u0, torch.float64))
    o.step(20)
    g.step(20)
    got = g.velocity().cpu().numpy()
    assert rel(got, o.velocity()) < 1e-12
    amp = np.sum(got * u0) / np.sum(u0 * u0)
    assert abs(amp - math.exp(-3 * nu * 20 * dt)) < 1e-4
    e, d = g.diagnostics()
    assert abs(e - o.energy()) < 1e-13 * o.energy()
    assert d < 1e-14


def test_diagnostics_match_oracle():
    n, L = 48, 4.0
    for prec, tol in (("fp64", 1e-13), ("fp32", 1e-6)):
        o, g = pair(n, L, 0.01, 1.0, 1e-3, prec)
        u = inputs.random_field(n, L, seed=9)
        o.set_velocity(u)
        g.set_velocity(dev(u, torch.float64 if prec == "fp64" else torch.float32))
        e, d = g.diagnostics()
        assert abs(e - o.energy()) < tol * o.energy()
        assert d < (1e-15 if prec == "fp64" else 1e-7) * 2 * math.pi / L * n * 0.05


def test_mean_free_mode():
    n, L = 24, 4.0
    o, g = pair(n, L, 0.01, 0.2, 1e-2, "fp64", mean="free")
    u = inputs.random_field(n, L, seed=4) + 0.1
    chi, us = random_mask(n, 5)
    o.set_velocity(u)
    o.set_mask(chi, us)
    g.set_velocity(dev(u, torch.float64))
    g.set_mask(dev(chi, torch.float64), dev(us, torch.float64))
    o.step(3)
    g.step(3)
    got = g.velocity().cpu().numpy()
    assert rel(got, o.velocity()) < 1e-12
    assert abs(got[0].mean() - o.velocity()[0].mean()) < 1e-13


def test_save_restore_is_exact():
    n, L = 32, 4.0
    g = Solver(n, L, 0.01, 0.1, 1e-3, precision="fp32")
    u = inputs.random_field(n, L, seed=8)
    g.set_velocity(dev(u, torch.float32))
    g.step(2)
    buf = g.state_buffer()
    g.save_state(buf)
    g.step(3)
    a = g.velocity().clone()
    g.restore_state(buf)
    g.step(3)
    assert torch.equal(a, g.velocity())


def plate_mask(n, L, profile):
    dx = L / n
    xw, vw, tri, fr = inputs.plate()
    prof = OM.PROFILE_TANH if profile == "tanh" else OM.PROFILE_COS
    chi, us, _, _ = OM.rasterise(n, L, xw, vw, tri, fr, 2 * dx, 1.5 * dx, prof)
    return chi, us


def test_fp32_plate_100_steps_vs_oracle():
    """Static plate configuration at 48^3 (tanh mask, eta = 1e-3,
    nu = 1/1800, dt = 5e-4, random k^-5/3 field): FP32 vs the FP64 oracle."""
    n, L, nu, eta, dt = 48, 4.0, 1.0 / 1800, 1e-3, 5e-4
    o, g = pair(n, L, nu, eta, dt, "fp32")
    u = inputs.random_field(n, L, seed=1234)
    chi, us = plate_mask(n, L, "tanh")
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
    got = g.velocity().double().cpu().numpy()
    err = rel(got, o.velocity())
    print("fp32 rel L2 after 100 steps %.3e, max force rel err %.3e" % (err, max(ferr)))
    assert err < 2e-5
    assert max(ferr) < 1e-4


def test_config_128_fp32_vs_fp64_and_oracle_step():
    """Static plate at 128^3, 100 steps: FP32 vs the FP64 GPU step (itself
    checked against the oracle for one step here)."""
    n, L, nu, eta, dt = 128, 4.0, 1.0 / 1800, 1e-3, 5e-4
    u = inputs.random_field(n, L, seed=1234)
    chi, us = plate_mask(n, L, "tanh")
    g64 = Solver(n, L, nu, eta, dt, precision="fp64")
    g32 = Solver(n, L, nu, eta, dt, precision="fp32")
    g64.set_velocity(dev(u, torch.float64))
    g64.set_mask(dev(chi, torch.float64), dev(us, torch.float64))
    g32.set_velocity(dev(u, torch.float32))
    g32.set_mask(dev(chi, torch.float32), dev(us, torch.float32))
    o = S.Solver(S.Params(n=n, L=L, nu=nu, eta=eta, dt=dt, x0=(2.0, 2.0, 2.0)))
    o.set_velocity(u)
    o.set_mask(chi, us)
    o.step(1)
    g64.step(1)
    g32.step(1)
    assert rel(g64.velocity().cpu().numpy(), o.velocity()) < 1e-12
    F, _ = g64.forces()
    assert np.allclose(F, o.F, rtol=1e-11)
    g64.step(99)
    g32.step(99)
    v64 = g64.velocity().cpu().numpy()
    err = rel(g32.velocity().double().cpu().numpy(), v64)
    F64, _ = g64.forces()
    F32, _ = g32.forces()
    print("128^3 fp32 vs fp64 after 100 steps: %.3e, force %.3e" %
          (err, np.linalg.norm(np.array(F32) - F64) / np.linalg.norm(F64)))
    assert err < 2e-5
