"""The allocation-free force entry point, ps_penalization_force_noalloc.

It serves callers that must not call cudaMalloc after start-up (a real-time
loop, where cudaMalloc can block; a process whose framework's memory pool
holds nearly all device memory, so a fresh cudaMalloc fails). Its only
scratch is a fixed array inside the library. Two calls in a row, in FP64 and
in FP32, must give the force and moment of the context's own reduction
(ps_step + ps_forces) on the same fields, and the oracle's exactly rounded
sums of the same (rounded) inputs. The file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from oracle import step as OS
from paper_2002_08642_gb300 import binding as B
from paper_2002_08642_gb300 import build as pbuild
from paper_2002_08642_gb300 import inputs
from paper_2002_08642_gb300.solver import Solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_force_matches_ps_forces_twice(precision):
    pbuild.build()
    n, L, nu, eta, dt = 32, 4.0, 1e-3, 0.05, 1e-3
    x0 = (1.9, 2.1, 2.05)
    fp64 = precision == "fp64"
    tdt = torch.float64 if fp64 else torch.float32
    ndt = np.float64 if fp64 else np.float32
    g = Solver(n, L, nu, eta, dt, precision=precision, x0=x0)
    stream = torch.cuda.current_stream().cuda_stream
    fm = torch.empty(6, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(17)
    for call in range(2):   # two calls in a row, different fields each time
        chi = np.zeros((n, n, n))
        chi[6 + call:20, 8:22, 5:25 - call] = rng.uniform(0.2, 1.0, (14 - call, 14, 20 - call))
        us = rng.standard_normal((3, n, n, n)) * 0.1
        u = inputs.random_field(n, L, seed=40 + call, rms=0.3)
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=ndt)).to("cuda", tdt)
        chi_d, us_d = d(chi), d(us)        # kept alive until the kernels ran
        g.set_velocity(d(u))
        g.set_mask(chi_d, us_d)
        u_now = g.velocity()               # the velocity ps_step reduces over
        g.step(1)
        F, M = g.forces()                  # existing entry point
        B.ps_penalization_force_noalloc(n, B.PS_FP64 if fp64 else B.PS_FP32, L, eta, x0, u_now.data_ptr(),
                                        chi_d.data_ptr(), us_d.data_ptr(), fm.data_ptr(), stream)
        got = fm.cpu().numpy()
        ref = np.concatenate([F, M])
        # the context reduces its own z-pass velocity; in FP32 that transform
        # rounds differently from the one ps_get_velocity runs
        tol = 1e-12 if fp64 else 1e-4
        assert np.allclose(got, ref, rtol=tol, atol=tol * np.abs(ref).max()), (call, got, ref)
        # oracle: exactly rounded sums of the same inputs, in double
        p = OS.Params(n=n, L=L, nu=nu, eta=eta, dt=dt, x0=x0)
        Fo, Mo = OS.penalization_force(p, u_now.cpu().double().numpy(), chi_d.cpu().double().numpy(),
                                       us_d.cpu().double().numpy())
        refo = np.concatenate([Fo, Mo])
        assert np.allclose(got, refo, rtol=1e-12, atol=1e-12 * np.abs(refo).max()), (call, got, refo)


def test_noalloc_rejects_grids_beyond_its_scratch():
    pbuild.build()
    fm = torch.empty(6, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PsError) as e:
        B.ps_penalization_force_noalloc(2048, B.PS_FP32, 4.0, 1e-3, (0, 0, 0), fm.data_ptr(), fm.data_ptr(),
                                        fm.data_ptr(), fm.data_ptr(), 0)
    assert e.value.status == B.PS_EINVAL
