"""Failure paths of the library, in forms that fault no GPU:

* a NaN in the state makes ps_diagnostics return PS_ENUMERIC;
* a bounded wait that gives up (ps_debug_wait_timeout: an mbarrier expecting
  bulk-copy bytes that no copy delivers, nothing in flight) sets the sticky
  device error flag, ps_forces then fails with PS_ECUDA until
  ps_clear_error;
* ps_diagnostics' max |k . c_k| of a state that is not solenoidal against
  the oracle's value on the same Fourier coefficients (a projected state
  only shows round-off there).
"""
import numpy as np
import pytest
import torch

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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nan_in_state_reports_enumeric(prec):
    n, L = 24, 4.0
    dtype = torch.float64 if prec == "fp64" else torch.float32
    g = Solver(n, L, 0.01, 0.1, 1e-3, precision=prec)
    u = inputs.random_field(n, L, seed=5)
    g.set_velocity(dev(u, dtype))
    e, d = g.diagnostics()          # finite state: fine
    assert np.isfinite(e) and e > 0
    u[1, 3, 4, 5] = np.nan
    g.set_velocity(dev(u, dtype))
    with pytest.raises(B.PsError) as ex:
        g.diagnostics()
    assert ex.value.status == B.PS_ENUMERIC
    g.close()


def test_wait_timeout_sets_sticky_error_until_cleared():
    n, L = 24, 4.0
    g = Solver(n, L, 0.01, 0.1, 1e-3, precision="fp64")
    g.set_velocity(dev(inputs.random_field(n, L, seed=6), torch.float64))
    chi = np.zeros((n, n, n))
    chi[8:14, 9:15, 7:16] = 1.0
    g.set_mask(dev(chi, torch.float64), dev(np.zeros((3, n, n, n)), torch.float64))
    g.step(1)
    F0, M0 = g.forces()
    assert max(abs(v) for v in F0) > 0
    B.ps_debug_wait_timeout(g.ctx, 2000)      # the wait gives up, the flag is set
    for _ in range(2):                        # sticky
        with pytest.raises(B.PsError) as ex:
            g.forces()
        assert ex.value.status == B.PS_ECUDA
        assert "gave up" in str(ex.value)
    g.clear_error()
    F1, M1 = g.forces()
    assert F1 == F0 and M1 == M0
    with pytest.raises(B.PsError) as ex:
        B.ps_debug_wait_timeout(g.ctx, 0)
    assert ex.value.status == B.PS_EINVAL
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_max_div_of_a_non_solenoidal_state_matches_oracle(prec):
    """The state buffer holds (after a 256-byte header) U as 3 x [K (ky)][K (kx)]
    [Kzp] complex Fourier coefficients c_k = DFT_k / n^3 of the kept modes
    (index c <-> mode c if c <= mmax, else c - K). Two modes get a
    longitudinal part; the oracle evaluates its max |k . u_hat| / n^3 and its
    energy on the same coefficients."""
    n, L = 24, 4.0
    fp64 = prec == "fp64"
    dtype = torch.float64 if fp64 else torch.float32
    cdt = torch.complex128 if fp64 else torch.complex64
    g = Solver(n, L, 0.01, 0.1, 1e-3, precision=prec)
    g.set_velocity(dev(inputs.random_field(n, L, seed=8), dtype))
    buf = g.state_buffer()
    g.save_state(buf)
    mm = (n - 1) // 3
    K, Kz = 2 * mm + 1, mm + 1
    ec = 16 if fp64 else 8
    Kzp = buf[256:].numel() // (2 * 3 * K * K * ec)
    assert 2 * 3 * K * K * Kzp * ec + 256 == buf.numel() and Kzp >= Kz
    U = buf[256:256 + 3 * K * K * Kzp * ec].view(cdt).view(3, K, K, Kzp)
    # longitudinal parts: mode (mx, my, mz) = (2, -1, 3) and (-3, 0, 1)
    U[0, K - 1, 2, 3] += 0.02 + 0.01j
    U[1, K - 1, 2, 3] += -0.01
    U[0, 0, K - 3, 1] += 0.03j
    g.restore_state(buf)
    e, d = g.diagnostics()

    o = S.Solver(S.Params(n=n, L=L, nu=0.01, eta=0.1, dt=1e-3))
    c = U.cpu().numpy().astype(np.complex128)
    for cy in range(K):
        my = cy if cy <= mm else cy - K
        for cx in range(K):
            mx = cx if cx <= mm else cx - K
            o.uh[:, mx % n, my % n, :Kz] = c[:, cy, cx, :Kz] * float(n) ** 3
    d_ref = o.max_divergence()
    assert d_ref > 1e-3   # far above round-off
    assert abs(d - d_ref) < (1e-13 if fp64 else 1e-6) * d_ref, (d, d_ref)
    assert abs(e - o.energy()) < (1e-13 if fp64 else 1e-6) * o.energy()
    g.close()
