"""Host mass-spring network through the C ABI (ps_ms_* of libps, Sec.
2.1-2.4) against the oracle and the paper's printed values. No GPU: the
network is host code."""
import math
import os

import numpy as np
import pytest

from oracle import massspring as OM
from paper_2002_08642_gb300 import binding as B
from paper_2002_08642_gb300 import build as pbuild
from paper_2002_08642_gb300.massspring import MassSpring, cantilever

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cantilever_large_deflection.txt")


@pytest.fixture(scope="module", autouse=True)
def _built():
    pbuild.build()


def random_network(seed=5, n=9):
    """Two bent veins of 3-D points joined by extension springs, first two
    nodes fixed (bending springs need a nonzero x extent)."""
    rng = np.random.default_rng(seed)
    x0 = np.zeros((n, 3))
    x0[:, 0] = np.arange(n) * 0.1
    x0[:, 1:] = 0.03 * rng.normal(size=(n, 2))
    x0[n // 2:, 1] += 0.15
    ext = [(i, i + 1) for i in range(n - 1)] + [(i, i + n // 2) for i in range(n - n // 2)]
    bend = [(i, i + 1, i + 2) for i in range(n - 2)]
    ke = rng.uniform(50.0, 200.0, len(ext))
    kb = rng.uniform(0.05, 0.2, len(bend))
    mass = rng.uniform(0.5, 1.5, n)
    fixed = np.zeros(n, bool)
    fixed[:2] = True
    return x0, mass, fixed, ext, ke, bend, kb


def test_forces_match_oracle():
    x0, mass, fixed, ext, ke, bend, kb = random_network()
    net = OM.Network(x0, mass, fixed, ext, ke, bend, kb)
    ms = MassSpring(x0, mass, ext, ke, bend, kb, fixed=fixed)
    rng = np.random.default_rng(8)
    for _ in range(3):
        x = x0 + 0.02 * rng.normal(size=x0.shape)
        want = net.forces(x)
        got = ms.forces(x)
        assert np.max(np.abs(got - want)) < 1e-7 * np.max(np.abs(want))
    assert np.max(np.abs(ms.forces(x0))) < 1e-12


def test_bdf2_trajectory_matches_oracle_in_moving_frame():
    """Five variable steps under a tip load in a spinning, accelerating
    frame: positions and velocities agree with the oracle's BDF2."""
    x0, mass, fixed, ext, ke, bend, kb = random_network(seed=11)
    net = OM.Network(x0, mass, fixed, ext, ke, bend, kb)
    ms = MassSpring(x0, mass, ext, ke, bend, kb, fixed=fixed)
    fe = np.zeros_like(x0)
    fe[-1] = (0.0, -0.5, 0.8)
    x, v = x0.copy(), np.zeros_like(x0)
    xm1 = vm1 = None
    dts = [2e-2, 3e-2, 2e-2, 1.5e-2, 2.5e-2]
    t, dprev = 0.0, None
    for dt in dts:
        t += dt
        fr = dict(A_O=(0.1, 0.0, -0.2), Omega=(0.3 * t, -0.1, 1.0), dOmega=(0.3, 0.0, 0.0))
        xn, vn, _ = OM.bdf2_step(net, x, v, xm1, vm1, dt, dprev, fe, tol=1e-12, frame=fr)
        xm1, vm1, x, v, dprev = x, v, xn, vn, dt
        it = ms.step(dt, fe, frame=fr, tol=1e-12)
        assert 1 <= it <= 10
    gx, gv = ms.state()
    assert np.max(np.abs(gx - x)) < 1e-8 * np.max(np.abs(x))
    assert np.max(np.abs(gv - v)) < 1e-6 * np.max(np.abs(v))
    assert np.all(gx[:2] == x0[:2]) and np.all(gv[:2] == 0)


def test_equilibrium_matches_oracle():
    npts = 12
    net = OM.cantilever(0.3, 0.24, npts, ke=1e7)
    fe = np.zeros((npts, 3))
    fe[-1, 1] = -7.84
    want = OM.equilibrium(net, fe, steps=8, tol=1e-12)
    ms = cantilever(0.3, 0.24, npts, 1e7)
    ms.equilibrium(fe, load_steps=8, tol=1e-12)
    got, v = ms.state()
    assert np.max(np.abs(got - want)) < 1e-8
    assert np.all(v == 0)


def test_large_deflection_table_at_64_points():
    """Sec. 2.4.1, Table 1 with the paper's 64 mass points: the tip agrees
    with the paper's own mass-spring column to 0.3 % plus half a printed
    unit, and with the continuum beam to the paper's 1 %."""
    for F, xr, yr, xm, ym in np.loadtxt(GOLDEN):
        ms = cantilever(0.3, 0.24, 64, 1e7)
        fe = np.zeros((64, 3))
        fe[-1, 1] = -F
        ms.equilibrium(fe, load_steps=8)
        x, _ = ms.state()
        dx, dy = x[-1, 0] * 100, x[-1, 1] * 100
        assert abs(dx - xm) <= 3e-3 * abs(xm) + 5e-3, (F, dx, xm)
        assert abs(dy - ym) <= 3e-3 * abs(ym) + 5e-3, (F, dy, ym)
        assert abs(dx - xr) < 1e-2 * abs(xr) and abs(dy - yr) < 1e-2 * abs(yr), (F, dx, dy)


def test_moving_frame_closed_form_and_order():
    """Free particles in a spinning, accelerating frame (no springs) follow
    R^T (X0 + V0 t - X_O) to second order."""
    x0 = np.array([[0.4, 0.1, -0.2], [-0.3, 0.5, 0.25]])
    v_in = np.array([[0.2, -0.1, 0.3], [0.0, 0.4, -0.2]])
    acc, tau = np.array([0.3, -0.2, 0.1]), 0.5

    def frame(t):
        phi = tau * math.exp(-t / tau) + t - tau
        c, s = math.cos(phi), math.sin(phi)
        R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
        fr = dict(A_O=R.T @ acc, Omega=(0.0, 0.0, 1.0 - math.exp(-t / tau)),
                  dOmega=(0.0, 0.0, math.exp(-t / tau) / tau))
        return R, 0.5 * acc * t * t, fr

    errs = []
    for m in (50, 100, 200):
        ms = MassSpring(x0, [1.0, 2.5], np.zeros((0, 2), int), [], v0=v_in)
        for k in range(m):
            ms.step(1.0 / m, frame=frame((k + 1) / m)[2], tol=1e-13)
        x, _ = ms.state()
        R, XO, _ = frame(1.0)
        errs.append(np.max(np.abs(x - (x0 + v_in - XO[None]) @ R)))
    assert errs[2] < 1e-4 and 3.6 < errs[0] / errs[1] < 4.4 and 3.8 < errs[1] / errs[2] < 4.2, errs


def test_banded_order_keeps_bandwidth_small():
    """A 20 x 12 membrane grid: the reverse Cuthill--McKee order gives a
    node bandwidth near the short side, not the node count."""
    nx, ny = 20, 12
    x0 = np.array([(i * 0.05, j * 0.05, 0.0) for i in range(nx) for j in range(ny)])
    ext = []
    for i in range(nx):
        for j in range(ny):
            a = i * ny + j
            if j + 1 < ny:
                ext.append((a, a + 1))
            if i + 1 < nx:
                ext.append((a, a + ny))
            if i + 1 < nx and j + 1 < ny:
                ext.append((a, a + ny + 1))
    fixed = np.zeros(nx * ny, bool)
    fixed[:ny] = True
    ms = MassSpring(x0, 1.0, ext, 100.0, fixed=fixed)
    nf, bw, _ = ms.info()
    assert nf == (nx - 1) * ny and bw <= ny + 2
    # a pull on the far edge: a BDF2 step converges in a few Newton iterations
    fe = np.zeros_like(x0)
    fe[-ny:, 2] = 0.1
    assert ms.step(1e-2, fe, tol=1e-6) <= 4


def test_rejects_bad_arguments():
    x0 = np.zeros((3, 3))
    x0[:, 0] = (0.0, 1.0, 2.0)
    with pytest.raises(B.PsError) as e:
        MassSpring(x0, 1.0, [(0, 3)], 1.0)
    assert e.value.status == B.PS_EINVAL
    with pytest.raises(B.PsError):
        MassSpring(x0, [1.0, 0.0, 1.0], [(0, 1)], 1.0)
    with pytest.raises(B.PsError):
        MassSpring(x0, 1.0, [(0, 1)], 1.0, bend=[(0, 1, 1)], kb=1.0)
    ms = MassSpring(x0, 1.0, [(0, 1), (1, 2)], 1.0)
    with pytest.raises(B.PsError):
        ms.step(-1.0)


# --------------------------------------------------------- membrane model
def _tri_sheet(m):
    """Regular triangular lattice on about [0, 1]^2: rows along x with
    spacing a = 1/m, row pitch a sqrt(3)/2, odd rows shifted by a/2; springs
    between nearest neighbours. Returns nodes, springs, left/right edge
    nodes per row and the weight (row pitch share) of each row."""
    a = 1.0 / m
    h = a * math.sqrt(3) / 2
    nrow = int(round(1.0 / h)) + 1
    pts, idx = [], {}
    for r in range(nrow):
        for c in range(m + 1 if r % 2 == 0 else m):
            idx[(r, c)] = len(pts)
            pts.append(((0.5 * a if r % 2 else 0.0) + c * a, r * h, 0.0))
    ext = []
    for (r, c), i in idx.items():
        nb = [(r, c + 1)] + ([(r + 1, c - 1), (r + 1, c)] if r % 2 == 0 else [(r + 1, c), (r + 1, c + 1)])
        ext += [(i, idx[q]) for q in nb if q in idx]
    left = [idx[(r, 0)] for r in range(nrow)]
    right = [idx[(r, m if r % 2 == 0 else m - 1)] for r in range(nrow)]
    w = [h * (0.5 if r in (0, nrow - 1) else 1.0) for r in range(nrow)]
    return np.array(pts), ext, left, right, w


def _cross_center_sheet(m):
    """Unit square of m x m cells: cell edges plus a centre node joined to
    the four corners."""
    a = 1.0 / m
    pts = [(i * a, j * a, 0.0) for j in range(m + 1) for i in range(m + 1)]
    ext = []
    for j in range(m + 1):
        for i in range(m + 1):
            if i < m:
                ext.append((j * (m + 1) + i, j * (m + 1) + i + 1))
            if j < m:
                ext.append((j * (m + 1) + i, (j + 1) * (m + 1) + i))
    for j in range(m):
        for i in range(m):
            c = len(pts)
            pts.append(((i + 0.5) * a, (j + 0.5) * a, 0.0))
            ext += [(c, jj * (m + 1) + ii) for ii, jj in ((i, j), (i + 1, j), (i, j + 1), (i + 1, j + 1))]
    left = [j * (m + 1) for j in range(m + 1)]
    right = [j * (m + 1) + m for j in range(m + 1)]
    w = [a * (0.5 if j in (0, m) else 1.0) for j in range(m + 1)]
    return np.array(pts), ext, left, right, w


def _k_over_Es(sheet, T=0.005):
    """Sec. 2.4.2: uniaxial tension T per unit length on the left and right
    edges of a sheet of unit springs (k = 1), E_s = T / strain; the static
    state is reached by large damped BDF2 steps (no node is fixed: the
    loads balance), as the paper reaches it by damped dynamics."""
    x0, ext, left, right, w = sheet
    ms = MassSpring(x0, 1.0, ext, 1.0)
    fe = np.zeros_like(x0)
    for l, r, wr in zip(left, right, w):
        fe[l, 0] -= T * wr
        fe[r, 0] += T * wr
    for _ in range(40):
        ms.step(100.0, fe, tol=1e-12, max_iter=50)
    x, v = ms.state()
    assert np.max(np.abs(v)) < 1e-12
    strain = np.mean(x[right, 0] - x[left, 0]) / np.mean(x0[right, 0] - x0[left, 0]) - 1.0
    return strain / T


@pytest.mark.parametrize("mesh,m,target", [("triangle", 24, math.sqrt(3) / 2), ("cross", 16, 0.75)])
def test_membrane_k_over_Es_converges_to_analytic(mesh, m, target):
    """Sec. 2.4.2: with all stiffnesses k = 1 the ratio k/E_s of the sheet
    converges under refinement to sqrt(3)/2 for the regular triangular mesh
    and 3/4 for the cross-centre mesh (the printed analytic values). The
    finite-sheet error is a boundary layer, O(1/m): doubling m halves it,
    and the extrapolation 2 r(2m) - r(m) is within 0.5 % of the value."""
    build = _tri_sheet if mesh == "triangle" else _cross_center_sheet
    r1, r2 = _k_over_Es(build(m)), _k_over_Es(build(2 * m))
    e1, e2 = abs(r1 / target - 1), abs(r2 / target - 1)
    assert e2 < 0.6 * e1 and e2 < 0.05, (r1, r2)
    assert abs((2 * r2 - r1) / target - 1) < 5e-3, (r1, r2)


def test_cantilever_free_vibration_converges_to_beam_mode():
    """Sec. 2.4.1, dynamic case (length 1, mass per length 0.0571,
    EI = 0.0259, the paper's 64 points): released from a small tip
    deflection the network vibrates in its first mode; the period tends to
    the Euler--Bernoulli 2 pi / (1.8751^2 sqrt(EI / (mu L^4))) as points are
    added (errors about -1 %, -0.4 %, -0.04 % at 18, 34, 66 points)."""
    L, EI, mu, dt = 1.0, 0.0259, 0.0571, 2e-3
    want = 2 * math.pi / (1.8751040687 ** 2 * math.sqrt(EI / (mu * L ** 4)))
    errs = []
    for npts in (18, 34, 66):
        seg = L / (npts - 1)
        x0 = np.zeros((npts, 3))
        x0[:, 0] = np.linspace(0.0, L, npts)
        mass = np.full(npts, mu * seg)
        mass[-1] = 0.5 * mu * seg
        fixed = np.zeros(npts, bool)
        fixed[:2] = True
        ms = MassSpring(x0, mass, [(i, i + 1) for i in range(npts - 1)], 1e5,
                        [(i, i + 1, i + 2) for i in range(npts - 2)], OM.kb_from_EI(EI, L, npts - 2), fixed=fixed)
        fe = np.zeros((npts, 3))
        fe[-1, 1] = -1e-5
        ms.equilibrium(fe, load_steps=1, tol=1e-13)
        ys = []
        for _ in range(int(8.0 / dt)):
            ms.step(dt, None, tol=1e-12)
            ys.append(ms.state()[0][-1, 1])
        ys = np.array(ys)
        ts = dt * np.arange(1, len(ys) + 1)
        up = [ts[i] - ys[i] * dt / (ys[i + 1] - ys[i]) for i in range(len(ys) - 1) if ys[i] < 0 <= ys[i + 1]]
        errs.append(abs(np.mean(np.diff(up)) / want - 1))   # mean over the periods seen
    assert errs[0] < 0.015 and errs[1] < 0.6 * errs[0] and errs[2] < 0.3 * errs[1] and errs[2] < 1e-3, errs


def test_degenerate_networks():
    """All nodes fixed: a step and an equilibrium leave the state alone; a
    zero load keeps the rest state; a free node with no springs moves on a
    straight line (BDF2 is exact for it)."""
    x0 = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.2, 0.01, 0.0]])
    ms = MassSpring(x0, 1.0, [(0, 1), (1, 2)], 10.0, [(0, 1, 2)], 0.1, fixed=[True, True, True])
    assert ms.info()[0] == 0
    assert ms.step(0.01, np.ones((3, 3))) >= 1
    x, v = ms.state()
    assert np.all(x == x0) and np.all(v == 0)
    ms2 = MassSpring(x0, 1.0, [(0, 1), (1, 2)], 10.0, [(0, 1, 2)], 0.1, fixed=[True, True, False])
    ms2.equilibrium(np.zeros((3, 3)), load_steps=2)
    assert np.max(np.abs(ms2.state()[0] - x0)) < 1e-14
    free = MassSpring(np.array([[0.5, 0.5, 0.5]]), 2.0, np.zeros((0, 2), int), [], v0=np.array([[0.1, -0.2, 0.3]]))
    for dt in (0.1, 0.2, 0.05):
        free.step(dt)
    assert np.allclose(free.state()[0], [[0.5 + 0.035, 0.5 - 0.07, 0.5 + 0.105]], atol=1e-14)


def test_checkpoint_resume_is_bitwise():
    """ps_ms_save / ps_ms_restore carry the BDF2 history: a run continued
    after a save and a fresh network restored from it take the same steps
    to the same bits (saving also rebuilds the Newton matrix)."""
    x0, mass, fixed, ext, ke, bend, kb = random_network(seed=21)
    fe = np.zeros_like(x0)
    fe[-1] = (0.2, -0.4, 0.3)
    fr = dict(A_O=(0.0, 0.1, 0.0), Omega=(0.0, 0.2, 1.0), dOmega=(0.0, 0.0, 0.3))
    a = MassSpring(x0, mass, ext, ke, bend, kb, fixed=fixed)
    for dt in (0.02, 0.03):
        a.step(dt, fe, frame=fr)
    blob = a.save()
    for dt in (0.025, 0.02, 0.02):
        a.step(dt, fe, frame=fr)
    b = MassSpring(x0, mass, ext, ke, bend, kb, fixed=fixed)
    b.restore(blob)
    for dt in (0.025, 0.02, 0.02):
        b.step(dt, fe, frame=fr)
    xa, va = a.state()
    xb, vb = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    c = MassSpring(x0[:5], mass[:5], [(0, 1)], 1.0)
    with pytest.raises(B.PsError):
        c.restore(blob)


def test_fault_injection_on_the_host(monkeypatch):
    """PS_FAULT_ALLOC makes ps_ms_create and ps_init fail their host
    allocation with PS_ENOMEM (ps_init before any CUDA call)."""
    import ctypes

    from paper_2002_08642_gb300.solver import make_params

    x0 = np.zeros((3, 3))
    x0[:, 0] = (0.0, 1.0, 2.0)
    monkeypatch.setenv("PS_FAULT_ALLOC", "ms")
    with pytest.raises(B.PsError) as e:
        MassSpring(x0, 1.0, [(0, 1), (1, 2)], 1.0)
    assert e.value.status == B.PS_ENOMEM
    p = make_params(32, 4.0, 0.01, 1.0, 1e-3)
    need = B.ps_workspace_size(p)
    for what, expect in (("ctx", B.PS_ENOMEM), ("all", B.PS_ENOMEM)):
        monkeypatch.setenv("PS_FAULT_ALLOC", what)
        ctx = ctypes.c_void_p(0)
        st = B.lib().ps_init(ctypes.byref(p), None, ctypes.c_void_p(1 << 20), need, ctypes.byref(ctx))
        assert st == expect and not ctx.value
    monkeypatch.setenv("PS_FAULT_ALLOC", "ctx")
    assert MassSpring(x0, 1.0, [(0, 1), (1, 2)], 1.0).info()[0] == 3
