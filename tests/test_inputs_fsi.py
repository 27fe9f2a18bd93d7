"""The coupled loop's synthetic inputs: the structured vein/membrane wing
and the revolving frames (span axis along wing x)."""
import math

import numpy as np

from paper_2002_08642_gb300 import inputs


def test_fsi_wing_structure():
    ns, nc = 6, 4
    w = inputs.fsi_wing(ns=ns, nc=nc, veins=(0, 2, 4))
    n = (ns + 1) * (nc + 1)
    assert w["x0"].shape == (n, 3) and np.all(w["x0"][:, 2] == 0)
    assert w["tri"].shape == (2 * ns * nc, 3)
    # every triangle edge is an extension spring, each once
    edges = {tuple(sorted(e)) for e in w["ext"].tolist()}
    assert len(edges) == len(w["ext"])
    for t in w["tri"].tolist():
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            assert (min(a, b), max(a, b)) in edges
    # veins: consecutive spanwise triples on the chosen chord lines
    assert len(w["bend"]) == 3 * (ns - 1)
    for i, j, k in w["bend"].tolist():
        assert j - i == k - j == nc + 1
    # the two root stations are clamped; mass sums to the total
    assert w["fixed"].sum() == 2 * (nc + 1) and np.all(w["fixed"][:2 * (nc + 1)])
    assert math.isclose(w["mass"].sum(), 0.281)
    # span along wing x from 0 to 1, chord symmetric about y = 0
    assert math.isclose(w["x0"][:, 0].max(), 1.0) and math.isclose(w["x0"][:, 1].sum(), 0.0, abs_tol=1e-12)


def test_revolving_frames():
    fr, ms = inputs.revolving_frames(0.3, tau=0.4)
    R = fr["R"].reshape(3, 3)
    assert np.allclose(R @ R.T, np.eye(3)) and math.isclose(np.linalg.det(R), 1.0)
    # the wing's span (wing x) lies in the rotating horizontal plane, at the
    # revolving angle phi(t) about global z
    phi, rate = inputs.revolving_angle(0.3, 1.0, 0.4)
    span = R @ np.array([1.0, 0.0, 0.0])
    assert math.isclose(span[2], 0.0, abs_tol=1e-12)
    assert math.isclose(math.atan2(span[1], span[0]), phi + math.pi / 2, abs_tol=1e-12)
    # the network's frame: Omega and dOmega are the global rotation in wing axes
    assert np.allclose(R @ np.asarray(ms["Omega"]), (0.0, 0.0, rate))
    acc = math.exp(-0.3 / 0.4) / 0.4
    assert np.allclose(R @ np.asarray(ms["dOmega"]), (0.0, 0.0, acc))
    assert np.allclose(fr["Omega"], (0.0, 0.0, rate))
