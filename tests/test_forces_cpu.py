"""Lift and drag of the revolving wing (Sec. 4.2 definitions)."""
import math

import numpy as np
import pytest

from paper_2002_08642_gb300 import inputs
from paper_2002_08642_gb300.forces import lift_drag


def test_lift_and_drag_directions():
    # span along global +x, rotating about +z: the span tip moves along +y
    R = np.eye(3)
    L, D = lift_drag((0.3, -2.0, 1.5), R, span_axis=(1.0, 0.0, 0.0))
    assert L == 1.5 and D == 2.0
    # the revolving wing of the benchmark recipe (span along wing y, pitched
    # 45 degrees about it, at its start angle)
    xw0, tri = inputs.elliptic_wing_mesh(50)
    _, _, fr = inputs.revolving_wing(0.0, xw0, np.zeros(len(xw0)), omega=math.pi / 2)
    R = fr["R"].reshape(3, 3)
    s = R @ np.array([0.0, 1.0, 0.0])
    d = np.cross([0.0, 0.0, 1.0], s / np.linalg.norm(s))
    F = np.array([0.1, 0.2, 0.7]) - 3.0 * d
    L, D = lift_drag(F, R)
    assert L == pytest.approx(0.7) and D == pytest.approx(3.0 - float(np.dot([0.1, 0.2, 0.7], d)))
    with pytest.raises(ValueError):
        lift_drag((0, 0, 1), np.eye(3), span_axis=(0.0, 0.0, 1.0))
