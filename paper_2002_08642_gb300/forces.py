"""Lift and drag of the revolving wing from the penalization force (Sec.
4.2: the lift is the force along the vertical axis Oz; the drag is the force
perpendicular to the plane of the vertical and the wing's spanwise axis,
counted positive against the wing's motion; coefficients divide by the
force unit M L T^-2 of the normalisation, here rho = L = T = 1)."""
import numpy as np


def lift_drag(F, R, span_axis=(0.0, 1.0, 0.0), omega_z=1.0):
    """(lift, drag) of the force F (global frame) on a wing whose wing-frame
    span axis is ``span_axis`` and whose frame has rotation R (global =
    X_O + R x_wing), revolving about +z with rate sign ``omega_z``.

    The direction of motion of the span is d = sign(omega_z) z x s (s the
    global span direction projected on the horizontal plane, normalised);
    lift = F_z, drag = -F . d."""
    F = np.asarray(F, dtype=np.float64)
    s = np.asarray(R, dtype=np.float64).reshape(3, 3) @ np.asarray(span_axis, dtype=np.float64)
    s = np.array([s[0], s[1], 0.0])
    norm = np.linalg.norm(s)
    if norm == 0.0:
        raise ValueError("the span axis is vertical: no drag direction")
    s /= norm
    d = np.sign(omega_z) * np.cross([0.0, 0.0, 1.0], s)
    return float(F[2]), float(-np.dot(F, d))
