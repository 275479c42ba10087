"""Parameter-shift gradients of the Trotterised ansatz energy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Not in the paper (which hands E(theta) to an unnamed optimiser, Sec. II-A and
Sec. III-D). Each Pauli rotation exp(-i phi_k P_k / 2) with P_k^2 = I satisfies
dE/dphi_k = [E(phi_k + pi/2) - E(phi_k - pi/2)] / 2, and phi_k = scale_k theta_e, so
dE/dtheta_e = sum_{k : param(k) = e} scale_k [E(phi_k + pi/2) - E(phi_k - pi/2)] / 2,
shifting one rotation at a time.
"""
import numpy as np


def rotation_angles(rot_pidx, rot_scale, theta):
    return np.asarray(rot_scale) * np.asarray(theta)[np.asarray(rot_pidx)]


def parameter_shift(energy_of_angles, rot_pidx, rot_scale, theta, sel):
    """energy_of_angles(phis) -> E; returns dE/dtheta_e for e in sel."""
    phis = rotation_angles(rot_pidx, rot_scale, theta)
    out = []
    for e in sel:
        g = 0.0
        for k in np.nonzero(np.asarray(rot_pidx) == e)[0]:
            p = phis.copy(); p[k] += np.pi / 2
            m = phis.copy(); m[k] -= np.pi / 2
            g += rot_scale[k] * (energy_of_angles(p) - energy_of_angles(m)) / 2
        out.append(g)
    return np.array(out)
