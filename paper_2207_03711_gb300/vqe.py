"""VQE outer loop over the C ABI (the optimiser around Eq. 5 of the paper).

The paper minimises E(theta) = <psi(theta)|H|psi(theta)> over the UCCSD amplitudes with
a classical optimiser on the host and the simulator as the energy oracle (Sec. II-B).
This module is that host loop: every energy and gradient comes from vqe_energy /
vqe_gradient (parameter shift with shared-prefix forks over the handle's slots); the
optimiser itself (BFGS from SciPy, Adam, or plain gradient descent) runs on the host.
"""
import numpy as np

from . import vqe_energy, vqe_gradient


def minimize(mps, circ, ham, theta0, iters=100, lr=0.05, method="bfgs", gtol=1e-6, callback=None):
    """Minimise E(theta) from theta0. Returns (theta, energy, history) where history is a
    list of (iteration, energy, gradient norm). Stops when the gradient norm falls below
    gtol or after iters iterations."""
    theta = np.array(theta0, dtype=np.float64, copy=True)
    sel = np.arange(theta.size, dtype=np.int32)
    if method == "bfgs":
        from scipy.optimize import minimize as sp_minimize
        history = []

        def fun(x):
            e = vqe_energy(mps, circ, ham, x)
            g = vqe_gradient(mps, circ, ham, x, sel)
            history.append((len(history), float(e), float(np.linalg.norm(g))))
            if callback is not None:
                callback(len(history) - 1, e, g)
            return e, g

        res = sp_minimize(fun, theta, jac=True, method="BFGS", options={"gtol": gtol, "maxiter": iters})
        return np.asarray(res.x), float(res.fun), history
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    b1, b2, eps = 0.9, 0.999, 1e-12
    history = []
    for it in range(iters):
        e = vqe_energy(mps, circ, ham, theta)
        g = vqe_gradient(mps, circ, ham, theta, sel)
        gn = float(np.linalg.norm(g))
        history.append((it, float(e), gn))
        if callback is not None:
            callback(it, e, g)
        if gn < gtol:
            break
        if method == "adam":
            m = b1 * m + (1 - b1) * g
            v = b2 * v + (1 - b2) * g * g
            mh = m / (1 - b1 ** (it + 1))
            vh = v / (1 - b2 ** (it + 1))
            theta -= lr * mh / (np.sqrt(vh) + eps)
        elif method == "gd":
            theta -= lr * g
        else:
            raise ValueError(f"unknown method {method!r}")
    e = vqe_energy(mps, circ, ham, theta)
    return theta, float(e), history
