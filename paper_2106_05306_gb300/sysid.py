"""System identification through the adjoint: recover a cloth's stretch stiffness,
bending stiffness and friction coefficient from an observed trajectory (the
paper's "System Identification" application, Sec. 5, on synthetic data).

The loss is the trajectory mismatch L(theta) = 1/2 sum_{n in obs} |x_n(theta) - x^_n|^2
over the observed steps; its gradient comes from one dc_rollout and one
dc_backward (the per-step loss goes in as dL/dx_n).  Stiffnesses are optimised in
log space, friction linearly, with scipy's L-BFGS-B inside bounds; the loss is
scaled so that the optimiser's first step (a full gradient step of its unit-
curvature model) moves no variable by more than first_step.  Every
simulation and gradient step runs in libdc; this module only sets parameters,
moves arrays and calls the optimiser.
"""
from __future__ import annotations

import math

import numpy as np

NAMES = ("k_stretch", "k_bend", "mu")
LOG = {"k_stretch": True, "k_bend": True, "mu": False}


class SystemID:
    """cloth: a Cloth with parameters set (the fixed ones are kept); x0, v0: the
    initial state; observed: dict {step n: (m, 3) positions x^_n}; fit: the names
    of the parameters to recover."""

    def __init__(self, cloth, x0, v0, n_steps, observed, fit=("k_stretch", "mu")):
        import torch
        self.cloth = cloth
        self.dev = torch.device(cloth.device)
        self.x0 = torch.as_tensor(np.asarray(x0, dtype=np.float64), device=self.dev)
        self.v0 = torch.as_tensor(np.asarray(v0, dtype=np.float64), device=self.dev)
        self.n_steps = int(n_steps)
        self.obs = {int(n): torch.as_tensor(np.asarray(x, dtype=np.float64), device=self.dev)
                    for n, x in observed.items()}
        if any(n < 0 or n > self.n_steps for n in self.obs):
            raise ValueError("observed steps must lie in [0, n_steps]")
        self.fit = tuple(fit)
        for name in self.fit:
            if name not in NAMES:
                raise ValueError(f"unknown parameter {name}")
        self.history = []

    def theta(self):
        return {k: float(self.cloth.params[k]) for k in NAMES}

    def _to_z(self, th):
        return np.array([math.log(th[k]) if LOG[k] else th[k] for k in self.fit])

    def _from_z(self, z):
        th = self.theta()
        for k, v in zip(self.fit, z):
            th[k] = math.exp(v) if LOG[k] else float(v)
        return th

    def loss_and_grad(self, z):
        """L and dL/dz at the parameters encoded by z (one rollout + one backward)."""
        import torch
        th = self._from_z(z)
        self.cloth.set_theta(th["k_stretch"], th["k_bend"], th["mu"])
        _, _, traj = self.cloth.rollout(self.x0, self.v0, self.n_steps, traj=True)
        dtraj = torch.zeros_like(traj)
        L = 0.0
        for n, xh in self.obs.items():
            d = traj[n] - xh
            dtraj[n] = d
            L += 0.5 * float((d * d).sum())
        zero = torch.zeros_like(self.x0)
        _, _, dth = self.cloth.backward(zero, None, dtraj, allow_nonconverged=True)
        dth = dth.cpu().numpy().reshape(-1)
        g = np.array([dth[NAMES.index(k)] * (th[k] if LOG[k] else 1.0) for k in self.fit])
        self.history.append((dict(th), L))
        return L, g

    def run(self, theta0, bounds=None, maxiter=50, gtol=1e-12, ftol=1e-15, first_step=0.2):
        """Minimise from theta0 (dict); bounds: dict name -> (lo, hi) in natural units.
        Returns the recovered parameters, the final loss and the optimiser record."""
        from scipy.optimize import minimize
        th0 = self.theta()
        th0.update(theta0)
        z0 = self._to_z(th0)
        L0, g0 = self.loss_and_grad(z0)
        scale = first_step / max(float(np.max(np.abs(g0))), 1e-300)

        def scaled(z):
            L, g = self.loss_and_grad(z)
            return scale * L, scale * g
        bz = None
        if bounds:
            bz = []
            for k in self.fit:
                lo, hi = bounds.get(k, (None, None))
                if LOG[k]:
                    bz.append((math.log(lo) if lo else None, math.log(hi) if hi else None))
                else:
                    bz.append((lo, hi))
        res = minimize(scaled, z0, jac=True, method="L-BFGS-B", bounds=bz,
                       options={"maxiter": maxiter, "gtol": gtol, "ftol": ftol})
        th = self._from_z(res.x)
        self.cloth.set_theta(th["k_stretch"], th["k_bend"], th["mu"])
        return {"theta": th, "loss": float(res.fun) / scale, "initial_loss": L0, "iterations": int(res.nit),
                "evaluations": int(res.nfev), "message": str(res.message), "history": self.history}
