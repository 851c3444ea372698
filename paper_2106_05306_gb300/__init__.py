"""GB300-native differentiable cloth: a PD time step with dry frictional contact
and its adjoint (DiffCloth, arXiv 2106.05306), behind the C ABI of libdc.

This module only marshals arguments: every step of the simulation and of its
gradient runs in libdc's CUDA kernels.  There is no CPU fallback; without the
built library every call raises.

    cloth = Cloth(rest_pos, tris, pins)
    cloth.set_params(k_stretch=1e3, k_bend=1e-3, mu=0.3, h=1/120, obstacles=[...])
    xN, vN = cloth.rollout(x0, v0, n_steps)            # torch float64 (m, 3) tensors
    dx0, dv0, dtheta = cloth.backward(dL_dxN)          # dtheta = dL/d(k_stretch, k_bend, mu)

``rollout_fn`` wraps rollout/backward as a torch.autograd.Function.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import (DC_CAPSULE, DC_MAX_OBSTACLES, DC_PLANE, DC_SPHERE, DCError, check, dc_params, dc_stats,
                   load)

__all__ = ["Cloth", "rollout_fn", "DCError", "load"]

_KIND = {"plane": DC_PLANE, "sphere": DC_SPHERE, "capsule": DC_CAPSULE}


def _torch():
    import torch
    return torch


def _obstacle_struct(ob, out):
    if isinstance(ob, dict):
        get = ob.get
    else:
        def get(k, d=None):
            return getattr(ob, k, d)
    kind = get("kind")
    out.kind = _KIND[kind] if isinstance(kind, str) else int(kind)
    p = [0.0] * 7
    if out.kind == DC_PLANE:
        p[0:3] = list(get("normal"))
        p[3] = float(get("offset", 0.0))
    elif out.kind == DC_SPHERE:
        p[0:3] = list(get("center"))
        p[3] = float(get("radius"))
    else:
        p[0:3] = list(get("a"))
        p[3:6] = list(get("b"))
        p[6] = float(get("radius"))
    for i in range(7):
        out.p[i] = float(p[i])


class Cloth:
    """One cloth mesh on the GPU (a libdc context)."""

    def __init__(self, rest_pos, tris, pins=(), device="cuda", stream=None):
        torch = _torch()
        lib = load()
        self._lib = lib
        self.device = torch.device(device)
        rest = np.ascontiguousarray(np.asarray(rest_pos, dtype=np.float64).reshape(-1, 3))
        tri = np.ascontiguousarray(np.asarray(tris, dtype=np.int32).reshape(-1, 3))
        pin = np.ascontiguousarray(np.asarray(pins, dtype=np.int32).reshape(-1))
        self.m = rest.shape[0]
        self.n_tris = tri.shape[0]
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.stream = stream
        ctx = ctypes.c_void_p()
        st = lib.dc_create_mesh(ctypes.byref(ctx), self.m, rest.ctypes.data, self.n_tris, tri.ctypes.data,
                                len(pin), pin.ctypes.data if len(pin) else None, ctypes.c_void_p(stream))
        check(st, None)
        self._ctx = ctx
        self.params = None
        self._theta = None

    # ------------------------------------------------------------------ params
    def set_params(self, k_stretch=1e3, k_bend=1e-3, density=0.1, mu=0.3, h=1.0 / 120.0,
                   gravity=(0.0, -9.8, 0.0), contact_margin=1e-6, n_pd_iters=20, obstacles=(),
                   adj_tol=1e-10, adj_max_iters=2000, adj_restart=200, checkpoint_every=1, adj_precond=0):
        p = dc_params()
        self._lib.dc_default_params(ctypes.byref(p))
        p.k_stretch, p.k_bend, p.density, p.mu, p.h = k_stretch, k_bend, density, mu, h
        for i in range(3):
            p.gravity[i] = float(gravity[i])
        p.contact_margin = contact_margin
        p.n_pd_iters = int(n_pd_iters)
        p.adj_tol = adj_tol
        p.adj_max_iters = int(adj_max_iters)
        p.adj_restart = int(adj_restart)
        p.checkpoint_every = int(checkpoint_every)
        p.adj_precond = int(adj_precond)
        obstacles = list(obstacles)
        if len(obstacles) > DC_MAX_OBSTACLES:
            raise ValueError(f"at most {DC_MAX_OBSTACLES} obstacles")
        p.n_obstacles = len(obstacles)
        for i, ob in enumerate(obstacles):
            _obstacle_struct(ob, p.obstacles[i])
        check(self._lib.dc_set_params(self._ctx, ctypes.byref(p)), self._ctx)
        self.params = dict(k_stretch=k_stretch, k_bend=k_bend, density=density, mu=mu, h=h, gravity=tuple(gravity),
                           contact_margin=contact_margin, n_pd_iters=n_pd_iters, obstacles=obstacles,
                           adj_tol=adj_tol, adj_max_iters=adj_max_iters, adj_restart=adj_restart,
                           checkpoint_every=checkpoint_every, adj_precond=adj_precond)
        self._theta = (float(k_stretch), float(k_bend), float(mu))
        return self

    def set_theta(self, k_stretch, k_bend, mu):
        """Change the differentiable parameters (refactorises P when they change)."""
        th = (float(k_stretch), float(k_bend), float(mu))
        if th != self._theta:
            kw = dict(self.params)
            kw.update(k_stretch=th[0], k_bend=th[1], mu=th[2])
            self.set_params(**kw)

    # ------------------------------------------------------------------ helpers
    def _arr(self, a, name):
        torch = _torch()
        if isinstance(a, np.ndarray):
            a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
        if not isinstance(a, torch.Tensor):
            raise TypeError(f"{name}: expected a torch tensor or numpy array")
        if a.dtype != torch.float64:
            raise TypeError(f"{name}: expected float64, got {a.dtype}")
        if a.numel() != 3 * self.m:
            raise ValueError(f"{name}: expected {self.m} x 3 values, got {tuple(a.shape)}")
        return a.contiguous()

    def _like(self, a, shape=None):
        torch = _torch()
        shape = (self.m, 3) if shape is None else shape
        return torch.empty(shape, dtype=torch.float64, device=a.device,
                           pin_memory=(a.device.type == "cpu" and a.is_pinned()))

    # ------------------------------------------------------------------ API
    def step(self, x, v):
        x = self._arr(x, "x")
        v = self._arr(v, "v")
        x1, v1 = self._like(x), self._like(x)
        check(self._lib.dc_step(self._ctx, x.data_ptr(), v.data_ptr(), x1.data_ptr(), v1.data_ptr()), self._ctx)
        return x1, v1

    def rollout(self, x0, v0, n_steps, traj=False):
        x0 = self._arr(x0, "x0")
        v0 = self._arr(v0, "v0")
        xN, vN = self._like(x0), self._like(x0)
        tr = self._like(x0, (n_steps + 1, self.m, 3)) if traj else None
        check(self._lib.dc_rollout(self._ctx, int(n_steps), x0.data_ptr(), v0.data_ptr(), xN.data_ptr(),
                                   vN.data_ptr(), tr.data_ptr() if tr is not None else None), self._ctx)
        self.n_steps = int(n_steps)
        return (xN, vN, tr) if traj else (xN, vN)

    def backward(self, dL_dx, dL_dv=None, dL_dtraj=None, allow_nonconverged=False):
        torch = _torch()
        gx = self._arr(dL_dx, "dL_dx")
        gv = self._arr(dL_dv, "dL_dv") if dL_dv is not None else None
        gt = None
        if dL_dtraj is not None:
            gt = dL_dtraj if isinstance(dL_dtraj, torch.Tensor) else torch.from_numpy(np.asarray(dL_dtraj))
            gt = gt.to(torch.float64).contiguous()
        dx0, dv0 = self._like(gx), self._like(gx)
        dth = torch.empty(3, dtype=torch.float64, device=gx.device)
        st = self._lib.dc_backward(self._ctx, gx.data_ptr(), gv.data_ptr() if gv is not None else None,
                                   gt.data_ptr() if gt is not None else None, dx0.data_ptr(), dv0.data_ptr(),
                                   dth.data_ptr())
        if not (allow_nonconverged and st == 6):
            check(st, self._ctx)
        return dx0, dv0, dth

    def global_solve(self, rhs):
        rhs = self._arr(rhs, "rhs")
        out = self._like(rhs)
        check(self._lib.dc_global_solve(self._ctx, rhs.data_ptr(), out.data_ptr()), self._ctx)
        return out

    def stats(self):
        s = dc_stats()
        check(self._lib.dc_get_stats(self._ctx, ctypes.byref(s)), self._ctx)
        return {k: getattr(s, k) for k, _ in s._fields_}

    def set_kernel_timer(self, kernel_class):
        """Time every launch of one kernel class (name from _lib.KT_CLASSES) on the context's stream."""
        from ._lib import KT_CLASSES
        check(self._lib.dc_set_kernel_timer(self._ctx, KT_CLASSES[kernel_class]), self._ctx)

    def sync(self):
        check(self._lib.dc_sync(self._ctx), self._ctx)

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.dc_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rollout_function():
    torch = _torch()

    class ClothRollout(torch.autograd.Function):
        """(x0, v0, theta) -> (x_N, v_N) through n_steps of libdc; theta = (k_stretch, k_bend, mu).

        Backward re-runs the checkpointed segments and solves one adjoint system per
        step (dc_backward).  One rollout per Cloth may be pending backward at a time."""

        @staticmethod
        def forward(ctx, cloth, n_steps, x0, v0, theta):
            th = theta.detach().cpu().tolist()
            cloth.set_theta(*th)
            xN, vN = cloth.rollout(x0.detach(), v0.detach(), n_steps)
            ctx.cloth = cloth
            ctx.theta_device = theta.device
            return xN, vN

        @staticmethod
        def backward(ctx, gx, gv):
            cloth = ctx.cloth
            if gx is None:
                gx = torch.zeros((cloth.m, 3), dtype=torch.float64, device=cloth.device)
            dx0, dv0, dth = cloth.backward(gx.contiguous(), gv.contiguous() if gv is not None else None)
            return None, None, dx0, dv0, dth.to(ctx.theta_device)

    return ClothRollout


_FN = None


def rollout_fn(cloth: Cloth, x0, v0, theta, n_steps: int):
    """Differentiable rollout: returns (x_N, v_N); gradients flow to x0, v0 and theta."""
    global _FN
    if _FN is None:
        _FN = _rollout_function()
    return _FN.apply(cloth, int(n_steps), x0, v0, theta)
