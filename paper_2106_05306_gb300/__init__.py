"""GB300-native differentiable cloth: a PD time step with dry frictional contact
and its adjoint (DiffCloth, arXiv 2106.05306), behind the C ABI of libdc.

This module only marshals arguments: every step of the simulation and of its
gradient runs in libdc's CUDA kernels.  There is no CPU fallback; without the
built library every call raises.

    cloth = Cloth(rest_pos, tris, pins)
    cloth.set_params(k_stretch=1e3, k_bend=1e-3, mu=0.3, h=1/120, obstacles=[...])
    xN, vN = cloth.rollout(x0, v0, n_steps)            # torch float64 (m, 3) tensors
    dx0, dv0, dtheta = cloth.backward(dL_dxN)          # dtheta = dL/d(k_stretch, k_bend, mu)

    batch = ClothBatch([(rest_0, tris_0, pins_0), (rest_1, tris_1, pins_1), ...])
    batch.set_params([dict(k_stretch=..., mu=..., obstacles=[...]), ...])
    xN, vN = batch.rollout(x0, v0, n_steps)            # concatenated (sum m_i, 3) tensors
    dx0, dv0, dtheta = batch.backward(dL_dxN)          # dtheta: (n_instances, 3)

``rollout_fn`` wraps rollout/backward as a torch.autograd.Function.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import (COMPLIANCE, DC_CAPSULE, DC_MAX_OBSTACLES, DC_MESH, DC_PLANE, DC_SPHERE, LAYOUTS, STATUS_NAMES, DCError,
                   check, dc_instance, dc_params, dc_request, dc_result, dc_server_config, dc_server_stats, dc_stats,
                   load)

__all__ = ["Cloth", "ClothBatch", "Server", "rollout_fn", "batch_hbm_bytes", "fma_peak", "DCError", "load"]

_KIND = {"plane": DC_PLANE, "sphere": DC_SPHERE, "capsule": DC_CAPSULE, "mesh": DC_MESH}

_PARAM_DEFAULTS = dict(k_stretch=1e3, k_bend=1e-3, density=0.1, mu=0.3, h=1.0 / 120.0, gravity=(0.0, -9.8, 0.0),
                       contact_margin=1e-6, n_pd_iters=20, obstacles=(), adj_tol=1e-10, adj_max_iters=2000,
                       adj_restart=200, checkpoint_every=1, adj_precond=0, global_solver=0,
                       contact_compliance="rowsum", adj_fallback=1, factor_on_gpu=0)


def _torch():
    import torch
    return torch


def _obstacle_struct(ob, out, mesh_ids=None):
    if isinstance(ob, dict):
        get = ob.get
    else:
        def get(k, d=None):
            return getattr(ob, k, d)
    kind = get("kind")
    out.kind = _KIND[kind] if isinstance(kind, str) else int(kind)
    p = [0.0] * 7
    if out.kind == DC_MESH:
        if mesh_ids is None or id(ob) not in mesh_ids:
            raise ValueError("a mesh obstacle must be registered with the context (set_params does this)")
        p[0] = float(mesh_ids[id(ob)])
    elif out.kind == DC_PLANE:
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


def _make_params(lib, kw, mesh_ids=None) -> dc_params:
    unknown = set(kw) - set(_PARAM_DEFAULTS)
    if unknown:
        raise TypeError(f"unknown parameter(s): {sorted(unknown)}")
    q = dict(_PARAM_DEFAULTS)
    q.update(kw)
    p = dc_params()
    lib.dc_default_params(ctypes.byref(p))
    p.k_stretch, p.k_bend, p.density, p.mu, p.h = q["k_stretch"], q["k_bend"], q["density"], q["mu"], q["h"]
    for i in range(3):
        p.gravity[i] = float(q["gravity"][i])
    p.contact_margin = q["contact_margin"]
    p.n_pd_iters = int(q["n_pd_iters"])
    p.adj_tol = q["adj_tol"]
    p.adj_max_iters = int(q["adj_max_iters"])
    p.adj_restart = int(q["adj_restart"])
    p.checkpoint_every = int(q["checkpoint_every"])
    p.adj_precond = int(q["adj_precond"])
    p.global_solver = int(q["global_solver"])
    cm = q["contact_compliance"]
    p.contact_compliance = COMPLIANCE[cm] if isinstance(cm, str) else int(cm)
    p.adj_fallback = int(q["adj_fallback"])
    p.factor_on_gpu = int(q["factor_on_gpu"])
    obstacles = list(q["obstacles"])
    if len(obstacles) > DC_MAX_OBSTACLES:
        raise ValueError(f"at most {DC_MAX_OBSTACLES} obstacles")
    p.n_obstacles = len(obstacles)
    for i, ob in enumerate(obstacles):
        _obstacle_struct(ob, p.obstacles[i], mesh_ids)
    q["obstacles"] = obstacles
    q["gravity"] = tuple(q["gravity"])
    return p, q


def _mesh_arrays(rest_pos, tris, pins):
    rest = np.ascontiguousarray(np.asarray(rest_pos, dtype=np.float64).reshape(-1, 3))
    tri = np.ascontiguousarray(np.asarray(tris, dtype=np.int32).reshape(-1, 3))
    pin = np.ascontiguousarray(np.asarray(pins, dtype=np.int32).reshape(-1))
    return rest, tri, pin


class _Context:
    """Common marshalling of a libdc context (one cloth or a batch)."""

    def _init_common(self, ctx, device):
        self._ctx = ctx
        self.device = device
        n = ctypes.c_int32()
        check(self._lib.dc_get_layout(self._ctx, ctypes.byref(n), None), self._ctx)
        offs = np.zeros(n.value + 1, dtype=np.int64)
        check(self._lib.dc_get_layout(self._ctx, ctypes.byref(n), offs.ctypes.data), self._ctx)
        self.n_instances = int(n.value)
        self.node_offsets = offs
        self.m = int(offs[-1])
        self.params = None
        self.layout = "node_major"

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

    def _node_shape(self):
        return (3, self.m) if self.layout == "component_major" else (self.m, 3)

    def _like(self, a, shape=None):
        torch = _torch()
        shape = self._node_shape() if shape is None else shape
        return torch.empty(shape, dtype=torch.float64, device=a.device,
                           pin_memory=(a.device.type == "cpu" and a.is_pinned()))

    def split(self, a):
        """Split a concatenated (m, 3) node array into the per-instance (m_i, 3) views."""
        o = self.node_offsets
        return [a[int(o[i]):int(o[i + 1])] for i in range(self.n_instances)]

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
        tr = self._like(x0, (n_steps + 1,) + self._node_shape()) if traj else None
        check(self._lib.dc_rollout(self._ctx, int(n_steps), x0.data_ptr(), v0.data_ptr(), xN.data_ptr(),
                                   vN.data_ptr(), tr.data_ptr() if tr is not None else None), self._ctx)
        self.n_steps = int(n_steps)
        return (xN, vN, tr) if traj else (xN, vN)

    def _backward(self, dL_dx, dL_dv, dL_dtraj, allow_nonconverged, dth_shape):
        torch = _torch()
        gx = self._arr(dL_dx, "dL_dx")
        gv = self._arr(dL_dv, "dL_dv") if dL_dv is not None else None
        gt = None
        if dL_dtraj is not None:
            gt = dL_dtraj if isinstance(dL_dtraj, torch.Tensor) else torch.from_numpy(np.asarray(dL_dtraj))
            gt = gt.to(torch.float64).contiguous()
        dx0, dv0 = self._like(gx), self._like(gx)
        dth = torch.empty(dth_shape, dtype=torch.float64, device=gx.device,
                          pin_memory=(gx.device.type == "cpu" and gx.is_pinned()))
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

    def _register_meshes(self, obstacles):
        """Registers the mesh obstacles of a parameter set with the context (once per
        obstacle object) and returns {id(obstacle): mesh id}."""
        if not hasattr(self, "_meshes"):
            self._meshes = {}          # id(obstacle) -> (obstacle, mesh id); keeps the objects alive
        for ob in obstacles:
            kind = ob.get("kind") if isinstance(ob, dict) else getattr(ob, "kind", None)
            if kind != "mesh" and kind != DC_MESH:
                continue
            if id(ob) in self._meshes:
                continue
            V = ob["vertices"] if isinstance(ob, dict) else ob.vertices
            F = ob["triangles"] if isinstance(ob, dict) else ob.triangles
            V = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(-1, 3))
            F = np.ascontiguousarray(np.asarray(F, dtype=np.int32).reshape(-1, 3))
            mid = ctypes.c_int32()
            check(self._lib.dc_add_obstacle_mesh(self._ctx, V.shape[0], V.ctypes.data, F.shape[0], F.ctypes.data,
                                                 ctypes.byref(mid)), self._ctx)
            self._meshes[id(ob)] = (ob, mid.value)
        return {k: v[1] for k, v in self._meshes.items()}

    def set_layout(self, layout):
        """Node arrays of later calls: "node_major" ((m, 3), the default) or
        "component_major" ((3, m): all x, then all y, then all z)."""
        check(self._lib.dc_set_layout(self._ctx, LAYOUTS[layout]), self._ctx)
        self.layout = layout
        return self

    def set_graphs(self, enable=True):
        """Replay the forward steps of rollouts as captured CUDA graphs (results unchanged)."""
        check(self._lib.dc_set_graphs(self._ctx, 1 if enable else 0), self._ctx)
        return self

    def autotune(self):
        """Pick the block sizes of the element and node kernels by timing them (results unchanged)."""
        check(self._lib.dc_autotune(self._ctx), self._ctx)
        return self

    def stats(self):
        s = dc_stats()
        check(self._lib.dc_get_stats(self._ctx, ctypes.byref(s)), self._ctx)
        return {k: getattr(s, k) for k, _ in s._fields_ if k != "reserved_"}

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


class Cloth(_Context):
    """One cloth mesh on the GPU (a libdc context)."""

    def __init__(self, rest_pos, tris, pins=(), device="cuda", stream=None):
        torch = _torch()
        self._lib = load()
        device = torch.device(device)
        rest, tri, pin = _mesh_arrays(rest_pos, tris, pins)
        self.n_tris = tri.shape[0]
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.stream = stream
        ctx = ctypes.c_void_p()
        st = self._lib.dc_create_mesh(ctypes.byref(ctx), rest.shape[0], rest.ctypes.data, self.n_tris,
                                      tri.ctypes.data, len(pin), pin.ctypes.data if len(pin) else None,
                                      ctypes.c_void_p(stream))
        check(st, None)
        self._init_common(ctx, device)
        self._theta = None
        # rollout_fn's backward accepts adjoint steps stopped at their rounding
        # floor above adj_tol when this is set (they are counted in stats())
        self.allow_nonconverged = False

    def set_params(self, **kw):
        p, q = _make_params(self._lib, kw, self._register_meshes(kw.get("obstacles", ())))
        check(self._lib.dc_set_params(self._ctx, ctypes.byref(p)), self._ctx)
        self.params = q
        self._theta = (float(q["k_stretch"]), float(q["k_bend"]), float(q["mu"]))
        return self

    def set_theta(self, k_stretch, k_bend, mu):
        """Change the differentiable parameters (refactorises P when they change)."""
        th = (float(k_stretch), float(k_bend), float(mu))
        if th != self._theta:
            kw = dict(self.params)
            kw.update(k_stretch=th[0], k_bend=th[1], mu=th[2])
            self.set_params(**kw)

    def backward(self, dL_dx, dL_dv=None, dL_dtraj=None, allow_nonconverged=False):
        return self._backward(dL_dx, dL_dv, dL_dtraj, allow_nonconverged, (3,))


class ClothBatch(_Context):
    """Several cloth meshes of any sizes packed into one libdc context: every phase of
    the step and of the adjoint is one launch over all of them.  Node arrays are the
    concatenation of the instances' (m_i, 3) arrays (``node_offsets``)."""

    def __init__(self, meshes, device="cuda", stream=None):
        torch = _torch()
        self._lib = load()
        device = torch.device(device)
        arrays = [_mesh_arrays(*mesh) for mesh in meshes]
        if not arrays:
            raise ValueError("ClothBatch needs at least one mesh")
        inst = (dc_instance * len(arrays))()
        for i, (rest, tri, pin) in enumerate(arrays):
            inst[i].n_nodes = rest.shape[0]
            inst[i].n_tris = tri.shape[0]
            inst[i].n_pins = len(pin)
            inst[i].rest_pos = rest.ctypes.data
            inst[i].tris = tri.ctypes.data
            inst[i].pins = pin.ctypes.data if len(pin) else None
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.stream = stream
        ctx = ctypes.c_void_p()
        check(self._lib.dc_create_batch(ctypes.byref(ctx), len(arrays), ctypes.addressof(inst),
                                        ctypes.c_void_p(stream)), None)
        self._init_common(ctx, device)

    def instance_nonconverged(self):
        """Per instance: adjoint steps since creation that stopped above adj_tol
        (which instances a non-converged backward concerns)."""
        import numpy as np
        out = np.zeros(self.n_instances, dtype=np.int64)
        check(self._lib.dc_get_instance_nonconverged(self._ctx, out.ctypes.data), self._ctx)
        return out

    def set_params(self, params):
        """params: one dict for every instance, or a list of n_instances dicts.  Only
        k_stretch, k_bend, density, mu and obstacles may differ between instances."""
        if isinstance(params, dict):
            params = [params] * self.n_instances
        params = list(params)
        built = [_make_params(self._lib, kw, self._register_meshes(kw.get("obstacles", ()))) for kw in params]
        arr = (dc_params * len(built))(*[b[0] for b in built])
        check(self._lib.dc_set_params_batch(self._ctx, len(built), ctypes.addressof(arr)), self._ctx)
        self.params = [b[1] for b in built]
        return self

    def set_instance_steps(self, steps):
        """Per-instance step counts for the next rollouts (None: one count for all):
        instance i takes steps[i] steps, then keeps its state."""
        if steps is None:
            check(self._lib.dc_set_instance_steps(self._ctx, None), self._ctx)
            return self
        arr = np.ascontiguousarray(np.asarray(steps, dtype=np.int32).reshape(-1))
        if arr.shape[0] != self.n_instances:
            raise ValueError(f"expected {self.n_instances} step counts")
        check(self._lib.dc_set_instance_steps(self._ctx, arr.ctypes.data), self._ctx)
        return self

    def set_theta(self, theta):
        """Per-instance differentiable parameters, shape (n_instances, 3) = (k_stretch,
        k_bend, mu); refactorises when they change."""
        th = [tuple(float(v) for v in row) for row in np.asarray(theta, dtype=np.float64).reshape(-1, 3)]
        if len(th) != self.n_instances:
            raise ValueError(f"theta: expected {self.n_instances} x 3 values")
        cur = [(q["k_stretch"], q["k_bend"], q["mu"]) for q in self.params]
        if th != cur:
            kws = []
            for q, (ks, kb, mu) in zip(self.params, th):
                kw = dict(q)
                kw.update(k_stretch=ks, k_bend=kb, mu=mu)
                kws.append(kw)
            self.set_params(kws)

    def backward(self, dL_dx, dL_dv=None, dL_dtraj=None, allow_nonconverged=False):
        return self._backward(dL_dx, dL_dv, dL_dtraj, allow_nonconverged, (self.n_instances, 3))


class Server:
    """Request server (dc_server_*): forward + adjoint rollouts submitted at any time,
    admitted by free slot and HBM budget, run concurrently on one GPU.

    ``submit`` copies its arguments and returns a ticket; ``wait(ticket)`` blocks
    until that request is done and returns its results (numpy arrays) and timings."""

    def __init__(self, n_slots=4, n_prep_threads=4, hbm_budget_bytes=None, max_prepared=None, device=0, max_batch=1):
        self._lib = load()
        if hbm_budget_bytes is None:
            torch = _torch()
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget_bytes = int(0.8 * free)
        cfg = dc_server_config(n_slots=int(n_slots), n_prep_threads=int(n_prep_threads),
                               hbm_budget_bytes=int(hbm_budget_bytes),
                               max_prepared=int(max_prepared if max_prepared is not None else 2 * n_slots + 2),
                               device=int(device), max_batch=int(max_batch))
        srv = ctypes.c_void_p()
        check(self._lib.dc_server_create(ctypes.byref(srv), ctypes.byref(cfg)), None)
        self._srv = srv
        self._sizes = {}
        self.hbm_budget_bytes = int(hbm_budget_bytes)

    def submit(self, rest_pos, tris, pins, x0, v0, dL_dx, n_steps, params=None, dL_dv=None):
        rest, tri, pin = _mesh_arrays(rest_pos, tris, pins)
        f64 = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1, 3)) for a in (x0, v0, dL_dx)]
        gv = np.ascontiguousarray(np.asarray(dL_dv, dtype=np.float64).reshape(-1, 3)) if dL_dv is not None else None
        m = rest.shape[0]
        for a in f64 + ([gv] if gv is not None else []):
            if a.shape[0] != m:
                raise ValueError(f"expected {m} x 3 values, got {a.shape}")
        p, _ = _make_params(self._lib, dict(params or {}))
        req = dc_request(n_nodes=m, n_tris=tri.shape[0], n_pins=len(pin), n_steps=int(n_steps),
                         rest_pos=rest.ctypes.data, tris=tri.ctypes.data,
                         pins=pin.ctypes.data if len(pin) else None, x0=f64[0].ctypes.data, v0=f64[1].ctypes.data,
                         dL_dx_final=f64[2].ctypes.data, dL_dv_final=gv.ctypes.data if gv is not None else None,
                         params=p)
        t = ctypes.c_int64()
        check(self._lib.dc_server_submit(self._srv, ctypes.byref(req), ctypes.byref(t)), None)
        self._sizes[t.value] = m
        return t.value

    def wait(self, ticket):
        m = self._sizes.pop(ticket)
        out = {k: np.empty((m, 3)) for k in ("x_final", "v_final", "dL_dx0", "dL_dv0")}
        r = dc_result(x_final=out["x_final"].ctypes.data, v_final=out["v_final"].ctypes.data,
                      dL_dx0=out["dL_dx0"].ctypes.data, dL_dv0=out["dL_dv0"].ctypes.data)
        check(self._lib.dc_server_wait(self._srv, int(ticket), ctypes.byref(r)), None)
        out.update(status=STATUS_NAMES.get(r.status, r.status), dL_dparams=np.array(list(r.dL_dparams)),
                   slot=r.slot, t_submit=r.t_submit, t_admit=r.t_admit, t_done=r.t_done,
                   device_bytes=r.device_bytes, device_bytes_peak=r.device_bytes_peak, adj_iters=r.adj_iters,
                   message=r.message.decode())
        return out

    def stats(self):
        s = dc_server_stats()
        check(self._lib.dc_server_get_stats(self._srv, ctypes.byref(s)), None)
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "_srv", None):
            self._lib.dc_server_destroy(self._srv)
            self._srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fma_peak(precision=64, n_iter=None):
    """Measured FMA throughput of the current GPU's CUDA cores (TFLOP/s) in FP64 or FP32."""
    lib = load()
    if n_iter is None:
        n_iter = 1000 if precision == 64 else 20000
    out = ctypes.c_double()
    check(lib.dc_fma_peak(int(precision), int(n_iter), ctypes.byref(out)), None)
    return float(out.value)


def front_factor(A, p, threads=512, use_tc=True, use_gscr=False):
    """One dense front through the adjoint preconditioner's front kernel (a test
    hook): A is a symmetric (n, n) array, p the pivot count.  Returns (F, Linv):
    F holds D and the unit-lower L in its first p columns and the Schur complement
    in its trailing lower triangle (float32, (n, n)); Linv is the inverse of L's
    pivot block ((p, p))."""
    import numpy as np
    lib = load()
    A = np.asfortranarray(np.asarray(A, dtype=np.float32))
    n = A.shape[0]
    out = np.zeros((n, n), dtype=np.float32, order="F")
    linv = np.zeros((p, p), dtype=np.float32, order="F")
    check(lib.dc_debug_front_factor(int(n), int(p), A.ctypes.data, out.ctypes.data, linv.ctypes.data,
                                    int(threads), int(bool(use_tc)), int(bool(use_gscr))), None)
    return out, linv


def batch_hbm_bytes(meshes, params, n_steps):
    """Device bytes a ClothBatch of these meshes (list of (rest_pos, tris, pins)) with
    these parameters (one dict per mesh, or one for all) would hold at most through
    a rollout of n_steps steps and its backward; computed on the host."""
    lib = load()
    arrays = [_mesh_arrays(*mesh) for mesh in meshes]
    inst = (dc_instance * len(arrays))()
    for i, (rest, tri, pin) in enumerate(arrays):
        inst[i].n_nodes = rest.shape[0]
        inst[i].n_tris = tri.shape[0]
        inst[i].n_pins = len(pin)
        inst[i].rest_pos = rest.ctypes.data
        inst[i].tris = tri.ctypes.data
        inst[i].pins = pin.ctypes.data if len(pin) else None
    if isinstance(params, dict):
        params = [params] * len(arrays)
    prm = (dc_params * len(arrays))(*[_make_params(lib, kw)[0] for kw in params])
    out = ctypes.c_int64()
    check(lib.dc_batch_hbm_bytes(len(arrays), ctypes.addressof(inst), ctypes.addressof(prm), int(n_steps),
                                 ctypes.byref(out)), None)
    return int(out.value)


def _rollout_function():
    torch = _torch()

    class ClothRollout(torch.autograd.Function):
        """(x0, v0, theta) -> (x_N, v_N) through n_steps of libdc; theta = (k_stretch, k_bend, mu).

        Backward re-runs the checkpointed segments and solves one adjoint system per
        step (dc_backward).  One rollout per Cloth may be pending backward at a time."""

        @staticmethod
        def forward(ctx, cloth, n_steps, x0, v0, theta):
            th = theta.detach().cpu()
            if isinstance(cloth, ClothBatch):
                cloth.set_theta(th.numpy())
            else:
                cloth.set_theta(*th.tolist())
            xN, vN = cloth.rollout(x0.detach(), v0.detach(), n_steps)
            ctx.cloth = cloth
            ctx.theta_device = theta.device
            return xN, vN

        @staticmethod
        def backward(ctx, gx, gv):
            cloth = ctx.cloth
            if gx is None:
                gx = torch.zeros((cloth.m, 3), dtype=torch.float64, device=cloth.device)
            dx0, dv0, dth = cloth.backward(gx.contiguous(), gv.contiguous() if gv is not None else None,
                                           allow_nonconverged=getattr(cloth, "allow_nonconverged", False))
            return None, None, dx0, dv0, dth.to(ctx.theta_device)

    return ClothRollout


_FN = None


def rollout_fn(cloth, x0, v0, theta, n_steps: int):
    """Differentiable rollout: returns (x_N, v_N); gradients flow to x0, v0 and theta.
    For a Cloth theta is (k_stretch, k_bend, mu); for a ClothBatch it is one such
    row per instance, shape (n_instances, 3), and x0 / v0 are concatenated."""
    global _FN
    if _FN is None:
        _FN = _rollout_function()
    return _FN.apply(cloth, int(n_steps), x0, v0, theta)
