"""Shared helpers for the GPU parity tests: the same seeded scene goes to the
CUDA library (through the C ABI binding) and to the CPU oracle."""
import dataclasses

import numpy as np

STATE_TOL = 1e-9      # per-step state parity: max|a - b| / max(max|b|, 1e-3)
GRAD_TOL = 1e-7       # gradient parity: |a - b|_2 / |b|_2


def make_cloth(sc, device="cuda", **over):
    import paper_2106_05306_gb300 as dc
    from paper_2106_05306_gb300 import build
    build.build()
    p = dataclasses.replace(sc.params, **{k: v for k, v in over.items() if hasattr(sc.params, k)})
    extra = {k: v for k, v in over.items() if not hasattr(sc.params, k)}
    cloth = dc.Cloth(sc.rest_pos, sc.tris, sc.pins, device=device)
    cloth.set_params(k_stretch=p.k_stretch, k_bend=p.k_bend, density=p.density, mu=p.mu, h=p.h,
                     gravity=p.gravity, contact_margin=p.contact_margin, n_pd_iters=p.n_pd_iters,
                     contact_compliance=p.contact_compliance, obstacles=extra.pop("obstacles", sc.obstacles),
                     **extra)
    return cloth


def oracle_model(sc, **over):
    from oracle import cloth as oc
    return oc.model_from_scene(sc, **{k: v for k, v in over.items() if hasattr(sc.params, k)})


def rel_inf(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-3))


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def cuda(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


def params_kw(sc, **over):
    """The set_params keyword arguments of a scene (with overrides)."""
    p = dataclasses.replace(sc.params, **{k: v for k, v in over.items() if hasattr(sc.params, k)})
    kw = dict(k_stretch=p.k_stretch, k_bend=p.k_bend, density=p.density, mu=p.mu, h=p.h, gravity=p.gravity,
              contact_margin=p.contact_margin, n_pd_iters=p.n_pd_iters, contact_compliance=p.contact_compliance,
              obstacles=sc.obstacles)
    kw.update({k: v for k, v in over.items() if not hasattr(sc.params, k)})
    return kw


def make_batch(scs, device="cuda", **over):
    import paper_2106_05306_gb300 as dc
    from paper_2106_05306_gb300 import build
    build.build()
    batch = dc.ClothBatch([(s.rest_pos, s.tris, s.pins) for s in scs], device=device)
    batch.set_params([params_kw(s, **over) for s in scs])
    return batch


# ---------------------------------------------------------------- oracle in worker processes
# The large parity tests run the oracle along the GPU's own trajectory: every
# step is recomputed from the GPU's (x_n, v_n), so the comparison isolates one
# step (or one adjoint solve) at a time, and the independent steps and Hessian
# assemblies run in a pool of spawned processes (the adjoint solves themselves
# stay sequential, per cloth).

_MODELS = {}


def _scene(spec):
    import scenes
    kind, arg, over = spec
    if kind == "batch":
        sc = scenes.batch_instance(arg)
    elif kind == "capsules":
        sc = scenes.capsule_field(seed=arg)
    else:
        sc = scenes.draped_cloth()
    return sc, over


def _model(spec):
    if spec not in _MODELS:
        from oracle import cloth as oc
        sc, over = _scene(spec)
        _MODELS[spec] = oc.model_from_scene(sc, **dict(over))
    return _MODELS[spec]


def _job_step(job):
    from oracle import cloth as oc
    spec, x, v = job
    return oc.step(_model(spec), x, v)


def _job_hessian(job):
    from oracle import cloth as oc
    spec, x1 = job
    return oc.hessian_W(_model(spec), x1)


def _job_gradient(job):
    from oracle import cloth as oc
    spec, recs, hs, gx, permc = job
    return oc.rollout_gradient(_model(spec), recs, gx, hessians=hs, permc_spec=permc)


def oracle_along(specs, trajs, v0s, h, losses, pool, gradient=True, second_ordering=False):
    """For each cloth i (oracle scene spec, GPU positions trajs[i] = x_0..x_N,
    initial velocity v0s[i]): the oracle's step from every GPU state (velocities
    recovered as (x_{n+1} - x_n)/h), and the oracle's direct adjoint of sum(xi * x_N)
    along those steps (gradient=False: steps only).  Returns (records, gradients);
    with second_ordering, gradients[i] is a pair: the adjoint with the sparse LU's
    default column ordering and with another one (their difference is the
    rounding the oracle's own KKT solves amplify)."""
    jobs, index = [], []
    for i, (spec, tr) in enumerate(zip(specs, trajs)):
        v = np.asarray(v0s[i], dtype=np.float64)
        for n in range(len(tr) - 1):
            jobs.append((spec, tr[n], v))
            index.append(i)
            v = (tr[n + 1] - tr[n]) / h
    out = pool.map(_job_step, jobs, chunksize=1)
    recs = [[] for _ in specs]
    for i, (_, _, rec) in zip(index, out):
        recs[i].append(rec)
    if not gradient:
        return recs, None
    hs = pool.map(_job_hessian, [(specs[i], r.x_np1) for i in range(len(specs)) for r in recs[i]], chunksize=1)
    hper, k = [], 0
    for i in range(len(specs)):
        hper.append(hs[k:k + len(recs[i])])
        k += len(recs[i])
    orders = [None, "MMD_ATA"] if second_ordering else [None]
    jobs = [(specs[i], recs[i], hper[i], losses[i], o) for i in range(len(specs)) for o in orders]
    out = pool.map(_job_gradient, jobs, chunksize=1)
    grads = [tuple(out[len(orders) * i:len(orders) * (i + 1)]) if second_ordering else out[i]
             for i in range(len(specs))]
    return recs, grads


def spawn_pool():
    import multiprocessing
    import os
    return multiprocessing.get_context("spawn").Pool(os.cpu_count() or 1)
