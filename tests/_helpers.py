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
