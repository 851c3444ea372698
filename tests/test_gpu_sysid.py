"""System identification through the GPU adjoint (the paper's system-identification
application, on synthetic data): recover the stretch stiffness and the friction
coefficient of a cloth sliding down a slope while it breathes, from positions
observed every third step.  The observations come from the CPU oracle at the
true parameters; the identification runs libdc's rollout and backward inside
scipy's L-BFGS-B."""
import math

import numpy as np
import pytest

import scenes
from oracle import cloth as oc
from tests._helpers import make_cloth

pytestmark = pytest.mark.gpu


def test_recover_stretch_stiffness_and_friction():
    from paper_2106_05306_gb300.sysid import SystemID
    sc = scenes.sliding_breathing_scene()
    true = {"k_stretch": 600.0, "mu": 0.55}
    M = oc.model_from_scene(sc, **true)
    xs, _, recs = oc.rollout(M, sc.x0, sc.v0, sc.n_steps)
    assert all(np.all(r.cases == oc.SLIP) for r in recs)       # sliding the whole time
    observed = {n: xs[n] for n in range(3, sc.n_steps + 1, 3)}
    cloth = make_cloth(sc, k_stretch=1000.0, mu=0.4)
    sid = SystemID(cloth, sc.x0, sc.v0, sc.n_steps, observed, fit=("k_stretch", "mu"))
    out = sid.run({}, bounds={"k_stretch": (10.0, 1e5), "mu": (0.0, 1.5)}, maxiter=40)
    th = out["theta"]
    print(out["iterations"], out["evaluations"], out["initial_loss"], out["loss"], th)
    assert abs(th["k_stretch"] / true["k_stretch"] - 1.0) < 1e-4
    assert abs(th["mu"] - true["mu"]) < 1e-5
    assert out["loss"] < 1e-10 * out["initial_loss"]
    cloth.close()
