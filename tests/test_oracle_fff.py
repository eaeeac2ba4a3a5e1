"""Pins of the flattening-filter-free variant (no scatter sub-source) in the
oracle: the plan and the sampled particles hold no scatter photons, and the
Eq. 3 counts still add up to the requested histories."""
import numpy as np

from oracle import oracle as O
from paper_1503_01725_b300 import workloads as W


def test_fff_plan_has_no_scatter_photons():
    m = W.fff_model()
    assert m.w[1].sum() == 0.0 and m.w[0].sum() > 0 and m.w[2].sum() > 0
    plan = O.Plan(m, W.beams(W.square_field(10.0)), 100_003)
    assert plan.count.sum() == 100_003
    assert plan.count[:, 1].sum() == 0
    assert not np.any(plan.entries[:, 1] == 1)
    assert np.all(plan.wpsl[1] == 0.0)
    s = O.sample(plan, 4, 0, 100_003, z_surf=W.SSD)      # plan order: sub-source major
    assert not np.any(s["stype"] == 1)
    assert np.any(s["stype"] == 2)
    # the primary fluence is peaked on the axis: more histories per PSL near it
    c = plan.count[0, 0].sum(axis=0)
    n = plan.n_xy
    assert c[n // 2 - 1: n // 2 + 1, n // 2 - 1: n // 2 + 1].mean() > 1.5 * c[n // 2 - 1: n // 2 + 1, 1:3].mean()
