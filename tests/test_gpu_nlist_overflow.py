"""Recovery from a Verlet-list overflow.

A box whose neighbour list outgrows its capacity (a droplet condensing in a dilute
box, a compressed state, or a capacity set too small) ends with MDEOS_ENBR on the
device; mdeos_poll re-plans it with twice the capacity and runs it again.  The
list's content and order do not depend on its capacity, so the recovered result
must equal, bit for bit, the result of a run whose list was large enough at once.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2508_06012_gb300 as m
    m.build()
    return m


FIELDS = ("P", "T", "sigma", "epot", "ekin", "e_achieved", "P_se", "T_se", "T_target", "e_cold",
          "L", "pairs_per_step", "cand_per_step", "status", "natoms", "nlist_builds", "path",
          "warm")


def _reqs(m):
    return [
        # dilute and cold: liquid droplets condense out of the vapour
        dict(rho=0.3, e=m.e_from_temperature(0.7, 2048), natoms=2048, steps_equil=200,
             steps_avg=200, seed=11, element_id=1),
        dict(rho=0.85, e=m.e_from_temperature(1.2, 864), natoms=864, steps_equil=100,
             steps_avg=100, seed=12, element_id=2),
        dict(rho=1.15, e=m.e_from_temperature(2.5, 4000), natoms=4000, steps_equil=100,
             steps_avg=100, seed=13, element_id=3),
        dict(rho=0.9, e=m.e_from_temperature(1.5, 5324), natoms=5324, steps_equil=60,
             steps_avg=60, seed=14, element_id=4),      # global-memory path
    ]


def test_overflowed_boxes_are_rerun_and_match_a_large_list(m):
    reqs = _reqs(m)
    with m.Engine() as eng:
        ref = eng.evaluate(reqs)
    with m.Engine(nlist_capacity=16) as eng:
        got = eng.evaluate(reqs)
    assert (ref["status"] == 0).all() and (ref["nlist_retries"] == 0).all()
    assert (got["status"] == 0).all(), got["status"]
    assert (got["nlist_retries"] >= 2).all(), got["nlist_retries"]  # 16 -> 32 -> 64 -> ...
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f]), f


def test_rerun_keeps_the_warm_start_state(m):
    """A warm-started request that overflows is re-run from the same stored state
    (the failed attempt neither used up nor invalidated it)."""
    reqs = _reqs(m)[1:3]
    cfg_kw = dict(warm_slots=8, warm_atoms=4096)
    # the final states of a first evaluation, imported into two fresh handles: one
    # with lists too small (its warm-started boxes overflow and are re-run), one not
    h = m.mdeos_create(m.mdeos_config_default(**cfg_kw))
    t = m.mdeos_submit(h, reqs)
    m.mdeos_poll(h, t, len(reqs))
    first_state = [m.mdeos_warm_export(h, r["element_id"], r["natoms"]) for r in reqs]
    m.mdeos_destroy(h)
    h2 = m.mdeos_create(m.mdeos_config_default(nlist_capacity=16, **cfg_kw))
    h3 = m.mdeos_create(m.mdeos_config_default(**cfg_kw))
    for hh in (h2, h3):
        for r, (x, v, L) in zip(reqs, first_state):
            m.mdeos_warm_import(hh, r["element_id"], x[:, :3], v[:, :3], L)
    r2 = m.mdeos_poll(h2, m.mdeos_submit(h2, reqs), len(reqs))
    r3 = m.mdeos_poll(h3, m.mdeos_submit(h3, reqs), len(reqs))
    m.mdeos_destroy(h2)
    m.mdeos_destroy(h3)
    assert (r2["warm"] == 1).all() and (r3["warm"] == 1).all()
    assert (r2["nlist_retries"] >= 1).all() and (r3["nlist_retries"] == 0).all()
    for f in FIELDS:
        assert np.array_equal(r2[f], r3[f]), f
