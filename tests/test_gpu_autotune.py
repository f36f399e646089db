"""GPU test of the autotuner (mdeos_autotune): one launch shape (skin, warps per box)
per atom count from the candidate sets, later evaluations still exact and
deterministic, and an explicit cfg.skin overriding the tuned table."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
CAND = (0.2, 0.25, 0.3, 0.35, 0.4, 0.5)


@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2508_06012_gb300 as m
    m.build()
    return m


def _reqs(m):
    rng = np.random.default_rng(5)
    out = []
    for k in range(24):
        n = int([256, 864, 2048, 4000][k % 4])
        out.append(dict(rho=float(rng.uniform(0.5, 1.0)), e=m.e_from_temperature(1.5, n),
                        natoms=n, steps_equil=50, steps_avg=50, seed=100 + k))
    return out


def test_autotune_table_and_evaluation(m):
    reqs = _reqs(m)
    h = m.mdeos_create()
    try:
        tab = m.mdeos_autotune(h, reqs, steps=40)
        assert sorted(tab[:, 0].astype(int)) == [256, 864, 2048, 4000]
        assert all(any(abs(s - c) < 1e-6 for c in CAND) for s in tab[:, 1])
        # warps per box: the planner's (4 for 256 atoms, 8 for 864, 16 for 2048, 32
        # for 4000 atoms) or up to two doublings of it
        w0 = {256: 4, 864: 8, 2048: 16, 4000: 32}
        for row in tab:
            assert int(row[2]) in [w for w in (w0[int(row[0])] * 2 ** k for k in range(3))
                                   if w <= 32], row
        assert (tab[:, 3] > 0).all()
        r1 = m.mdeos_poll(h, m.mdeos_submit(h, reqs), len(reqs))
        r2 = m.mdeos_poll(h, m.mdeos_submit(h, reqs), len(reqs))
        assert (r1["status"] == 0).all() and r1.tobytes() == r2.tobytes()
    finally:
        m.mdeos_destroy(h)


def test_explicit_skin_overrides_tuned_table(m):
    reqs = _reqs(m)
    tuned = m.mdeos_create(m.mdeos_config_default(skin=0.3))
    plain = m.mdeos_create(m.mdeos_config_default(skin=0.3))
    try:
        m.mdeos_autotune(tuned, reqs, steps=40)
        a = m.mdeos_poll(tuned, m.mdeos_submit(tuned, reqs), len(reqs))
        b = m.mdeos_poll(plain, m.mdeos_submit(plain, reqs), len(reqs))
        assert a.tobytes() == b.tobytes()
    finally:
        m.mdeos_destroy(tuned)
        m.mdeos_destroy(plain)
