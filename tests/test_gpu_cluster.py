"""Boxes on thread-block clusters (eos_cluster_kernel): a batch of few small boxes
(fewer than half the SMs, all searched without cells) runs every box on a cluster of
up to 8 CTAs, each CTA holding the whole box, computing the forces and lists of its
share of the atoms and sending the forces to the others.  Forces are the same FP32
sums in the same order and box sums are exact, so a clustered box must give the same
bytes as the same box packed with many others on one CTA's warp group."""
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


def _small(m, k0, count, steps=(200, 200)):
    rng = np.random.default_rng(11 + k0)
    out = []
    for k in range(count):
        n = int([256, 300, 384, 500, 729][k % 5])
        T = float(rng.uniform(1.0, 2.0))
        out.append(dict(rho=float(rng.uniform(0.5, 1.0)), e=m.e_from_temperature(T, n), natoms=n,
                        steps_equil=steps[0], steps_avg=steps[1], seed=1000 + k0 + k,
                        element_id=0))
    return out


def _filler(m, count):
    rng = np.random.default_rng(5)
    return [dict(rho=float(rng.uniform(0.6, 0.9)), e=m.e_from_temperature(1.5, 864), natoms=864,
                 steps_equil=40, steps_avg=40, seed=50000 + k) for k in range(count)]


def test_clustered_boxes_equal_packed_boxes(m):
    reqs = _small(m, 0, 10)
    with m.Engine() as eng, m.Engine(max_cluster=8) as eng8:
        alone = eng.evaluate(reqs)          # 10 boxes: clusters of 4 CTAs (152 SMs)
        one = eng8.evaluate(reqs[:1])       # 1 box: a cluster of 8
        mixed = eng.evaluate(reqs + _filler(m, 300))[:10]  # packed, no clusters
    assert (alone["status"] == 0).all()
    assert alone.tobytes() == mixed.tobytes()
    assert one.tobytes() == alone[:1].tobytes()


def test_cluster_plan_shape(m):
    """The batch API reports the launch: 10 small boxes run as 10 clusters of 4."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    reqs = _small(m, 20, 10, steps=(40, 40))
    h = m.mdeos_create()
    try:
        b = m.mdeos_batch_create(h, reqs)
        info = m.mdeos_batch_info(b)
        C = 1
        while C < 4 and 2 * C * 10 <= nsm:
            C *= 2
        assert info["items"] == 10 and info["ctas"] == 10 * C
        m.mdeos_batch_launch(b)
        r = m.mdeos_batch_results(b, 10)
        with m.Engine() as eng:
            ref = eng.evaluate(reqs + _filler(m, 200))[:10]
        assert (r["status"] == 0).all() and r.tobytes() == ref.tobytes()
        m.mdeos_batch_destroy(b)
    finally:
        m.mdeos_destroy(h)


def test_cluster_warm_start_and_overflow(m):
    """Warm starts and a list overflow (re-run with a larger list) on clustered boxes
    give the packed path's bytes too."""
    reqs = _small(m, 40, 6, steps=(60, 60))
    for k, q in enumerate(reqs):
        q["element_id"] = 700 + k
    cfg = dict(warm_slots=16, warm_atoms=1024)
    with m.Engine(**cfg) as a, m.Engine(**cfg) as b:
        for it in range(2):  # cold, then warm
            ra = a.evaluate(reqs)
            rb = b.evaluate(reqs + _filler(m, 200))[:6]
            assert ra.tobytes() == rb.tobytes(), it
        assert (ra["warm"] == 1).all()
    with m.Engine(nlist_capacity=16) as a, m.Engine(nlist_capacity=16) as b:
        ra = a.evaluate(reqs)
        rb = b.evaluate(reqs + _filler(m, 200))[:6]
        assert (ra["nlist_retries"] > 0).any() and (ra["status"] == 0).all()
        for f in ("P", "T", "e_achieved", "sigma", "status", "nlist_builds"):
            assert np.array_equal(ra[f], rb[f]), f


def _big(count, natoms=(5000, 9000, 16384), steps=(40, 40), seed0=0):
    rng = np.random.default_rng(31 + seed0)
    out = []
    for k in range(count):
        n = int(natoms[k % len(natoms)])
        out.append(dict(rho=float(rng.uniform(0.5, 1.0)), e=float(rng.uniform(0.5, 1.5)),
                        natoms=n, steps_equil=steps[0], steps_avg=steps[1], seed=700 + seed0 + k))
    return out


def test_big_boxes_on_clusters_equal_one_cta(m):
    """Boxes above the shared-memory limit on clusters of 4 and 8 CTAs (each CTA a slab
    of the cell-ordered slots, box sums exchanged in rank order) give the bytes of the
    same boxes on one CTA each (max_cluster = 1: no clusters)."""
    reqs = _big(3)
    with m.Engine(max_cluster=1) as one, m.Engine() as four, m.Engine(max_cluster=8) as eight:
        r1 = one.evaluate(reqs)
        r4 = four.evaluate(reqs)
        r8 = eight.evaluate(reqs)
    assert (r1["status"] == 0).all() and (r1["nlist_builds"] > 1).all()
    assert r4.tobytes() == r1.tobytes()
    assert r8.tobytes() == r1.tobytes()


def test_big_cluster_plan_shape_and_overflow(m):
    """The batch API reports 2 big boxes as 2 clusters of 4; a list overflow on a
    clustered big box ends it in every CTA alike and the re-planned run equals the
    one-CTA run."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    reqs = _big(2, natoms=(6000, 7000), steps=(20, 20), seed0=50)
    h = m.mdeos_create()
    try:
        b = m.mdeos_batch_create(h, reqs)
        info = m.mdeos_batch_info(b)
        C = 1
        while 2 * C <= 4 and 2 * (2 * C) * 2 <= nsm:
            C *= 2
        assert info["items"] == 2 and info["ctas"] == 2 * C
        m.mdeos_batch_launch(b)
        r = m.mdeos_batch_results(b, 2)
        m.mdeos_batch_destroy(b)
    finally:
        m.mdeos_destroy(h)
    with m.Engine(max_cluster=1) as one:
        ref = one.evaluate(reqs)
    assert (r["status"] == 0).all() and r.tobytes() == ref.tobytes()
    with m.Engine(nlist_capacity=16) as a, m.Engine(nlist_capacity=16, max_cluster=1) as b1:
        ra = a.evaluate(reqs)
        rb = b1.evaluate(reqs)
    assert (ra["nlist_retries"] > 0).all() and (ra["status"] == 0).all()
    for f in ("P", "T", "e_achieved", "sigma", "status", "nlist_builds"):
        assert np.array_equal(ra[f], rb[f]), f
