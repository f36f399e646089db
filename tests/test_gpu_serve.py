"""GPU tests of the serving loop (mdeos_serve_*): every served result equals the same
request evaluated alone, bit for bit (packing never changes a box's arithmetic);
per-request completion; shedding, back-pressure and the HBM budget."""
import time

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


@pytest.fixture(scope="module")
def h(m):
    hd = m.mdeos_create()
    yield hd
    m.mdeos_destroy(hd)


def _stream_requests(m, k, seed, steps=(60, 60)):
    """Requests shaped like the serving workload (atom counts log-uniform 256..32000,
    rho ~ U[0.3, 1.2], T ~ log-U[0.7, 3]) with short schedules."""
    from paper_2508_06012_gb300 import workloads as w
    return [dict(rho=b["rho"], e=m.e_from_temperature(b["T"], b["natoms"]), natoms=b["natoms"],
                 steps_equil=b["steps_equil"], steps_avg=b["steps_avg"], seed=b["seed"])
            for b in w.serving_stream(seed, k, steps[0], steps[1])]


def test_served_results_equal_solo_runs(m, h):
    reqs = _stream_requests(m, 40, 11)
    with m.Server(h, max_batch=8) as srv:
        ids = []
        rng = np.random.default_rng(3)
        for k in range(0, len(reqs), 5):          # arrivals in bursts while launches run
            ids.extend(srv.enqueue(reqs[k:k + 5]))
            time.sleep(float(rng.uniform(0, 0.02)))
        got = srv.wait_all(len(reqs), timeout_s=300)
        st = srv.stats()
    assert len(got) == len(reqs) and sorted(got["id"]) == sorted(ids)
    assert st["launches"] >= 1 and st["cuda_errors"] == 0 and st["shed"] == 0
    assert (got["t_arrival"] <= got["t_launch"]).all() and (got["t_launch"] <= got["t_done"]).all()
    by_id = {int(g["id"]): g for g in got}
    with m.Engine() as eng:
        solo = eng.evaluate(reqs)
    for i, rid in enumerate(ids):
        assert by_id[int(rid)]["result"].tobytes() == solo[i].tobytes(), i


@pytest.mark.parametrize("cluster", [2, 4, 8])
def test_served_results_on_clusters_equal_solo_runs(m, h, cluster):
    """The serving grid in thread-block clusters (boxes above 4096 atoms on a whole
    cluster, smaller items one per CTA in rounds) serves the bytes of solo runs."""
    reqs = _stream_requests(m, 24, 23)
    with m.Server(h, max_batch=8, cluster=cluster) as srv:
        ids = srv.enqueue(reqs)
        got = srv.wait_all(len(reqs), timeout_s=300)
        st = srv.stats()
    assert st["cuda_errors"] == 0 and st["shed"] == 0
    by_id = {int(g["id"]): g for g in got}
    with m.Engine() as eng:
        solo = eng.evaluate(reqs)
    for i, rid in enumerate(ids):
        assert by_id[int(rid)]["result"].tobytes() == solo[i].tobytes(), i


def test_serve_cluster_size_is_checked(m, h):
    """The serving grid's cluster size is 0, 1, 2, 4 or 8; anything else is rejected."""
    for bad in (3, 16, -1):
        with pytest.raises(m.MdeosError):
            m.Server(h, cluster=bad)


def test_requests_complete_before_their_launch_ends(m, h):
    """Results are reported per box: small boxes sharing a launch with one large box
    are seen long before it finishes."""
    big = dict(rho=0.8, e=1.5, natoms=32000, steps_equil=500, steps_avg=500, seed=1)
    small = [dict(rho=0.8, e=1.5, natoms=256, steps_equil=50, steps_avg=50, seed=2 + k)
             for k in range(10)]
    with m.Server(h, max_batch=64) as srv:
        ids = srv.enqueue([big] + small)
        got = srv.wait_all(11, timeout_s=300)
    t = {int(g["id"]): g["t_done"] for g in got}
    assert (got["result"]["status"] == 0).all()
    t_big = t[int(ids[0])]
    assert max(t[int(i)] for i in ids[1:]) < 0.5 * t_big


def test_queue_cap_and_wait_limit_shed(m, h):
    r = dict(rho=0.8, e=1.5, natoms=256, steps_equil=50, steps_avg=50, seed=5)
    with m.Server(h, max_batch=4, max_queue=5) as srv:
        srv.enqueue([dict(r, seed=s) for s in range(20)])
        got = srv.wait_all(20, timeout_s=120)
    st = got["result"]["status"]
    assert (st == m.MDEOS_ECANCELLED).sum() == 15 and (st == 0).sum() == 5
    long = dict(rho=0.8, e=1.5, natoms=20000, steps_equil=400, steps_avg=400, seed=6)
    with m.Server(h, max_inflight=1, max_batch=4, max_wait_s=0.05) as srv:
        srv.enqueue([long])
        time.sleep(0.2)                      # the only in-flight slot holds the long box
        srv.enqueue([dict(r, seed=s) for s in range(6)])
        got = srv.wait_all(7, timeout_s=300)
    st = got["result"]["status"]
    assert (st == m.MDEOS_ECANCELLED).sum() == 6 and (st == 0).sum() == 1


def test_hbm_budget_and_inflight_cap(m, h):
    with pytest.raises(m.MdeosError) as ei:                # per-SM scratch does not fit
        m.Server(h, hbm_budget_bytes=1 << 20)
    assert ei.value.status == m.MDEOS_ENOMEM
    r = dict(rho=0.8, e=1.5, natoms=256, steps_equil=40, steps_avg=40, seed=7)
    with m.Server(h, max_inflight=3, max_batch=2, hbm_budget_bytes=60 << 30) as srv:
        srv.enqueue([dict(r, seed=s, natoms=n) for s, n in
                     enumerate([256, 500, 9000, 256, 4000, 12000, 864, 256])])
        got = srv.wait_all(8, timeout_s=300)
        st = srv.stats()
    assert (got["result"]["status"] == 0).all()
    assert st["peak_inflight"] <= 3 and 0 < st["device_bytes"] <= 60 << 30


def test_idle_exit_and_relaunch(m, h):
    """The server kernel leaves the GPU when idle and comes back for new work."""
    r = dict(rho=0.8, e=1.5, natoms=256, steps_equil=40, steps_avg=40, seed=9)
    with m.Server(h, idle_ms=5) as srv:
        srv.enqueue([r])
        a = srv.wait_all(1, timeout_s=60)
        time.sleep(0.2)                      # idle well past 5 ms: the grid exits
        srv.enqueue([dict(r, seed=10)])
        b = srv.wait_all(1, timeout_s=60)
        st = srv.stats()
    assert a["result"]["status"][0] == 0 and b["result"]["status"][0] == 0
    assert st["launches"] >= 2


def _element_requests(m, sizes, seed, round_k):
    """One request per element (element_id k + 1) for a hydro-like step; each round
    moves every element's density a little, as a Lagrangian mesh does."""
    rng = np.random.default_rng(seed)
    out = []
    for k, n in enumerate(sizes):
        rho = 0.8 + 0.01 * round_k + 0.05 * rng.uniform()
        out.append(dict(rho=rho, e=m.e_from_temperature(1.4, n), natoms=n, steps_equil=100,
                        steps_avg=100, seed=1000 + 31 * k + round_k, element_id=k + 1))
    return out


def test_served_warm_starts_equal_the_handle_store(m):
    """Element states kept by the server give the same warm-started results, bit for
    bit, as the handle's own warm store fed the same requests."""
    sizes = [256, 500, 864, 1372, 2048, 4000, 300, 1111]
    rounds = [_element_requests(m, sizes, 5, k) for k in range(3)]
    hs = m.mdeos_create()
    served = []
    try:
        with m.Server(hs, warm=1) as srv:
            for reqs in rounds:   # one hydro step after the other
                ids = srv.enqueue(reqs)
                got = srv.wait_all(len(reqs), timeout_s=300)
                by = {int(g["id"]): g["result"] for g in got}
                served.append(np.array([by[int(i)] for i in ids]))
            ss = srv.store_stats()
    finally:
        m.mdeos_destroy(hs)
    with m.Engine(warm_slots=64, warm_atoms=4096) as eng:
        ref = [eng.evaluate(reqs) for reqs in rounds]
    for k in range(3):
        assert (served[k]["status"] == 0).all(), served[k]["status"]
        assert (served[k]["warm"] == (0 if k == 0 else 1)).all(), (k, served[k]["warm"])
        assert served[k].tobytes() == ref[k].tobytes(), k
    assert ss["warm_starts"] == 2 * len(sizes) and ss["stored"] == len(sizes)


def test_admission_waits_for_element_store_memory(m):
    """A store with room for two 2048-atom elements and six such elements arriving
    at once: two run, the others wait and are admitted as results come back; at no
    time do more than two hold store memory.  A second round reuses or reclaims the
    blocks (least recently used first)."""
    per = (16 + 32 * 2048 + 255) // 256 * 256
    reqs = [dict(rho=0.8, e=m.e_from_temperature(1.3, 2048), natoms=2048, steps_equil=60,
                 steps_avg=60, seed=50 + k, element_id=100 + k) for k in range(6)]
    hs = m.mdeos_create()
    try:
        with m.Server(hs, warm=1, warm_bytes=2 * per) as srv:
            srv.enqueue(reqs)
            got = srv.wait_all(6, timeout_s=300)
            st, ss = srv.stats(), srv.store_stats()
            assert len(got) == 6 and (got["result"]["status"] == 0).all()
            assert st["peak_inflight"] <= 2, st
            assert ss["memory_waits"] >= 4 and ss["evictions"] >= 4, ss
            assert ss["store_bytes"] == 2 * per and ss["stored"] == 2
            srv.enqueue(reqs[4:])          # the two most recent elements: still stored
            got2 = srv.wait_all(2, timeout_s=300)
            assert (got2["result"]["warm"] == 1).all()
    finally:
        m.mdeos_destroy(hs)
