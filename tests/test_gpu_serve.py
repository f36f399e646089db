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
            for b in w.config4(seed, k, steps[0], steps[1])]


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
