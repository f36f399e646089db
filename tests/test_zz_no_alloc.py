"""The entry point that allocates no device memory (mdeos_submit_noalloc).

It serves callers that cannot allocate device memory where they need an EOS answer,
such as a hydrocode's material-model callback inside its time step.  Its scratch
lives in a static device array shared by every call, so this test calls it twice in
a row (the second call must not see the first call's leftovers) and compares both
with the ordinary submit/poll entry point.  This file is collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _requests(m):
    from paper_2508_06012_gb300 import workloads as w
    boxes = w.random_boxes(17, 40, 60, 4096, steps_equil=80, steps_avg=80)
    reqs = [dict(rho=b["rho"], e=m.e_from_temperature(b["T"], b["natoms"]), natoms=b["natoms"],
                 steps_equil=b["steps_equil"], steps_avg=b["steps_avg"], seed=b["seed"],
                 element_id=100 + k) for k, b in enumerate(boxes)]
    reqs.append(dict(rho=0.8, e=2.0, natoms=1, steps_equil=40, steps_avg=40, seed=1))  # rejected
    return reqs


def _same(a, b):
    for f in ("status", "natoms", "path", "nlist_builds", "element_id"):
        assert np.array_equal(a[f], b[f]), f
    for f in ("P", "T", "sigma", "epot", "ekin", "e_achieved", "P_se", "T_se", "T_target",
              "e_cold", "L", "pairs_per_step", "cand_per_step"):
        assert np.allclose(a[f], b[f], rtol=1e-12, atol=0.0), f


def test_noalloc_matches_submit_on_two_calls_in_a_row():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2508_06012_gb300 as m
    m.build()
    reqs = _requests(m)
    n = len(reqs)
    with m.Engine() as eng:
        ref = eng.evaluate(reqs)
    assert (ref["status"][:-1] == 0).all() and ref["status"][-1] == m.MDEOS_EINVAL
    torch.cuda.set_device(0)
    out = torch.zeros(n * m.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    free = []
    for call in range(2):
        out.fill_(0xFF)  # stale bytes the call must overwrite
        torch.cuda.synchronize()
        free_before, _ = torch.cuda.mem_get_info()
        alloc_before = torch.cuda.memory_allocated()
        m.mdeos_submit_noalloc(reqs, out.data_ptr(), m.mdeos_config_default(device=0))
        torch.cuda.synchronize()
        free.append(free_before - torch.cuda.mem_get_info()[0])
        assert torch.cuda.memory_allocated() == alloc_before
        got = np.frombuffer(out.cpu().numpy().tobytes(), dtype=m.RESULT_DTYPE)
        _same(got, ref)
    # The first call may load the module's code and static array onto the device;
    # after it, a call takes no device memory at all (slack for the driver's own
    # bookkeeping, far below one CTA's 0.7 MB of Verlet lists).
    assert free[1] <= (1 << 20), free


def test_noalloc_refuses_a_capturing_stream():
    """Its host tables are freed on return, so a graph recording the copies would
    replay from freed memory: the call is refused while the stream is captured."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2508_06012_gb300 as m
    m.build()
    torch.cuda.set_device(0)
    reqs = _requests(m)[:2]
    out = torch.zeros(len(reqs) * m.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    m.mdeos_submit_noalloc(reqs, out.data_ptr(), m.mdeos_config_default(device=0))  # set-up call
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    x = torch.zeros(4, device="cuda")
    err = None
    with torch.cuda.stream(s):
        g.capture_begin()
        x.add_(1.0)
        try:
            m.mdeos_submit_noalloc(reqs, out.data_ptr(), m.mdeos_config_default(device=0),
                                   stream=s.cuda_stream)
        except m.MdeosError as exc:
            err = exc
        g.capture_end()
    assert err is not None and "capturing" in str(err)
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
