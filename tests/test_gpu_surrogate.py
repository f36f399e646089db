"""GPU tests of the surrogate EOS (mdeos_surrogate_*) against the FP64 surrogate oracle
(oracle/surrogate.py): the tensor-core GEMM, the forward pass, the gradients and the
Adam step on identical parameters and batches, and the disagreement gate.

Tolerances: GEMM results within the FP32 accumulation bound K * 2^-23 * sum|a b|.
Forward and gradients: the oracle applies the same bfloat16 roundings in FP64; where
an FP32 value and its FP64 counterpart straddle a bfloat16 rounding boundary the two
round one ulp apart, so the comparison bounds the mean and the worst difference and
requires the GPU to sit much closer to the bfloat16 oracle than the bfloat16 oracle
sits to the plain FP64 network.
"""
import numpy as np
import pytest

from oracle import surrogate as S

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


def _bits(a):
    import torch
    u = S.bf16(a).astype(np.float32).view(np.uint32) >> 16
    return torch.from_numpy(u.astype(np.uint16).view(np.int16).copy()).cuda()


# (128, 128, 1024) and (100, 128, 1000) run with K split over several CTAs (few tiles,
# long K), the second with a last split that ends inside a staged chunk
@pytest.mark.parametrize("M,N,K,ta,tb", [(1, 1, 1, 0, 0), (64, 64, 32, 0, 1), (100, 70, 45, 1, 0),
                                         (128, 128, 1024, 1, 0), (257, 128, 128, 0, 1),
                                         (100, 128, 1000, 1, 1)])
def test_tensor_core_gemm(m, M, N, K, ta, tb):
    rng = np.random.default_rng(M + N + K)
    A = S.bf16(rng.standard_normal((M, K)))
    B = S.bf16(rng.standard_normal((K, N)))
    Ast = A.T.copy() if ta else A          # stored transposed: A(m, k) = Ast[k, m]
    Bst = B.T.copy() if tb else B          # stored transposed: B(k, n) = Bst[n, k]
    sa = (1, M) if ta else (K, 1)
    sb = (1, K) if tb else (N, 1)
    C = m.mdeos_debug_gemm_bf16(_bits(Ast.ravel()), _bits(Bst.ravel()), M, N, K, sa, sb, (N, 1))
    C = C.cpu().numpy()[:M * N].reshape(M, N).astype(np.float64)
    ref = A @ B
    bound = K * 2.0 ** -23 * (np.abs(A) @ np.abs(B)) + 1e-30
    assert (np.abs(C - ref) <= bound).all()


def test_split_k_gemm_is_reproducible(m):
    """The partial tiles of a split K are summed in a fixed order: the same product
    twice gives the same bytes."""
    rng = np.random.default_rng(7)
    M, N, K = 128, 128, 2048
    A = S.bf16(rng.standard_normal((K, M)))   # stored transposed, as the weight gradients
    B = S.bf16(rng.standard_normal((K, N)))
    c1 = m.mdeos_debug_gemm_bf16(_bits(A.ravel()), _bits(B.ravel()), M, N, K, (1, M), (N, 1), (N, 1))
    c2 = m.mdeos_debug_gemm_bf16(_bits(A.ravel()), _bits(B.ravel()), M, N, K, (1, M), (N, 1), (N, 1))
    assert c1.cpu().numpy().tobytes() == c2.cpu().numpy().tobytes()
    ref = A.T @ B
    bound = K * 2.0 ** -23 * (np.abs(A.T) @ np.abs(B)) + 1e-30
    assert (np.abs(c1.cpu().numpy()[:M * N].reshape(M, N) - ref) <= bound).all()


def test_hidden_layer_tanh_error_bound(m):
    """The kernels' own tanh (exp2 form, odd series below 1/4) against the exact tanh:
    relative error below 2e-6 on a dense grid, across the branch point, for tiny and
    huge arguments; saturation and NaN propagation."""
    import torch
    g = np.linspace(-12.0, 12.0, 400001)
    tiny = 10.0 ** np.linspace(-30, -1, 2001)
    edge = np.array([0.25, np.nextafter(np.float32(0.25), np.float32(0)), 0.2499, 0.2501,
                     44.0, 88.0, 1e30, 0.0])
    x = np.concatenate([g, tiny, -tiny, edge, -edge]).astype(np.float32)
    y = m.mdeos_debug_tanh(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    ref = np.tanh(x.astype(np.float64))
    nz = np.abs(ref) > 1e-36
    rel = np.abs(y[nz] - ref[nz]) / np.abs(ref[nz])
    assert rel.max() < 2e-6, float(rel.max())
    assert (y[np.abs(x) >= 44.0] == np.sign(x[np.abs(x) >= 44.0])).all()
    yn = m.mdeos_debug_tanh(torch.tensor([float("nan")], device="cuda")).cpu().numpy()
    assert np.isnan(yn).all()


def _params(seed, E=4):
    rng = np.random.default_rng(seed)
    p = S.init_params(seed, E)
    for e in range(E):   # non-zero biases so every term of the forward pass matters
        d = S.unpack(p[e])
        for name in ("b1", "b2", "b3", "b4"):
            d[name] = 0.1 * rng.standard_normal(d[name].shape)
        p[e] = S.pack(d)
    return p.astype(np.float32).astype(np.float64)


NORM = np.array([0.75, -1.0, 0.25, 2.0, 1.5, 1.2, 2.0, 0.6])


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0.3, 1.2, n), rng.uniform(-5.0, 3.0, n)], axis=1)


@pytest.mark.parametrize("path", [0, 1], ids=["tcgen05", "mma"])
def test_forward_matches_oracle(m, h, path):
    """1000 inputs in chunks of 512: several 128-row tiles and a ragged tail."""
    p = _params(11)
    x = _inputs(1000, 12)
    with m.Surrogate(h, 4, 512, seed=1) as sg:
        sg.set_params(p, NORM)
        sg.set_infer_path(path)
        mean, sd, pm = sg.predict(x, per_model=True)
    xn = (x - NORM[:2]) / NORM[2:4]
    ref16 = np.array([S.forward(p[e], xn)[0] for e in range(4)])
    ref64 = np.array([S.forward(p[e], xn, bf16_mode=False)[0] for e in range(4)])
    d = np.abs(pm - ref16)
    assert d.max() <= 2e-2 and d.mean() <= 2e-4, (d.max(), d.mean())
    assert d.mean() < 0.1 * np.abs(ref16 - ref64).mean()
    phys = ref16 * NORM[6:8] + NORM[4:6]
    assert np.allclose(mean, phys.mean(axis=0), atol=5e-2)
    assert np.allclose(sd, phys.std(axis=0), atol=5e-2)


@pytest.mark.parametrize("E,n,maxb", [(1, 1, 64), (16, 129, 128), (3, 127, 4096), (4, 777, 300)])
def test_tensor_core_path_matches_layered_path(m, h, E, n, maxb):
    """The fused tcgen05 kernel against the layered mma.sync path on the same weights:
    the same bf16 roundings, another FP32 summation order, so outputs agree to FP32
    rounding except where a hidden unit rounds one bf16 ulp apart."""
    p = _params(51, E)
    x = _inputs(n, 52)
    out = {}
    with m.Surrogate(h, E, maxb, seed=1) as sg:
        sg.set_params(p, NORM)
        for path in (m.SURROGATE_INFER_TC, m.SURROGATE_INFER_MMA):
            sg.set_infer_path(path)
            out[path] = sg.predict(x, per_model=True)
        with pytest.raises(m.MdeosError):
            sg.set_infer_path(2)
    a, b = out[m.SURROGATE_INFER_TC][2], out[m.SURROGATE_INFER_MMA][2]
    assert np.isfinite(a).all() and a.shape == (E, n, 2)
    d = np.abs(a.astype(np.float64) - b)
    assert d.max() <= 2e-2 and d.mean() <= 1e-4, (d.max(), d.mean())
    assert np.median(d) <= 1e-5


def test_device_inference_equals_host_prediction(m, h):
    import torch
    p = _params(61)
    x = _inputs(5000, 62)
    with m.Surrogate(h, 4, 2048, seed=1) as sg:
        sg.set_params(p, NORM)
        mean, sd = sg.predict(x)
        xd = torch.from_numpy(x).cuda()
        md = torch.zeros_like(xd)
        sdd = torch.zeros_like(xd)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            sg.infer_device(xd, md, sdd, stream=st)
        st.synchronize()
        sg.infer_device(xd[:0], md[:0], sdd[:0])          # empty input
    assert md.cpu().numpy().tobytes() == mean.tobytes()
    assert sdd.cpu().numpy().tobytes() == sd.tobytes()


def test_gradients_match_oracle(m, h):
    p = _params(21)
    x = _inputs(300, 22)
    y = np.stack([x[:, 0] * (x[:, 1] + 3.0), 0.5 * x[:, 1] + 2.0], axis=1)
    with m.Surrogate(h, 4, 512, seed=1) as sg:
        sg.set_params(p, NORM)
        g, loss = sg.grads(x, y)
    xn = (x - NORM[:2]) / NORM[2:4]
    yn = (y - NORM[4:6]) / NORM[6:8]
    losses = []
    for e in range(4):
        l16, g16 = S.loss_and_grad(p[e], xn, yn)
        _, g64 = S.loss_and_grad(p[e], xn, yn, bf16_mode=False)
        losses.append(l16)
        dg = np.linalg.norm(g[e] - g16)
        assert dg <= 2e-2 * np.linalg.norm(g16), (e, dg / np.linalg.norm(g16))
        assert dg <= 0.5 * np.linalg.norm(g16 - g64)
    assert loss == pytest.approx(np.mean(losses), rel=1e-4)


def test_adam_step_matches_oracle(m, h):
    p = _params(31, 2)
    x = _inputs(256, 32)
    y = np.stack([x[:, 0] ** 2, x[:, 1]], axis=1)
    with m.Surrogate(h, 2, 256, seed=1) as sg:
        sg.set_params(p, NORM)
        g, _ = sg.grads(x, y)
        sg.train(x, y, epochs=1, batch=256, lr=1e-3, set_norm=False)   # one step, same batch
        p1, _ = sg.get_params()
    for e in range(2):
        ge = g[e].astype(np.float64)
        ref, _, _ = S.adam_step(p[e], ge, np.zeros(S.NPARAM), np.zeros(S.NPARAM), 1, lr=1e-3)
        # first step = lr g / (|g| + eps): where |g| is far above eps it does not depend on
        # the batch summation order (the training step sums in another order)
        big = np.abs(ge) > 1e-6
        assert big.mean() > 0.9
        assert np.abs(p1[e] - ref)[big].max() <= 2e-7
        assert np.abs(p1[e] - p[e]).max() <= 1e-3 * (1 + 1e-5)   # first step: at most lr


def test_training_fit_and_disagreement_gate(m, h):
    """A smooth EOS-like map is learned; off the training domain the members disagree
    and the gate sends those requests to MD."""
    rng = np.random.default_rng(41)
    n = 8192
    x = _inputs(n, 42)
    y = np.stack([x[:, 0] * (2.0 / 3.0) * (x[:, 1] + 6.0) - x[:, 0] ** 2,
                  (x[:, 1] + 6.0) / 1.5 - x[:, 0]], axis=1)
    with m.Surrogate(h, 4, 1024, seed=5) as sg:
        losses = sg.train(x, y, epochs=30, batch=512, lr=2e-3, seed=3)
        assert losses[-1] < 0.01 * losses[0], losses[[0, -1]]
        xin = _inputs(500, 43)
        yin = np.stack([xin[:, 0] * (2.0 / 3.0) * (xin[:, 1] + 6.0) - xin[:, 0] ** 2,
                        (xin[:, 1] + 6.0) / 1.5 - xin[:, 0]], axis=1)
        mean, sd = sg.predict(xin)
        assert np.abs(mean - yin).mean() < 0.05
        xout = np.stack([rng.uniform(4.0, 6.0, 200), rng.uniform(20.0, 40.0, 200)], axis=1)
        _, sd_out = sg.predict(xout)
        assert np.median(sd_out[:, 0]) > 10 * np.median(sd[:, 0])
        thr = float(np.percentile(sd[:, 0] / np.maximum(np.abs(mean[:, 0]), 1.0), 99))
        reqs = [dict(rho=float(r), e=float(e), natoms=108, steps_equil=20, steps_avg=20, seed=k)
                for k, (r, e) in enumerate(xin[:20])]
        reqs += [dict(rho=1.0, e=50.0, natoms=108, steps_equil=20, steps_avg=20, seed=99)]
        out, used = sg.gated_eval(reqs, thr)
    assert used[-1] == 1 and out["path"][-1] >= 0            # off-domain: MD
    assert (used[:20] == 0).sum() >= 15                       # in-domain: mostly surrogate
    assert (out["path"][:20][used[:20] == 0] == -2).all()


def test_trained_network_gains_over_md_only(m, h):
    """What the learned part gains: an ensemble trained on MD answers of this library
    (256-atom boxes, a liquid (rho, T) domain), its gate tuned on validation MD, then
    test queries answered by the gated path against MD for every query.  The gated
    path must answer most queries from the network, with the accepted answers'
    pressure error no larger than the target the gate was tuned for (vs MD), and so
    run that many fewer MD boxes; MD-only runs one box per query.

    A run lifted to the energy e samples e_achieved, within ~T sqrt(3 / 2N) of e (the
    lifting's last rescale happens at one instant), so an MD answer is the pressure at
    e_achieved: the network is trained on (rho, e_achieved) and its error is measured
    at the state each reference run sampled, which is what the gate is tuned on.  The
    domain is the single-phase fluid (above the critical temperature, below the
    freezing density): past the freezing line a box lifted from the FCC lattice can stay
    crystalline, and the MD answers then jump between branches."""
    def reqs(n, seed):
        r = np.random.default_rng(seed)
        rho, T = r.uniform(0.5, 0.9, n), r.uniform(1.3, 2.8, n)
        return [dict(rho=float(rho[k]), e=m.e_from_temperature(float(T[k]), 256), natoms=256,
                     steps_equil=300, steps_avg=600, seed=int(seed * 100000 + k)) for k in range(n)]

    def sampled(qs, res):
        return np.stack([np.array([q["rho"] for q in qs]), res["e_achieved"]], axis=1)

    train, val, test = reqs(4000, 1), reqs(400, 2), reqs(400, 3)
    with m.Engine() as eng:
        rt, rv, rtest = eng.evaluate(train), eng.evaluate(val), eng.evaluate(test)
    assert (rt["status"] == 0).mean() > 0.99
    assert (rv["status"] == 0).all() and (rtest["status"] == 0).all()
    ok = rt["status"] == 0
    x = sampled(train, rt)[ok]
    y = np.stack([rt["P"], rt["T"]], axis=1)[ok]
    target = 0.03  # 256-atom, 600-step MD answers scatter by ~1.5 % themselves
    with m.Surrogate(h, 4, 1024, seed=3) as sg:
        sg.set_output_transform(m.SURROGATE_P_ASINH)
        sg.train(x, y, epochs=150, batch=256, lr=2e-3, seed=4)
        sg.train(x, y, epochs=100, batch=256, lr=3e-4, seed=5, set_norm=False)
        # gate threshold: the largest spread level whose accepted validation queries
        # meet the target (RMS of |dP| / max(|P|, 1) against MD)
        mv, sv = sg.predict(sampled(val, rv))
        err = np.abs(mv[:, 0] - rv["P"]) / np.maximum(np.abs(rv["P"]), 1.0)
        dis = sv[:, 0] / np.maximum(np.abs(mv[:, 0]), 1.0)
        order = np.argsort(dis)
        rms = np.sqrt(np.cumsum(err[order] ** 2) / np.arange(1, len(order) + 1))
        k = int(np.flatnonzero(rms <= target)[-1])
        thr = float(dis[order][k])
        out, used = sg.gated_eval(test, thr)
        mt, _ = sg.predict(sampled(test, rtest))
    answered = used == 0
    e_test = np.abs(mt[:, 0] - rtest["P"]) / np.maximum(np.abs(rtest["P"]), 1.0)
    print(f"gate: threshold {thr:.4f}, answers {answered.mean():.1%} of test queries, "
          f"RMS error {np.sqrt(np.mean(e_test[answered] ** 2)):.4f} (all queries "
          f"{np.sqrt(np.mean(e_test ** 2)):.4f})")
    assert answered.mean() >= 0.5
    assert np.sqrt(np.mean(e_test[answered] ** 2)) <= 1.5 * target
    assert (out["status"] == 0).all()
    assert (out["path"][answered] == -2).all() and (out["path"][~answered] >= 0).all()
    # an MD-answered query is the same run as the reference (same request, same seed)
    assert np.array_equal(out["P"][~answered], rtest["P"][~answered])
    # MD boxes run: the gated path's MD share against one per query without it
    assert int((~answered).sum()) <= len(test) // 2


def test_misfit_map_flags_a_rough_region(m, h):
    """The misfit map holds the RMS relative residual of the ensemble mean per cell of
    its training inputs: where the data are rough (here: noise added for rho > 0.8)
    every member misses them alike, the map is high there, and the gate with a misfit
    threshold sends such requests to MD while it still answers the smooth region."""
    rng = np.random.default_rng(3)
    n = 8192
    x = np.stack([rng.uniform(0.5, 1.0, n), rng.uniform(1.0, 3.0, n)], axis=1)
    P = 2.0 * x[:, 0] * x[:, 1] + x[:, 0] ** 2
    rough = x[:, 0] > 0.8
    Pn = P * (1.0 + np.where(rough, 0.1, 0.0) * rng.normal(size=n))
    y = np.stack([Pn, x[:, 1] / 1.5], axis=1)
    with m.Surrogate(h, 4, 2048, seed=5) as sg:
        sg.train(x, y, epochs=40, batch=512, lr=2e-3, seed=3)
        sg.fit_misfit(x, y, bins=10, min_count=8)
        xs = np.stack([np.full(50, 0.6), np.linspace(1.2, 2.8, 50)], axis=1)
        xr = np.stack([np.full(50, 0.95), np.linspace(1.2, 2.8, 50)], axis=1)
        ms, mr = sg.misfit(xs), sg.misfit(xr)
        assert np.isfinite(ms).all() and np.isfinite(mr).all()
        assert np.median(mr) > 0.05 > 0.02 > np.median(ms), (np.median(ms), np.median(mr))
        assert np.isinf(sg.misfit(np.array([[0.3, 2.0], [0.7, 5.0]]))).all()  # outside the map
        reqs = [dict(rho=float(r), e=float(e), natoms=108, steps_equil=20, steps_avg=20, seed=k)
                for k, (r, e) in enumerate(np.concatenate([xs[::10], xr[::10]]))]
        sg.set_misfit_threshold(0.03)
        out, used = sg.gated_eval(reqs, 1e9)  # the spread alone would answer everything
        assert (used[:5] == 0).all() and (used[5:] == 1).all(), used
        assert (out["path"][5:] >= 0).all() and (out["status"] == 0).all()
        sg.set_misfit_threshold(float("inf"))
        _, used = sg.gated_eval(reqs, 1e9)
        assert (used == 0).all()
