"""Serving (fsg_server_*): requests of different n, d (2, 10, 64) and L run
concurrently on the server's slots; every result must equal the same request
run alone through fsg_build_graph_host, whatever the mix, the admission
order or the HBM budget.  Host-side failures (an injected allocation failure,
a cancelled request, malformed or oversized requests) release their slot and
budget and leave the other results unchanged."""
import time

import numpy as np
import pytest

from paper_2310_13870_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_13870_gb300 import fsg as _fsg
    import os
    if not os.path.exists(_fsg.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    _fsg.load()
    return _fsg


def _requests():
    rng = np.random.default_rng(0)
    reqs = []
    for k in range(10):
        d = [2, 10, 64][k % 3]
        n = int(rng.integers(300, 4000))
        X = inputs.gaussian_mixture(n=n, d=d, k=4, box=4.0, seed=100 + k)
        reqs.append((X, 1.5 if d > 2 else 0.3, int(rng.choice([8, 16, 32])), 500 + k))
    return reqs


def _params(fsg, X, sigma, split):
    if split and X.shape[1] > 16:  # d = 64 requests in split precision (approximate KDE too for "approx")
        return fsg.params(sigma, precision=fsg.FSG_PREC_SPLIT_BF16, kde_eps=1e-3 if split == "approx" else 0.0)
    return fsg.params(sigma)


def _alone(fsg, X, sigma, L, seed, split=False):
    src, dst, w = fsg.fsg_build_graph_host(X, _params(fsg, X, sigma, split), L, seed)
    return src.copy(), dst.copy(), w.copy()


def _drain(server, expect, timeout_s=120):
    got = {}
    t0 = time.time()
    while len(got) < expect and time.time() - t0 < timeout_s:
        for rec, arrays in server.poll(wait_ms=100):
            got[rec["id"]] = (rec, arrays)
    assert len(got) == expect
    return got


@pytest.mark.parametrize("budget_mb,slots,admission,split", [(8192, 8, 0, False), (64, 2, 0, False),
                                                           (8192, 8, 1, False), (64, 1, 1, False), (8192, 8, 0, True),
                                                           (8192, 8, 0, "approx")])
def test_results_equal_alone_in_the_mix(fsg, budget_mb, slots, admission, split):
    reqs = _requests()
    want = [_alone(fsg, *r, split=split) for r in reqs]
    server = fsg.Server(hbm_budget_bytes=budget_mb << 20, max_slots=slots, admission=admission)
    ids = [server.submit(X, _params(fsg, X, s, split), L, seed) for X, s, L, seed in reqs]
    got = _drain(server, len(ids))
    for rid, (src, dst, w) in zip(ids, want):
        rec, (gs, gd, gw) = got[rid]
        assert rec["status"] == fsg.FSG_OK
        assert rec["latency_ms"] >= rec["queue_ms"] >= 0.0
        np.testing.assert_array_equal(gs, src)
        np.testing.assert_array_equal(gd, dst)
        np.testing.assert_array_equal(gw, w)
    assert server.info() == {"pending": 0, "in_flight": 0, "bytes_in_use": 0}
    server.close()


def test_in_mix_results_match_the_oracle(fsg):
    # Results taken from the mix (eight slots, all requests in flight together)
    # against the FP64 oracle's Algorithm 2 directly, for one request of each
    # d: a flagged sample may move one edge, so the edge sets differ in at
    # most two pairs per flagged sample; every edge both have carries the
    # oracle's weight (Eq. 2, which pins both endpoints' degrees) within 1e-4.
    import math
    import oracle as ora
    reqs = _requests()
    server = fsg.Server(hbm_budget_bytes=8192 << 20, max_slots=8)
    ids = [server.submit(X, fsg.params(s), L, seed) for X, s, L, seed in reqs]
    got = _drain(server, len(ids))
    server.close()
    checked = set()
    for k in sorted(range(len(reqs)), key=lambda k: reqs[k][0].shape[0]):
        X, sigma, L, seed = reqs[k]
        if X.shape[1] in checked:
            continue
        checked.add(X.shape[1])
        rec, (gs, gd, gw) = got[ids[k]]
        assert rec["status"] == fsg.FSG_OK
        o = ora.build_graph(X, ora.gamma(sigma), L, seed)
        eg = {(min(a, b), max(a, b)): w for a, b, w in zip(gs.tolist(), gd.tolist(), gw.tolist())}
        eo = {(min(a, b), max(a, b)): w for a, b, w in zip(o["src"].tolist(), o["dst"].tolist(), o["w"].tolist())}
        assert len(eg) == len(gs)  # SET: no pair twice
        assert len(set(eg) ^ set(eo)) <= 2 * rec["n_flagged"], (X.shape, rec["n_flagged"])
        for key in set(eg) & set(eo):
            assert math.isclose(eg[key], eo[key], rel_tol=1e-4), (X.shape, key, eg[key], eo[key])
    assert checked == {2, 10, 64}


def test_response_ratio_lets_short_requests_overtake(fsg):
    # one slot: a long request (200k points) is admitted first, then three long
    # and three short requests queue behind it; by response ratio the short
    # ones run before the queued long ones, in arrival order after them.  Points
    # and outputs are pinned beforehand so that every submission is quick
    # next to the first request's run time.
    def pinned(a):
        return torch.from_numpy(a).pin_memory().numpy()

    first = pinned(inputs.gaussian_mixture(n=200_000, d=64, k=4, box=4.0, seed=6))
    big = pinned(inputs.gaussian_mixture(n=60_000, d=64, k=4, box=4.0, seed=7))
    small = pinned(inputs.gaussian_mixture(n=500, d=2, k=4, box=4.0, seed=8))
    L = 8
    outs = [tuple(pinned(np.empty(200_000 * L, dt)) for dt in (np.int32, np.int32, np.float32)) for _ in range(7)]
    order = {}
    for admission in (fsg.FSG_ADMIT_ARRIVAL, fsg.FSG_ADMIT_RESPONSE_RATIO):
        server = fsg.Server(hbm_budget_bytes=1 << 34, max_slots=1, admission=admission)
        kinds, t_sub = {}, {}

        def submit(X, sigma, seed, kind):
            t = time.perf_counter()
            rid = server.submit(X, fsg.params(sigma), L, seed, out=outs[len(kinds)])
            kinds[rid], t_sub[rid] = kind, t

        submit(first, 1.5, 0, "long")
        t0 = time.time()
        while server.info()["pending"] and time.time() - t0 < 10:
            time.sleep(0.0002)
        for k in range(3):
            submit(big, 1.5, 1 + k, "long")
        for k in range(3):
            submit(small, 0.3, 10 + k, "short")
        got = _drain(server, 7, timeout_s=300)
        assert all(rec["status"] == fsg.FSG_OK for rec, _ in got.values())
        admitted = sorted(got, key=lambda rid: t_sub[rid] + got[rid][0]["queue_ms"] * 1e-3)
        order[admission] = [kinds[rid] for rid in admitted]
        server.close()
    assert order[fsg.FSG_ADMIT_ARRIVAL] == ["long"] * 4 + ["short"] * 3
    assert order[fsg.FSG_ADMIT_RESPONSE_RATIO] == ["long"] + ["short"] * 3 + ["long"] * 3


def test_injected_allocation_failure_and_cancellation(fsg):
    reqs = _requests()
    want = [_alone(fsg, *r) for r in reqs]
    # every 3rd admission fails on the host as if its allocation had failed
    server = fsg.Server(hbm_budget_bytes=1 << 33, max_slots=1, inject_alloc_fail_every=3)
    ids = [server.submit(X, fsg.params(s), L, seed) for X, s, L, seed in reqs]
    server.cancel(ids[-1])
    got = _drain(server, len(ids))
    statuses = [got[i][0]["status"] for i in ids]
    assert statuses.count(fsg.FSG_ERR_OOM) >= 2
    assert statuses[-1] in (fsg.FSG_ERR_CANCELLED, fsg.FSG_ERR_OOM)
    for rid, (src, dst, w) in zip(ids, want):
        rec, arrays = got[rid]
        if rec["status"] == fsg.FSG_OK:
            np.testing.assert_array_equal(arrays[0], src)
            np.testing.assert_array_equal(arrays[2], w)
    assert server.info()["bytes_in_use"] == 0
    server.close()


def test_malformed_and_oversized_requests_are_refused(fsg):
    server = fsg.Server(hbm_budget_bytes=1 << 20, max_slots=2)
    X = inputs.gaussian_mixture(n=50_000, d=10, seed=1)
    with pytest.raises(fsg.FsgError) as e:
        server.submit(X, fsg.params(1.5), 32, 0)  # needs far more than 1 MiB
    assert e.value.status == fsg.FSG_ERR_BUSY
    with pytest.raises(fsg.FsgError) as e:
        server.submit(X[:10], fsg.params(-1.0), 8, 0)
    assert e.value.status == fsg.FSG_ERR_INVALID_ARG
    with pytest.raises(fsg.FsgError) as e:
        server.submit(X[:10], fsg.params(1.0), 65, 0)
    assert e.value.status == fsg.FSG_ERR_INVALID_ARG
    server.close()


def test_server_and_direct_calls_run_concurrently(fsg):
    # The server's worker thread launches kernels while this thread makes
    # direct calls on its own trees (the launchers' per-device shared-memory
    # limits are set under a lock, once per kernel and device): every result
    # equals the same work run alone.
    import threading
    reqs = _requests()
    want = [_alone(fsg, *r) for r in reqs]
    X = inputs.gaussian_mixture(n=30_000, d=12, seed=77)
    pts = torch.from_numpy(X).cuda()
    tree = fsg.fsg_build_tree(pts)
    ref = fsg.fsg_build_graph(tree, fsg.params(1.5), 32, 5)
    torch.cuda.synchronize()
    ref_w = ref.w[: int(ref.m.item())].cpu().numpy().copy()
    server = fsg.Server(hbm_budget_bytes=8192 << 20, max_slots=8)
    ids = [server.submit(Xr, fsg.params(s), L, seed) for Xr, s, L, seed in reqs]
    errors = []

    def direct():
        try:
            with torch.cuda.stream(torch.cuda.Stream()):
                for _ in range(5):
                    b = fsg.fsg_build_graph(tree, fsg.params(1.5), 32, 5)
                    torch.cuda.current_stream().synchronize()
                    np.testing.assert_array_equal(b.w[: int(b.m.item())].cpu().numpy(), ref_w)
        except Exception as e:  # reported on the main thread
            errors.append(e)

    th = threading.Thread(target=direct)
    th.start()
    got = _drain(server, len(ids))
    th.join()
    server.close()
    tree.close()
    assert not errors, errors
    for rid, (src, dst, w) in zip(ids, want):
        rec, (gs, gd, gw) = got[rid]
        assert rec["status"] == fsg.FSG_OK
        np.testing.assert_array_equal(gs, src)
        np.testing.assert_array_equal(gw, w)
