"""Continuous-batching server through the C ABI: every result matches the oracle's residual
bar, a request gives bit-identical x alone and in a mix of concurrent solves, admission never
exceeds the memory budget, and requests that can never fit are refused."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_12371_gb300 import capi, meshgen, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    capi.load()
    torch.cuda.init()


def requests(sizes, seed0=0):
    out = []
    for i, cells in enumerate(sizes):
        m, b = workloads.serving_request(seed0 + i, cells)
        out.append((m, b))
    return out


def wait_all(srv, tickets, ms, timeout=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets):
        for t, m in zip(tickets, ms):
            if t in res:
                continue
            x = np.empty(m.n)
            r = capi.spmv_server_poll(srv, t, x)
            if r is not None:
                res[t] = (x, r)
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.001)
    return [res[t] for t in tickets]


def relres(oracle, m, x, b):
    return np.linalg.norm(b - oracle.spmv(m.row_ptr, m.col_idx, m.values, x)) / np.linalg.norm(b)


def test_alone_equals_in_mix(oracle):
    reqs = requests([2e4, 8e3, 5e4, 1.2e4, 3e4, 9e3, 4e4, 2.5e4], seed0=100)
    opts = [capi.cg_default_options(rtol=1e-8, mixed=(i % 2)) for i in range(len(reqs))]
    # alone: one slot, one request at a time
    alone = []
    srv = capi.spmv_server_create(8 << 30, 1)
    for (m, b), o in zip(reqs, opts):
        t = capi.spmv_server_submit(srv, m.n, m.row_ptr, m.col_idx, m.values, b, o)
        alone.append(wait_all(srv, [t], [m])[0])
    capi.spmv_server_destroy(srv)
    # in a mix: four slots, everything submitted at once
    srv = capi.spmv_server_create(8 << 30, 4)
    tickets = [capi.spmv_server_submit(srv, m.n, m.row_ptr, m.col_idx, m.values, b, o)
               for (m, b), o in zip(reqs, opts)]
    mixed = wait_all(srv, tickets, [m for m, _ in reqs])
    st = capi.spmv_server_get_stats(srv)
    capi.spmv_server_destroy(srv)
    assert st["completed"] == len(reqs) and st["rejected"] == 0
    assert st["p99_latency_s"] >= st["p50_latency_s"] > 0
    assert st["setup_s"] > 0 and st["solve_s"] > 0 and st["teardown_s"] > 0
    for (m, b), (xa, ra), (xm, rm) in zip(reqs, alone, mixed):
        assert ra["status"] == rm["status"] == capi.SPMV_OK
        assert np.array_equal(xa, xm)
        assert ra["iterations"] == rm["iterations"]
        assert relres(oracle, m, xm, b) <= 1e-8
    # the server launches the kernels directly; cg_solve replays them as CUDA graphs (and the
    # persistent kernel runs them in one launch): same kernels, same order, same bits
    for (m, b), o, (xa, ra) in list(zip(reqs, opts, alone))[:2]:
        A = capi.Matrix(m.n, m.row_ptr, m.col_idx, m.values,
                        precision=capi.SPMV_PREC_DUAL if o.mixed else capi.SPMV_PREC_FP64)
        bd = torch.from_numpy(b).cuda()
        for persistent in (0, 1):
            xd = torch.zeros_like(bd)
            o.persistent = persistent
            r = capi.cg_solve(A.handle, bd, xd, o)
            assert r["iterations"] == ra["iterations"]
            assert np.array_equal(xd.cpu().numpy(), xa)
        A.close()


def test_budget_admission_and_refusal():
    reqs = requests([3e4, 3e4, 3e4, 3e4], seed0=7)
    m0 = reqs[0][0]
    # a budget that holds one of these solves but not two
    est_one = 4 * (m0.n + 1) + 12 * m0.nnz
    budget = 60 * m0.nnz + 120 * m0.n + (6 << 20)
    srv = capi.spmv_server_create(budget, 4)
    tickets = [capi.spmv_server_submit(srv, m.n, m.row_ptr, m.col_idx, m.values, b)
               for m, b in reqs]
    max_active = 0
    t0 = time.time()
    done = {}
    while len(done) < len(tickets):
        st = capi.spmv_server_get_stats(srv)
        max_active = max(max_active, st["active_slots"])
        assert st["bytes_in_use"] <= budget
        for t, (m, b) in zip(tickets, reqs):
            if t not in done:
                r = capi.spmv_server_poll(srv, t, np.empty(m.n))
                if r is not None:
                    done[t] = r
        assert time.time() - t0 < 120
    st = capi.spmv_server_get_stats(srv)
    assert st["peak_bytes"] <= budget
    assert max_active <= 1
    assert all(r["status"] == capi.SPMV_OK for r in done.values())
    # a request that can never fit is refused at submit
    big, bb = requests([2e5], seed0=3)[0]
    with pytest.raises(capi.SpmvError) as e:
        capi.spmv_server_submit(srv, big.n, big.row_ptr, big.col_idx, big.values, bb)
    assert e.value.status == capi.SPMV_ERR_BUDGET
    assert capi.spmv_server_get_stats(srv)["rejected"] == 1
    # unknown ticket
    assert capi.load().spmv_server_poll(srv, 10 ** 9, None, None) == capi.SPMV_ERR_INVALID_ARG
    capi.spmv_server_destroy(srv)
    assert est_one > 0


def test_destroy_with_requests_in_flight():
    reqs = requests([5e4] * 6, seed0=40)
    srv = capi.spmv_server_create(8 << 30, 2)
    for m, b in reqs:
        capi.spmv_server_submit(srv, m.n, m.row_ptr, m.col_idx, m.values, b)
    capi.spmv_server_destroy(srv)  # joins the running solves, frees the queued ones
    torch.cuda.synchronize()


def test_cancel_queued_and_running(oracle):
    (big, bb), (small, sb), (late, lb) = requests([3e5, 2e4, 2e4], seed0=60)
    srv = capi.spmv_server_create(8 << 30, 1)
    # rtol 0: the big solve only ends by its (large) iteration cap, or by cancellation
    endless = capi.cg_default_options(rtol=0.0, max_iter=200000)
    ta = capi.spmv_server_submit(srv, big.n, big.row_ptr, big.col_idx, big.values, bb, endless)
    tb = capi.spmv_server_submit(srv, small.n, small.row_ptr, small.col_idx, small.values, sb)
    t0 = time.time()
    while capi.spmv_server_get_stats(srv)["active_slots"] < 1:
        assert time.time() - t0 < 60
        time.sleep(0.001)
    time.sleep(0.2)  # the big solve is in its iteration loop; the small one waits in the queue
    st = capi.spmv_server_get_stats(srv)
    assert st["active_slots"] == 1 and st["queued"] == 1
    capi.spmv_server_cancel(srv, tb)  # queued: done at once
    xb = np.full(small.n, np.nan)
    rb = capi.spmv_server_poll(srv, tb, xb)
    assert rb is not None and rb["status"] == capi.SPMV_ERR_CANCELLED
    assert np.isnan(xb).all()  # x left untouched
    capi.spmv_server_cancel(srv, ta)  # running: stops at its next convergence check
    t1 = time.time()
    xa = np.full(big.n, np.nan)
    while True:
        ra = capi.spmv_server_poll(srv, ta, xa)
        if ra is not None:
            break
        assert time.time() - t1 < 30, "cancelled solve did not stop"
        time.sleep(0.001)
    assert ra["status"] == capi.SPMV_ERR_CANCELLED
    assert np.isnan(xa).all()
    st = capi.spmv_server_get_stats(srv)
    assert st["cancelled"] == 2 and st["completed"] == 0 and st["active_slots"] == 0
    assert st["bytes_in_use"] == 0
    # polled tickets are gone; the server keeps serving
    for t in (ta, tb):
        with pytest.raises(capi.SpmvError) as e:
            capi.spmv_server_cancel(srv, t)
        assert e.value.status == capi.SPMV_ERR_INVALID_ARG
    tc = capi.spmv_server_submit(srv, late.n, late.row_ptr, late.col_idx, late.values, lb,
                                 capi.cg_default_options(rtol=1e-8))
    (xc, rc), = wait_all(srv, [tc], [late])
    assert rc["status"] == capi.SPMV_OK
    assert relres(oracle, late, xc, lb) <= 1e-8
    # cancelling a finished request that is not yet polled keeps its own status
    td = capi.spmv_server_submit(srv, late.n, late.row_ptr, late.col_idx, late.values, lb,
                                 capi.cg_default_options(rtol=1e-8))
    t0 = time.time()
    while capi.spmv_server_get_stats(srv)["completed"] < 2:
        assert time.time() - t0 < 60
        time.sleep(0.001)
    capi.spmv_server_cancel(srv, td)
    (xd, rd), = wait_all(srv, [td], [late])
    assert rd["status"] == capi.SPMV_OK and np.array_equal(xd, xc)
    capi.spmv_server_destroy(srv)


def test_bad_request_fails_alone(oracle):
    """A request whose CSR is malformed (unsorted columns) or has no diagonal entry reports
    INVALID_CSR; the requests around it, on the same slots, are solved as usual."""
    (m1, b1), (m2, b2) = requests([2e4, 3e4], seed0=80)
    bad_ci = m1.col_idx.copy()
    lo, hi = m1.row_ptr[5], m1.row_ptr[6]
    bad_ci[lo:hi] = bad_ci[lo:hi][::-1]  # row 5 unsorted
    rp = np.array([0, 1, 2], np.int32)   # 2x2 without diagonal
    srv = capi.spmv_server_create(8 << 30, 2)
    t_good1 = capi.spmv_server_submit(srv, m1.n, m1.row_ptr, m1.col_idx, m1.values, b1)
    t_bad = capi.spmv_server_submit(srv, m1.n, m1.row_ptr, bad_ci, m1.values, b1)
    t_nodiag = capi.spmv_server_submit(srv, 2, rp, np.array([1, 0], np.int32), np.ones(2),
                                       np.ones(2))
    t_good2 = capi.spmv_server_submit(srv, m2.n, m2.row_ptr, m2.col_idx, m2.values, b2)
    dummy = meshgen.CsrMatrix(2, rp, np.array([1, 0], np.int32), np.ones(2))
    res = wait_all(srv, [t_good1, t_bad, t_nodiag, t_good2], [m1, m1, dummy, m2])
    assert res[1][1]["status"] == capi.SPMV_ERR_INVALID_CSR
    assert res[2][1]["status"] == capi.SPMV_ERR_INVALID_CSR
    for (x, r), (m, b) in ((res[0], (m1, b1)), (res[3], (m2, b2))):
        assert r["status"] == capi.SPMV_OK
        assert relres(oracle, m, x, b) <= 1e-8
    st = capi.spmv_server_get_stats(srv)
    assert st["completed"] == 4 and st["bytes_in_use"] == 0
    capi.spmv_server_destroy(srv)


def test_small_request_passes_a_blocked_large_one(oracle):
    """Admission is by fit, not strictly first-in-first-out: while a long solve holds most of
    the budget, a queued request too large for the rest waits, and a small request submitted
    after it is admitted and finishes first; the large one runs once memory frees up."""
    (ms, bs), (mb, bb) = requests([1e4, 6e4], seed0=300)
    o = capi.cg_default_options(rtol=1e-8)
    # the server's footprint estimates, read back as the peak of each request run alone
    probe = capi.spmv_server_create(8 << 30, 1)
    est = []
    for m, b in ((ms, bs), (mb, bb)):
        t = capi.spmv_server_submit(probe, m.n, m.row_ptr, m.col_idx, m.values, b, o)
        wait_all(probe, [t], [m])
        est.append(capi.spmv_server_get_stats(probe)["peak_bytes"])
    capi.spmv_server_destroy(probe)
    est_small, est_big = est
    assert est_big > 2 * est_small
    # room for one large and one small request, not for two large ones
    srv = capi.spmv_server_create(est_big + est_small + est_small // 2, 3)
    endless = capi.cg_default_options(rtol=0.0, max_iter=10 ** 7)
    t1 = capi.spmv_server_submit(srv, mb.n, mb.row_ptr, mb.col_idx, mb.values, bb, endless)
    t0 = time.time()
    while capi.spmv_server_get_stats(srv)["active_slots"] < 1:
        assert time.time() - t0 < 30.0
        time.sleep(0.001)
    t2 = capi.spmv_server_submit(srv, mb.n, mb.row_ptr, mb.col_idx, mb.values, bb, o)
    t3 = capi.spmv_server_submit(srv, ms.n, ms.row_ptr, ms.col_idx, ms.values, bs, o)
    x3, r3 = wait_all(srv, [t3], [ms])[0]
    assert r3["status"] == capi.SPMV_OK and relres(oracle, ms, x3, bs) <= 1e-8
    # the small one finished while the first large one still runs and the second still waits
    assert capi.spmv_server_poll(srv, t1, np.empty(mb.n)) is None
    assert capi.spmv_server_poll(srv, t2, np.empty(mb.n)) is None
    assert capi.spmv_server_get_stats(srv)["queued"] == 1
    capi.spmv_server_cancel(srv, t1)
    (x2, r2), (_, r1) = wait_all(srv, [t2, t1], [mb, mb])
    assert r1["status"] == capi.SPMV_ERR_CANCELLED
    assert r2["status"] == capi.SPMV_OK and relres(oracle, mb, x2, bb) <= 1e-8
    capi.spmv_server_destroy(srv)


def test_priority_streams_leave_results_unchanged(oracle):
    """Requests above the priority threshold run on high-priority streams; their results are
    the same bits as at the default priority."""
    reqs = requests([3e4, 1.2e4, 5e4], seed0=400)
    o = capi.cg_default_options(rtol=1e-8)
    outs = []
    for threshold in (0, 1, 20 << 20):
        srv = capi.spmv_server_create(8 << 30, 3)
        capi.spmv_server_set_priority_bytes(srv, threshold)
        ts = [capi.spmv_server_submit(srv, m.n, m.row_ptr, m.col_idx, m.values, b, o)
              for m, b in reqs]
        outs.append(wait_all(srv, ts, [m for m, _ in reqs]))
        capi.spmv_server_destroy(srv)
    for i, (m, b) in enumerate(reqs):
        x0, r0 = outs[0][i]
        assert r0["status"] == capi.SPMV_OK and relres(oracle, m, x0, b) <= 1e-8
        for out in outs[1:]:
            assert np.array_equal(out[i][0], x0)
