"""Row-block partition with halo exchange, host side, on CPU: two gloo ranks (world size 2),
each holding one part of an RCM-ordered Kuhn-tet matrix built by spmv_partition_create without
a GPU (the host plan).  The halo exchange through dist.TorchTransport delivers exactly the
entries each part's halo names; the parts' products (the oracle's SpMV on each part's CSR
over its extended vector) concatenate to the oracle's product of the whole matrix bit for
bit; the all-reduce sums the parts' scalars; and a textbook Jacobi-PCG run over the partition
with this transport (one exchange and two all-reduces per iteration) converges like the
oracle's solve of the whole system."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _system():
    import oracle
    from paper_2107_12371_gb300 import meshgen
    m, rng = meshgen.kuhn_tet_matrix(8, seed=11, dirichlet=True)
    perm = oracle.cm_order(m.row_ptr, m.col_idx)
    rp, ci, v = oracle.permute_csr(m.row_ptr, m.col_idx, m.values, perm)
    x = meshgen.uniform_vectors(rng, m.n)
    return m.n, rp, ci, v, x


def _worker(rank, world, port, row_begin, q):
    try:
        sys.path.insert(0, ROOT)
        import torch
        import torch.distributed as dist

        import oracle
        from paper_2107_12371_gb300 import capi, dist as pdist
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        dist.init_process_group("gloo", rank=rank, world_size=world)
        n, rp, ci, v, x = _system()
        P = capi.Partition(n, rp, ci, v, row_begin, rank, on_device=False)
        info = P.info
        lo, nl, hi = info["n_halo_lo"], info["n_local"], info["n_halo_hi"]
        r0, r1 = info["row_begin"], info["row_end"]
        T = pdist.TorchTransport(P, device=None)
        lrp, lci, lv = P.local_csr()

        def halo_exchange(x_own):
            send = torch.from_numpy(np.ascontiguousarray(x_own[P.send_rows]))
            recv = torch.zeros(info["recv_total"], dtype=torch.float64)
            T.exchange(send.data_ptr(), recv.data_ptr())
            r = recv.numpy()
            return np.concatenate([r[:lo], x_own, r[lo:]])

        # the exchange delivers exactly the halo's entries
        x_ext = halo_exchange(x[r0:r1].copy())
        assert np.array_equal(x_ext[:lo], x[P.halo_cols[:lo]])
        assert np.array_equal(x_ext[lo + nl:], x[P.halo_cols[lo:]])
        assert lo + nl + hi == info["n_ext"]
        # the part's product equals the whole matrix's rows bit for bit
        y_loc = oracle.spmv(lrp, lci, lv, x_ext, use_fma=True)
        y_all = oracle.spmv(rp, ci, v, x, use_fma=True)
        assert np.array_equal(y_loc, y_all[r0:r1])
        # the all-reduce sums the parts' values
        vals = np.array([1.0 + rank, 10.0 * rank])
        T.allreduce(vals)
        assert vals.tolist() == [3.0, 10.0]
        # textbook Jacobi-PCG over the partition: one halo exchange and two all-reduces of
        # scalars per iteration
        b = x[r0:r1].copy()
        diag = np.array([lv[k] for i in range(nl) for k in range(lrp[i], lrp[i + 1])
                         if lci[k] == lo + i])
        dinv = 1.0 / diag
        xs = np.zeros(nl)
        r = b.copy()
        p = dinv * r
        s = np.array([r @ p, r @ r, b @ b])
        T.allreduce(s)
        rho, rr, bb = s
        it = 0
        while rr > 1e-20 * bb and it < 1000:
            qv = oracle.spmv(lrp, lci, lv, halo_exchange(p), use_fma=True)
            pq = np.array([p @ qv])
            T.allreduce(pq)
            alpha = rho / pq[0]
            xs += alpha * p
            r -= alpha * qv
            s = np.array([r @ (dinv * r), r @ r])
            T.allreduce(s)
            it += 1
            beta = s[0] / rho
            rho, rr = s
            p = dinv * r + beta * p
        q.put((rank, it, xs.tolist(), r0, r1))
        dist.barrier()
        dist.destroy_process_group()
    except BaseException as e:  # report to the parent, then fail this process
        q.put((rank, "error", repr(e), 0, 0))
        raise


@pytest.mark.parametrize("split", ["even", "uneven"])
def test_partition_halo_and_allreduce_over_gloo(oracle, split):
    import torch.multiprocessing as mp
    n = 6 * 8 ** 3
    row_begin = [0, n // 2, n] if split == "even" else [0, n // 3, n]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, row_begin, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
    for item in got:
        assert item[1] != "error", item
    for p in procs:
        assert p.exitcode == 0
    got.sort()
    its = {g[1] for g in got}
    assert len(its) == 1
    n_, rp, ci, v, x = _system()
    xs = np.zeros(n_)
    for _, _, xp, r0, r1 in got:
        xs[r0:r1] = xp
    b = x
    res = np.linalg.norm(b - oracle.spmv(rp, ci, v, xs)) / np.linalg.norm(b)
    assert res <= 1e-10
    _, info = oracle.jacobi_pcg(rp, ci, v, b, rtol=1e-10)
    assert abs(its.pop() - info["iterations"]) <= 2


def test_partition_plan_rejects_bad_input():
    from paper_2107_12371_gb300 import capi
    n, rp, ci, v, _ = _system()
    with pytest.raises(capi.SpmvError) as e:
        capi.Partition(n, rp, ci, v, [0, n + 1, n], 0, on_device=False)
    assert e.value.status == capi.SPMV_ERR_INVALID_ARG
    bad = ci.copy()
    bad[3] = n + 5
    with pytest.raises(capi.SpmvError) as e:
        capi.Partition(n, rp, bad, v, [0, n // 2, n], 1, on_device=False)
    assert e.value.status == capi.SPMV_ERR_INVALID_CSR
    # one part: no halo, nothing sent
    P = capi.Partition(n, rp, ci, v, [0, n], 0, on_device=False)
    assert P.info["recv_total"] == 0 and P.info["send_total"] == 0
    lrp, lci, lv = P.local_csr()
    assert np.array_equal(lrp, rp) and np.array_equal(lci, ci)
