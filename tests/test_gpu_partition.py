"""Row-block partition with halo exchange on one GPU (parts emulated in one process): every
part's device handle, its pack kernel and its product through the C ABI; the parts' products
concatenated are the oracle's product of the whole matrix bit for bit, and the partitioned
Jacobi-PCG (two parts on two host threads, the transport an in-process exchange of device
buffers and a host all-reduce) reaches the oracle's residual with the oracle's iteration count
within 2.  No kernel waits on another: the parts meet only on the host."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_12371_gb300 import capi, dist as pdist, meshgen, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    capi.load()


def _rcm_system(oracle, kind, n):
    if kind == "kuhn":
        m, rng = meshgen.kuhn_tet_matrix(n, seed=2, dirichlet=True)
        x = meshgen.uniform_vectors(rng, m.n)
    elif kind == "c2":
        m, x = workloads.c2()
    else:
        m, rng = meshgen.mixed_matrix(n, seed=1, dirichlet=True)
        x = meshgen.uniform_vectors(rng, m.n)
    perm = oracle.cm_order(m.row_ptr, m.col_idx)
    rp, ci, v = oracle.permute_csr(m.row_ptr, m.col_idx, m.values, perm)
    return m.n, rp, ci, v, np.ascontiguousarray(x[perm])


class InProcess:
    """Transport between the parts of one process, one host thread per part: each part posts
    its send buffer, and after a barrier copies from every other part's buffer the run
    addressed to it (device copies); the all-reduce sums the parts' values in part order."""

    def __init__(self, parts):
        self.parts = parts
        self.barrier = threading.Barrier(len(parts), timeout=120)
        self.posted = {}
        self.vals = {}

    def exchange(self, p, send_ptr, recv_ptr):
        P = self.parts[p]
        self.posted[p] = send_ptr
        self.barrier.wait()
        recv = pdist._view(recv_ptr, P.info["recv_total"], "cuda")
        off = 0
        for q, c in enumerate(P.recv_counts):
            if c:
                Q = self.parts[q]
                src = pdist._view(self.posted[q], Q.info["send_total"], "cuda")
                so = int(np.sum(Q.send_counts[:p]))
                recv[off:off + c].copy_(src[so:so + c])
                off += int(c)
        torch.cuda.synchronize()
        self.barrier.wait()

    def allreduce(self, p, values):
        self.vals[p] = values.copy()
        self.barrier.wait()
        total = self.vals[0].copy()
        for q in range(1, len(self.parts)):
            total = total + self.vals[q]
        values[:] = total
        self.barrier.wait()


def _bounds(n, n_parts):
    return [int(round(i * n / n_parts)) for i in range(n_parts + 1)]


@pytest.mark.parametrize("kind,size,n_parts", [("kuhn", 20, 2), ("kuhn", 20, 3),
                                               ("mixed", 14, 4), ("c2", 0, 2)])
def test_partitioned_product_is_bit_exact(oracle, kind, size, n_parts):
    n, rp, ci, v, x = _rcm_system(oracle, kind, size)
    rb = _bounds(n, n_parts)
    parts = [capi.Partition(n, rp, ci, v, rb, p) for p in range(n_parts)]
    xd = torch.from_numpy(x).cuda()
    sends = []
    for P in parts:  # every part packs what the others read of its own entries
        s = torch.zeros(max(1, P.info["send_total"]), dtype=torch.float64, device="cuda")
        P.pack(xd[P.info["row_begin"]:P.info["row_end"]], s)
        sends.append(s)
    torch.cuda.synchronize()
    y = torch.empty_like(xd)
    for p, P in enumerate(parts):
        lo, nl = P.info["n_halo_lo"], P.info["n_local"]
        recv = []
        for q, c in enumerate(P.recv_counts):
            if c:
                so = int(np.sum(parts[q].send_counts[:p]))
                recv.append(sends[q][so:so + int(c)])
        recv = torch.cat(recv) if recv else torch.zeros(0, dtype=torch.float64, device="cuda")
        x_ext = torch.cat([recv[:lo], xd[P.info["row_begin"]:P.info["row_end"]], recv[lo:]])
        assert torch.equal(x_ext[:lo].cpu(), torch.from_numpy(x[P.halo_cols[:lo]]))
        P.apply(x_ext, y[P.info["row_begin"]:P.info["row_end"]])
        assert P.info["n_ext"] == x_ext.numel()
    torch.cuda.synchronize()
    ref = oracle.spmv(rp, ci, v, x, use_fma=True)
    assert np.array_equal(y.cpu().numpy(), ref)
    if kind != "c2":
        # RCM keeps every halo to the neighbouring parts
        for p, P in enumerate(parts):
            assert all(c == 0 for q, c in enumerate(P.recv_counts) if abs(q - p) > 1)


@pytest.mark.parametrize("kind,size,n_parts", [("kuhn", 16, 2), ("mixed", 12, 3)])
def test_partitioned_cg_matches_oracle(oracle, kind, size, n_parts):
    n, rp, ci, v, b = _rcm_system(oracle, kind, size)
    rb = _bounds(n, n_parts)
    streams = [torch.cuda.Stream() for _ in range(n_parts)]
    parts = [capi.Partition(n, rp, ci, v, rb, p, stream=streams[p]) for p in range(n_parts)]
    T = InProcess(parts)
    bd = torch.from_numpy(b).cuda()
    x = torch.full_like(bd, float("nan"))
    results = [None] * n_parts

    def run(p):
        P = parts[p]
        r0, r1 = P.info["row_begin"], P.info["row_end"]
        results[p] = P.solve(bd[r0:r1], x[r0:r1],
                             lambda s, r: T.exchange(p, s, r),
                             lambda vals: T.allreduce(p, vals),
                             stream=streams[p], rtol=1e-10)
    threads = [threading.Thread(target=run, args=(p,)) for p in range(n_parts)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    torch.cuda.synchronize()
    assert all(r is not None and r["status"] == capi.SPMV_OK for r in results), results
    its = {r["iterations"] for r in results}
    assert len(its) == 1
    xs = x.cpu().numpy()
    res = np.linalg.norm(b - oracle.spmv(rp, ci, v, xs)) / np.linalg.norm(b)
    assert res <= 1e-10
    assert abs(results[0]["rel_residual"] - res) <= 1e-12
    _, info = oracle.jacobi_pcg(rp, ci, v, b, rtol=1e-10)
    assert abs(its.pop() - info["iterations"]) <= 2
