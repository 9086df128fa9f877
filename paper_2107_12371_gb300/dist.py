"""Transport of the row-block partition (spmv_partition_*, cg_solve_partitioned): the halo
exchange and the scalar all-reduce over torch.distributed, one part per rank (rank = part).

Argument marshalling and communication only: the packing of send buffers, the products and
every step of the CG recurrence run in the library's kernels; this module moves the packed
entries and the partial sums between ranks (NCCL for device buffers, gloo for host ones).
"""
from __future__ import annotations

import ctypes

import numpy as np


def _view(ptr, count, device):
    """A float64 torch tensor over `count` entries at address `ptr` (no copy)."""
    import torch
    if device is None or torch.device(device).type == "cpu":
        if count == 0:
            return torch.empty(0, dtype=torch.float64)
        buf = (ctypes.c_double * count).from_address(ptr)
        return torch.from_numpy(np.ctypeslib.as_array(buf))

    class _Cai:
        __cuda_array_interface__ = {"shape": (count,), "typestr": "<f8", "data": (ptr, False),
                                    "version": 3, "strides": None}
    if count == 0:
        return torch.empty(0, dtype=torch.float64, device=device)
    return torch.as_tensor(_Cai(), device=device)


class TorchTransport:
    """Exchange and all-reduce of one part (Partition) over a torch.distributed group whose
    rank r holds part r.  device: where the send / receive buffers live (None = host)."""

    def __init__(self, part, device=None, group=None):
        self.part = part
        self.device = device
        self.group = group
        self.send_counts = [int(c) for c in part.send_counts]
        self.recv_counts = [int(c) for c in part.recv_counts]

    def exchange(self, send_ptr, recv_ptr):
        import torch.distributed as dist
        send = _view(send_ptr, sum(self.send_counts), self.device)
        recv = _view(recv_ptr, sum(self.recv_counts), self.device)
        ops = []
        off = 0
        for q, c in enumerate(self.send_counts):
            if c:
                ops.append(dist.P2POp(dist.isend, send[off:off + c], q, self.group))
            off += c
        off = 0
        for q, c in enumerate(self.recv_counts):
            if c:
                ops.append(dist.P2POp(dist.irecv, recv[off:off + c], q, self.group))
            off += c
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()

    def allreduce(self, values):
        import torch
        import torch.distributed as dist
        t = torch.from_numpy(np.array(values, dtype=np.float64))
        if self.device is not None and torch.device(self.device).type != "cpu":
            t = t.to(self.device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        values[:] = t.cpu().numpy()


def exchange_halo(part, transport, x_ext, send, stream=None):
    """Fill the halo of x_ext (a float64 tensor of n_ext entries: [low halo | own | high halo])
    from the other ranks: pack the own entries other parts read, exchange, place the runs."""
    import torch
    info = part.info
    lo, nl = info["n_halo_lo"], info["n_local"]
    recv = torch.empty(info["recv_total"], dtype=torch.float64, device=x_ext.device)
    if info["send_total"]:
        part.pack(x_ext[lo:lo + nl], send, stream)
        torch.cuda.synchronize(x_ext.device)
    transport.exchange(send.data_ptr(), recv.data_ptr())
    x_ext[:lo] = recv[:lo]
    x_ext[lo + nl:] = recv[lo:]
