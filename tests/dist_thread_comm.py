"""Test-only communicator: G ranks emulated as host threads of one process on one GPU.

Every rank issues its device work on the same (current, legacy default) CUDA stream, so the work of
all ranks runs in the order the host issued it; messages are device-to-device copies issued by the
receiving thread after a host barrier that follows every sender's packing. No kernel ever waits for
another rank's kernel (the ranks meet only on the host). Test infrastructure, not part of the
library."""

import threading


class Hub:
    def __init__(self, size):
        self.size = size
        self.barrier = threading.Barrier(size)
        self.mail = {}
        self.slots = [None] * size


class ThreadComm:
    def __init__(self, hub, rank):
        self.hub, self.rank, self.size = hub, rank, hub.size

    def exchange(self, sends, recvs):
        for q, t in sends.items():
            self.hub.mail[(self.rank, q)] = t
        return recvs

    def wait(self, recvs):
        self.hub.barrier.wait()  # every sender has queued its packing and posted its buffers
        for q, t in recvs.items():
            t.copy_(self.hub.mail[(q, self.rank)])
        self.hub.barrier.wait()  # every receiver has queued its copies before buffers are reused

    def allreduce(self, t):
        self.hub.slots[self.rank] = t.clone()
        self.hub.barrier.wait()
        total = self.hub.slots[0].clone()
        for r in range(1, self.size):
            total += self.hub.slots[r]
        self.hub.barrier.wait()
        t.copy_(total)
        return t

    def allgather_columns(self, X, shares):
        import torch

        self.hub.slots[self.rank] = X
        self.hub.barrier.wait()
        out = torch.cat([self.hub.slots[r] for r in range(self.size)], dim=1).contiguous()
        self.hub.barrier.wait()
        return out


def run_ranks(size, fn):
    """Run fn(comm) on `size` threads; returns the per-rank results (re-raises the first error)."""
    hub = Hub(size)
    res, err = [None] * size, [None] * size

    def body(r):
        try:
            res[r] = fn(ThreadComm(hub, r))
        except BaseException as exc:  # unblock the others, then report
            err[r] = exc
            hub.barrier.abort()

    ts = [threading.Thread(target=body, args=(r,)) for r in range(size)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(600)
    for e in err:
        if e is not None and not isinstance(e, threading.BrokenBarrierError):
            raise e
    for e in err:
        if e is not None:
            raise e
    return res
