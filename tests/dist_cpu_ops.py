"""Test-only device-op backend for the multi-GPU decomposition on CPU ranks (gloo): the same
interface as paper_1711_10622_gb300.decomposition.CudaOps, on torch float64 CPU tensors, with the
local products computed by the oracle (its CSR product on the rank's row block, which sums every
row in the same order as the global oracle product). Test infrastructure: never used by the
library."""

import numpy as np
import torch

import oracle


class CpuOps:
    def matrix(self, csr, n_cols):
        return csr if len(csr[0]) > 1 else None

    def zeros(self, rows, m):
        return torch.zeros((rows, m), dtype=torch.float64)

    def from_host(self, a, dtype=None):
        a = np.ascontiguousarray(a if dtype is None else a.astype(dtype))
        return torch.from_numpy(a.copy())

    def to_host(self, t):
        return t.numpy()

    def gspmv(self, A, X, Y):
        if A is None:
            return
        Y.copy_(torch.from_numpy(oracle.gspmv_csr(A, X.numpy())))

    def dots(self, pairs, rows):
        return torch.cat([(x[:rows] * y[:rows]).sum(dim=0) for x, y in pairs])

    def lincomb(self, coefs, vecs, out, rows):
        acc = None
        for c, v in zip(coefs, vecs):
            term = v[:rows] if c is None else v[:rows] * c
            acc = term.clone() if acc is None else acc + term
        out[:rows].copy_(acc)

    def gather(self, idx, X, out):
        out.copy_(X.index_select(0, idx.long()))
