"""The tolerance of the tensor-core Gram test, checked on the CPU.

tests/test_gpu_gram.py accepts |G - G_o|_ij <= (4 * 2^-20 + rows_per * 2^-22)
sqrt(G_ii G_jj).  Here the kernel's arithmetic is emulated in numpy: each
float32 value split into hi (truncated to TF32: the low 13 mantissa bits
cleared) and lo = x - hi (truncated to TF32 again, as the MMA reads it), the
products hi*hi + hi*lo + lo*hi summed in float32 over each CTA's rows, the
per-CTA partials added in float64.  The emulation must meet the tolerance,
and two plausible mistakes must not: dropping the lo terms (one TF32 product)
and dropping one 32-row stage of a CTA.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

NSM = 152   # CTAs of the kernel: one per SM of a GB300


def _tf32(x):
    return (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def _rows_per(m):
    stages = -(-m // 32)
    return 32 * -(-stages // min(NSM, stages))


def _inputs(m, d, seed):
    SA = W.dense_gaussian(m, d, seed)
    scale = torch.pow(10.0, torch.linspace(-3, 3, d, dtype=torch.float64)).to(torch.float32)
    SA = (SA * scale[torch.randperm(d, generator=torch.Generator().manual_seed(seed))]).contiguous()
    return SA.numpy()


def _emulate(X, lo_terms=True, drop_stage=False):
    m = X.shape[0]
    rp = _rows_per(m)
    hi = _tf32(X)
    lo = _tf32((X - hi).astype(np.float32))
    G = np.zeros((X.shape[1], X.shape[1]))
    for r0 in range(0, m, rp):
        r1 = min(m, r0 + rp)
        if drop_stage and r0 == 0 and r1 - r0 > 32:
            r0 += 32
        h, l = hi[r0:r1], lo[r0:r1]
        P = h.T @ h                      # float32 products of TF32 values: exact; float32 sums
        if lo_terms:
            P = P + (h.T @ l) + (l.T @ h)
        G += P.astype(np.float64)
    return G


def _err(G, X):
    Go = oracle.gram(X)
    dg = np.sqrt(np.diag(Go))
    return (np.abs(G - Go) / np.outer(dg, dg)).max()


@pytest.mark.parametrize("m,d", [(5000, 64), (65536, 256), (20000, 150)])
def test_emulated_kernel_meets_the_tolerance_and_mistakes_do_not(m, d):
    X = _inputs(m, d, seed=m % 89 + d)
    tol = 4 * 2.0 ** -20 + _rows_per(m) * 2.0 ** -22
    assert _err(_emulate(X), X) <= tol
    assert _err(_emulate(X, lo_terms=False), X) > 3 * tol
    assert _err(_emulate(X, drop_stage=True), X) > 3 * tol
