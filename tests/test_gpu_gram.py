"""GPU parity of cw_gram, the Gram matrix [SA | Sb]^T [SA | Sb] behind the
LSQR preconditioner (Section 7.6), against the float64 oracle.

Error model.  For d <= 256 the kernel splits each float32 value x into
hi = x truncated to TF32 and lo = x - hi, and forms hi*hi + hi*lo + lo*hi on
the tensor cores (lo itself truncated to TF32 there): each product is off by
at most 3 * 2^-20 |x y|.  The products are summed in float32 over one CTA's
rows (at most `rows_per` of them), then across CTAs as float32 two-word
sums (~44 bits, error negligible here); the Sb
column is float32 FMAs over the same rows.  With Cauchy-Schwarz,
    |G - G_o|_ij <= (3 * 2^-20 + rows_per * 2^-23) sqrt(G_ii G_jj).
The test allows 4 * 2^-20 + rows_per * 2^-22.  A kernel that dropped the
lo terms would be off by about 2^-10 relative on the diagonal (truncation
errors all have the sign of x^2), tens of times above that tolerance at the
sizes below; a dropped stage or a misplaced column is off by far more.
d > 256 takes the float32 CUDA-core tiles with the same bound (their row
chunks play the part of rows_per).  tests/test_gram_tolerance.py checks on the
CPU that an emulation of the kernel's arithmetic meets this tolerance and that
the emulated mistakes above do not.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cw():
    import paper_1207_6365_gb300 as cw
    cw.load()
    return cw


def _rows_per(m, d):
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    if d <= 256:
        stages = -(-m // 32)
        return 32 * -(-stages // min(nsm, stages))
    ntile = -(-d // 128)
    ntl = ntile * (ntile + 1) // 2
    return max(256, -(-m * ntl // nsm) + 32)


def _inputs(m, d, with_b, seed):
    SA = W.dense_gaussian(m, d, seed)
    # columns over six decades, as the columns of a sketch of a Zipf matrix
    scale = torch.pow(10.0, torch.linspace(-3, 3, d, dtype=torch.float64)).to(torch.float32)
    SA = (SA * scale[torch.randperm(d, generator=torch.Generator().manual_seed(seed))]).contiguous()
    Sb = W.dense_gaussian(m, 1, seed + 1)[:, 0].contiguous() if with_b else None
    return SA, Sb


def _check(cw, m, d, with_b, seed):
    SA, Sb = _inputs(m, d, with_b, seed)
    G = cw.cw_gram(SA.cuda(), Sb.cuda() if Sb is not None else None).cpu().numpy()
    Go = oracle.gram(SA.numpy(), Sb.numpy() if Sb is not None else None)
    assert G.shape == Go.shape
    np.testing.assert_array_equal(G, G.T)
    dg = np.sqrt(np.diag(Go))
    err = np.abs(G - Go) / np.maximum(np.outer(dg, dg), 1e-300)
    tol = 4 * 2.0 ** -20 + _rows_per(m, d) * 2.0 ** -22
    assert err.max() <= tol, (err.max(), tol, np.unravel_index(err.argmax(), err.shape))
    return G


@pytest.mark.parametrize("m,d,with_b", [
    (5000, 64, True),      # 16-byte loads, one accumulator block
    (5000, 7, True),       # element loads, one 16-column chunk
    (1, 3, True),          # one row
    (31, 16, False),       # one partial stage, no Sb
    (4867, 129, True),     # second accumulator block 16 columns wide
    (20000, 150, True),    # element loads, two blocks, ragged tail
    (3000, 200, False),
    (65536, 256, True),    # the full-size sketch of the large sparse problem
    (10000, 300, True),    # d > 256: the CUDA-core tiles
    (300, 1, True)])
def test_gram_matches_oracle(cw, m, d, with_b):
    _check(cw, m, d, with_b, seed=m % 89 + d)


def test_gram_is_deterministic(cw):
    SA, Sb = _inputs(40000, 96, True, 5)
    G1 = cw.cw_gram(SA.cuda(), Sb.cuda())
    G2 = cw.cw_gram(SA.cuda(), Sb.cuda())
    assert torch.equal(G1, G2)


def test_gram_without_sb_is_the_leading_block(cw):
    SA, Sb = _inputs(7000, 48, True, 9)
    G = cw.cw_gram(SA.cuda(), Sb.cuda())
    G0 = cw.cw_gram(SA.cuda())
    assert torch.equal(G[:48, :48], G0)


def test_gram_exact_on_small_integers(cw):
    """Integers below 2^11 are exact in TF32 (lo = 0) and their products and
    float32 partial sums below 2^24 are exact, so every entry is exact."""
    g = torch.Generator().manual_seed(17)
    m, d = 4000, 40
    SA = torch.randint(-7, 8, (m, d), generator=g).to(torch.float32)
    Sb = torch.randint(-7, 8, (m,), generator=g).to(torch.float32)
    G = cw.cw_gram(SA.cuda(), Sb.cuda()).cpu().numpy()
    Go = oracle.gram(SA.numpy(), Sb.numpy())
    assert math.isfinite(float(np.abs(Go).max()))
    np.testing.assert_array_equal(G, Go)
