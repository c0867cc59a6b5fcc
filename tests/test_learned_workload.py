"""Host-side checks of the learned-sketch workload recipe (no GPU)."""
import torch

import workloads as W


def test_family_basis_and_member():
    V, sig = W.family_basis(16, seed=7)
    assert torch.allclose(V.T @ V, torch.eye(16, dtype=torch.float64), atol=1e-12)
    assert torch.allclose(sig, torch.arange(1, 17, dtype=torch.float64) ** -1.5)
    V2, _ = W.family_basis(16, seed=7)
    assert torch.equal(V, V2)
    A, b = W.family_matrix(5, 8192, V, sig)
    assert A.shape == (8192, 16) and b.shape == (8192,) and A.dtype == torch.float32
    # remove the noise part's scale: A^T A = V diag(sig^2) V^T + O(noise)
    G = A.double().T @ A.double()
    target = V @ torch.diag(sig ** 2) @ V.T + (1e-3 ** 2) * 8192 * torch.eye(16, dtype=torch.float64)
    assert (G - target).abs().max() < 0.02
    A2, b2 = W.family_matrix(5, 8192, V, sig)
    assert torch.equal(A, A2) and torch.equal(b, b2)
    A3, _ = W.family_matrix(6, 8192, V, sig)
    assert not torch.equal(A, A3)


def test_haar_rinv_gives_the_sign_fixed_householder_q():
    """Z R^-1 (R the Cholesky factor of Z^T Z) is the Q of Z's Householder QR with
    R's diagonal made positive, to the rounding of the float32 Gram matrix."""
    Z = torch.randn(4096, 24, generator=torch.Generator().manual_seed(5))
    U = Z.double() @ W.haar_rinv(Z)
    q, r = torch.linalg.qr(Z.double())
    sg = torch.sign(torch.diagonal(r))
    assert (U - q * sg).abs().max() < 1e-5
    assert (U.T @ U - torch.eye(24, dtype=torch.float64)).abs().max() < 1e-5
