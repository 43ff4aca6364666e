"""Host-side solver utilities of the binding (no GPU): the closed-form 3x3 block inverse of the
block-Jacobi preconditioner and the CG solve itself on a small SPD matrix on the CPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2107_09568_gb300 as msasm  # noqa: E402


def test_inverse3_matches_the_definition():
    rng = np.random.default_rng(0)
    B = rng.standard_normal((200, 3, 3)) + 3.0 * np.eye(3)
    X = msasm._inverse3(torch.tensor(B)).numpy()
    assert np.abs(X @ B - np.eye(3)).max() <= 1e-13
    assert np.abs(B @ X - np.eye(3)).max() <= 1e-13


def test_cg_solve_block_spd_system_on_cpu():
    """A block tridiagonal SPD matrix (3 DOFs per point, interleaved) with two points clamped."""
    rng = np.random.default_rng(1)
    n_pts = 40
    n = 3 * n_pts
    K = np.zeros((n, n))
    for g in range(n_pts):
        M = rng.standard_normal((3, 3))
        K[3 * g:3 * g + 3, 3 * g:3 * g + 3] += M @ M.T + 6.0 * np.eye(3)
        if g + 1 < n_pts:
            C = 0.5 * rng.standard_normal((3, 3))
            K[3 * g:3 * g + 3, 3 * g + 3:3 * g + 6] += C
            K[3 * g + 3:3 * g + 6, 3 * g:3 * g + 3] += C.T
    f = rng.standard_normal(n)
    fixed = np.array([0, 1, 2, 3 * (n_pts - 1), 3 * (n_pts - 1) + 1, 3 * (n_pts - 1) + 2])
    Ks = torch.tensor(K).to_sparse_csr()
    u, iters, res = msasm.cg_solve(Ks, torch.tensor(f), torch.tensor(fixed), tol=1e-12, max_iter=2000,
                                   replace_every=5)
    free = np.setdiff1d(np.arange(n), fixed)
    ref = np.zeros(n)
    ref[free] = np.linalg.solve(K[np.ix_(free, free)], f[free])
    assert res < 1e-12 and iters < 2000
    assert np.abs(u.numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.all(u.numpy()[fixed] == 0.0)
