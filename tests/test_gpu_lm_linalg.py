"""The Levenberg-Marquardt trainer's linear algebra on the library's own
kernels (Sec. 3 fits the thermo network with the Levenberg-Marquardt
algorithm): the Gauss-Newton matrix G = X X^T on the tensor cores
(stev_gram_tf32: tcgen05 MMAs in TF32, FP32 accumulation in tensor memory,
TMA-staged operands) and the damped solve by preconditioned conjugate
gradients (stev_damped_cg), each against an FP64 numpy computation.

The sizes are ragged on purpose: n not a multiple of the 128-row tile, k not
a multiple of the 32-value block, so that the edge tiles' zero fill is
exercised; the larger case spans several tile rows and columns."""
import numpy as np
import pytest

from paper_1905_09395_b300 import binding

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,k", [(1, 1), (131, 45), (300, 1000), (700, 4113)])
def test_gram_of_small_integers_is_exact(n, k):
    """Integers of |x| <= 8 are exact in TF32 and their dot products (at most
    64 k < 2^24) are exact in FP32 accumulation: G must equal the integer
    Gram matrix bit for bit, and be symmetric."""
    rng = np.random.default_rng(n + k)
    ldx = (k + 3) // 4 * 4
    X = np.zeros((n, ldx), np.float32)
    X[:, :k] = rng.integers(-8, 9, size=(n, k))
    X[:, k:] = 1e30          # padding beyond k must not be read
    G = binding.gram_tf32(_dev(X), k).cpu().numpy().astype(np.float64)
    Xi = X[:, :k].astype(np.int64)
    np.testing.assert_array_equal(G, (Xi @ Xi.T).astype(np.float64))


@pytest.mark.parametrize("n,k", [(300, 1000), (700, 4113)])
def test_gram_within_the_tf32_bound(n, k):
    """Random normal X: |G - X X^T| <= (2^-9 + k 2^-23) (|X| |X|^T) element by
    element (each TF32 input keeps 10 mantissa bits, so a product is within
    2^-9 relative; FP32 accumulation of k terms adds k 2^-24 relative per
    term, doubled for slack), and the typical error is far below the bound."""
    rng = np.random.default_rng(7)
    ldx = (k + 3) // 4 * 4
    Xp = np.zeros((n, ldx), np.float32)
    Xp[:, :k] = rng.normal(size=(n, k))
    G = binding.gram_tf32(_dev(Xp), k).cpu().numpy().astype(np.float64)
    X64 = Xp[:, :k].astype(np.float64)
    ref = X64 @ X64.T
    scale = np.abs(X64) @ np.abs(X64).T
    err = np.abs(G - ref)
    assert np.all(err <= (2.0 ** -9 + k * 2.0 ** -23) * scale)
    assert np.median(err / scale) < 2.0 ** -11
    np.testing.assert_array_equal(G, G.T)


def test_damped_cg_solves_the_marquardt_system():
    rng = np.random.default_rng(3)
    n = 500
    M = rng.normal(size=(n, n))
    A = (M @ M.T / n + np.diag(rng.uniform(0.5, 2.0, n))).astype(np.float32)
    b = rng.normal(size=n).astype(np.float32)
    lam, eps = 0.05, 1e-6
    x, it = binding.damped_cg(_dev(A), _dev(b), lam, eps, max_iters=2000, rtol=1e-6)
    A64 = A.astype(np.float64)
    want = np.linalg.solve(A64 + lam * np.diag(np.diag(A64)) + eps * np.eye(n), b.astype(np.float64))
    got = x.cpu().numpy().astype(np.float64)
    print("CG: %d iterations, relative error %.3g" % (it, np.linalg.norm(got - want) /
                                                        np.linalg.norm(want)))
    assert 0 < it < 2000
    assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want)
    # deterministic: the same inputs give the same x
    x2, it2 = binding.damped_cg(_dev(A), _dev(b), lam, eps, max_iters=2000, rtol=1e-6)
    assert it2 == it
    np.testing.assert_array_equal(x2.cpu().numpy(), x.cpu().numpy())


def test_damped_cg_stops_at_max_iters():
    n = 64
    A = np.eye(n, dtype=np.float32) * np.linspace(1.0, 1e4, n, dtype=np.float32)
    A[0, 1] = A[1, 0] = 0.5
    b = np.ones(n, np.float32)
    _, it = binding.damped_cg(_dev(A), _dev(b), 0.0, 0.0, max_iters=1, rtol=1e-12)
    assert it == 1


def test_gram_rejects_bad_strides():
    import torch
    X = torch.zeros((4, 6), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.StevError):
        binding.gram_tf32(X)                 # ldx = 6 is not a multiple of 4
