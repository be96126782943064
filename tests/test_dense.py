"""Dense linear algebra of the tomographic operators on the tensor cores
(synim_linalg_gemm / synim_linalg_spd_solve), against FP64 numpy.

GEMM criterion: |C - C_64| <= 2e-6 * (|A| |B|)_{mn} + 1e-6 |beta C0|_{mn}
elementwise: three TF32 products (hi.hi + hi.lo + lo.hi) carry ~2^-21 of each
product, FP32 accumulation ~K 2^-24 of the absolute sum.  Shapes cover several
128 x 128 tiles, ragged edges in M, N and K (not multiples of 128 / 32), both
layouts of B, alpha / beta, K = 0, and few tiles with a long K (the split-K
path).

SPD solve criterion: Y S^-1 within 1e-4 relative (Frobenius) of FP64 for a
well-conditioned S (cond ~ 1e2) at sizes spanning several 128-row blocks and
a ragged last block; a matrix that is not positive definite is refused.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2606_07759_b300 import abi

pytestmark = pytest.mark.gpu


def _gemm(A, B, C, alpha, beta, b_kn):
    L = abi.load()
    M, K = A.shape
    N = C.shape[1]
    st = L.synim_linalg_gemm(M, N, K, alpha, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), int(b_kn), beta,
                             C.data_ptr(), C.stride(0), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, L.synim_last_error(None)


# (300, 128, 3000) and (1369, 100, 2411) have few output tiles and a long K:
# they take the split-K path (partials over blockIdx.z, added in order)
@pytest.mark.parametrize("M,N,K", [(256, 384, 256), (300, 170, 77), (129, 1, 33), (64, 200, 0), (517, 263, 1000),
                                   (300, 128, 3000), (1369, 100, 2411)])
@pytest.mark.parametrize("b_kn", [0, 1])
def test_gemm_matches_fp64(M, N, K, b_kn):
    g = torch.Generator().manual_seed(M * 1000 + N + K)
    A = torch.randn(M, K, generator=g, dtype=torch.float64)
    B = torch.randn(N, K, generator=g, dtype=torch.float64)
    C0 = torch.randn(M, N, generator=g, dtype=torch.float64)
    alpha, beta = 0.75, -1.25
    Bdev = (B.t().contiguous() if b_kn else B).float().cuda()
    C = C0.float().cuda()
    _gemm(A.float().cuda(), Bdev, C, alpha, beta, b_kn)
    A32, B32, C32 = A.float().double(), B.float().double(), C0.float().double()
    ref = alpha * A32 @ B32.t() + beta * C32
    bound = 2e-6 * abs(alpha) * (A32.abs() @ B32.abs().t()) + 1e-6 * abs(beta) * C32.abs() + 1e-30
    err = (C.double().cpu() - ref).abs()
    assert bool((err <= bound).all()), float((err / bound).max())


def test_gemm_on_strided_operands():
    # leading dimensions larger than the row length (sub-blocks of a bigger matrix)
    g = torch.Generator().manual_seed(7)
    big = torch.randn(400, 300, generator=g).cuda()
    A, B = big[:200, 10:110], big[200:390, 5:105]
    C = torch.zeros(200, 190, device="cuda")
    _gemm(A, B, C, 1.0, 0.0, 0)
    ref = A.double() @ B.double().t()
    assert float((C.double() - ref).abs().max()) <= 2e-6 * float((A.double().abs() @ B.double().abs().t()).max())


@pytest.mark.parametrize("n,m", [(128, 64), (300, 257), (650, 1000), (1300, 40)])
def test_spd_solve_matches_fp64(n, m):
    L = abi.load()
    rng = np.random.default_rng(n + m)
    X = rng.standard_normal((n, n))
    S = X @ X.T / n + np.eye(n)
    Y = rng.standard_normal((m, n))
    Sd = torch.from_numpy(S).float().cuda().contiguous()
    Yd = torch.from_numpy(Y).float().cuda().contiguous()
    st = L.synim_linalg_spd_solve(Sd.data_ptr(), n, n, Yd.data_ptr(), m, n,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, L.synim_last_error(None)
    ref = np.linalg.solve(S, Y.T).T
    rel = np.linalg.norm(Yd.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert rel < 1e-4, rel
    # the factor: L L^T = S on the lower triangle
    Lf = np.tril(Sd.double().cpu().numpy())
    assert np.abs(Lf @ Lf.T - S).max() <= 1e-4 * np.abs(S).max()


def test_spd_solve_refuses_an_indefinite_matrix():
    L = abi.load()
    n = 200
    S = np.eye(n)
    S[150, 150] = -1.0
    Sd = torch.from_numpy(S).float().cuda().contiguous()
    Yd = torch.ones(3, n, device="cuda")
    st = L.synim_linalg_spd_solve(Sd.data_ptr(), n, n, Yd.data_ptr(), 3, n,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 6  # SYNIM_ERR_NOT_CONVERGED
    assert b"positive definite" in L.synim_last_error(None)
