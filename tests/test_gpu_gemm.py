"""The eigensolver's complex GEMM (pwh_subspace_gemm) against numpy complex128
products: every tile shape (widths N from 1 to 200 select different tiles),
op(A) = A and A^H, ragged M and K, a long split-K reduction (K = 34,265, the
plane-wave count of the medium cell), K = 0, alpha/beta combinations, and the
large FP64 products that run on the tensor cores as integer slices.  Bars:
FP64 arithmetic max|C - C_ref| <= 4e-15 sqrt(K) max|A| max|B| (plus
|beta| |C0| rounding); FP32 arithmetic 4e-7 sqrt(K) max|A| max|B|."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_1709_10010_gb300 as pwh
    from paper_1709_10010_gb300 import build
    build.build()
    s = pwh.System(np.diag([6.0] * 3), ecut_ha=2.0)
    return torch, s


def cplx(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


SHAPES = [(63, 1, 17), (129, 5, 40), (300, 8, 33), (257, 9, 100), (64, 16, 64), (100, 17, 7),
          (513, 32, 129), (77, 33, 250), (128, 64, 16), (130, 65, 64), (384, 128, 384),
          (1000, 200, 31), (384, 96, 34265), (1, 1, 1), (5, 3, 0),
          # FP64 products of >= 2e8 flops run as exact integer slice products on
          # the tensor cores: long and short K, padded chunks, narrow outputs
          (34265, 128, 384), (5000, 40, 1200), (3000, 7, 2000), (576, 33, 34265),
          # narrow inner products of few rows (the Jacobi-Davidson projections)
          (128, 9, 34265), (100, 20, 5000),
          # long narrow products: A^H B over K >= 65,536 and A B over M >= 65,536
          # take the tensor cores down to 1 and 16 columns (6 stays on the FP32
          # pipe for A B)
          (128, 5, 80000), (640, 1, 80000), (70000, 20, 200), (70000, 6, 300)]


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("conj_a", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gemm_vs_numpy(env, M, N, K, conj_a, precision):
    torch, s = env
    rng = np.random.default_rng([M, N, K, int(conj_a)])
    A = cplx(rng, K, M) if conj_a else cplx(rng, M, K)      # stored A
    B = cplx(rng, K, N)
    C0 = cplx(rng, M, N)
    alpha, beta = (0.7 - 0.2j), (0.3 + 0.4j)
    opA = A.conj().T if conj_a else A
    ref = alpha * (opA @ B) + beta * C0
    dev = lambda X: torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    Ct = dev(C0)
    s.gemm(dev(A), dev(B), Ct, conj_a=conj_a, alpha=alpha, beta=beta, precision=precision)
    s.sync()
    C = Ct.cpu().numpy().T
    scale = np.sqrt(max(K, 1)) * (np.abs(A).max() if A.size else 0) * (np.abs(B).max() if B.size else 0)
    eps = 4e-15 if precision == "fp64" else 4e-7
    bar = eps * scale * abs(alpha) + 4e-15 * abs(beta) * np.abs(C0).max()
    assert np.abs(C - ref).max() <= bar, (np.abs(C - ref).max(), bar)


# FP64 products whose exact partials would pass 4 GiB run in parts: K
# segments of whole chunks added into C (A^H B over a long K), or pieces of the
# larger output dimension (a tall A B whose one chunk is already too large).
@pytest.mark.parametrize("M,N,K,conj_a", [(600, 600, 40000, True), (160000, 128, 512, False)])
def test_gemm_fp64_pieces(env, M, N, K, conj_a):
    torch, s = env
    rng = np.random.default_rng([M, N, K, 7])
    A = cplx(rng, K, M) if conj_a else cplx(rng, M, K)
    B = cplx(rng, K, N)
    C0 = cplx(rng, M, N)
    alpha, beta = (0.7 - 0.2j), (0.3 + 0.4j)
    opA = A.conj().T if conj_a else A
    ref = alpha * (opA @ B) + beta * C0
    dev = lambda X: torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    Ct = dev(C0)
    s.gemm(dev(A), dev(B), Ct, conj_a=conj_a, alpha=alpha, beta=beta, precision="fp64")
    s.sync()
    C = Ct.cpu().numpy().T
    scale = np.sqrt(K) * np.abs(A).max() * np.abs(B).max()
    bar = 4e-15 * scale * abs(alpha) + 4e-15 * abs(beta) * np.abs(C0).max()
    assert np.abs(C - ref).max() <= bar, (np.abs(C - ref).max(), bar)


# The eigensolver's coefficient pairs (alpha, beta) = (1, 0) and (-1, 1) take
# the FP32 epilogue of the tensor-core FP32 path; general pairs are covered
# above.
@pytest.mark.parametrize("M,N,K,conj_a", [(384, 128, 34265, True), (34265, 128, 384, False),
                                          (128, 64, 34265, True)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-1.0, 1.0)])
def test_gemm_mixed_solver_coefficients(env, M, N, K, conj_a, alpha, beta):
    torch, s = env
    rng = np.random.default_rng([M, N, K, int(conj_a), int(beta)])
    A = cplx(rng, K, M) if conj_a else cplx(rng, M, K)
    B = cplx(rng, K, N)
    C0 = cplx(rng, M, N)
    opA = A.conj().T if conj_a else A
    ref = alpha * (opA @ B) + beta * C0
    dev = lambda X: torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    Ct = dev(C0)
    s.gemm(dev(A), dev(B), Ct, conj_a=conj_a, alpha=alpha, beta=beta, precision="mixed")
    s.sync()
    C = Ct.cpu().numpy().T
    scale = np.sqrt(K) * np.abs(A).max() * np.abs(B).max()
    bar = 4e-7 * scale + 4e-15 * abs(beta) * np.abs(C0).max()
    assert np.abs(C - ref).max() <= bar, (np.abs(C - ref).max(), bar)
