"""GPU tests of the FP64-accurate tensor-core GEMM (lc_gemm_f64_tc, the
digit-sliced BF16 product the accept step's projections run on in mixed
mode), through the C ABI, against an extended-precision product on the host,
and of the closure with it against the FP64 SIMT GEMMs and the oracle."""
import numpy as np
import pytest

import oracle.closure as oc
from paper_2506_01120_gb300 import binding, inputs
from paper_2506_01120_gb300.build import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build()


def _rows(rng, n, k, spread):
    """Gaussian rows scaled by 2^u, u uniform in [-spread, spread]; row 0 is
    zero and row 1 has one entry 2^20 times the others when n > 2."""
    x = rng.standard_normal((n, k)) * np.exp2(rng.uniform(-spread, spread, size=(n, 1)))
    if n > 2:
        x[0] = 0.0
        x[1, k // 2] *= 2.0 ** 20
    return x


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (5, 7, 33), (128, 128, 64), (200, 300, 1000), (130, 129, 4096),
                                   (64, 96, 5000), (40, 50, 20000), (300, 17, 16384)])
def test_gemm_f64_tc_matches_extended_precision(M, N, K):
    """Error against the product in long double: of the order of an FP64
    dot product's, bounded here by 2^-48 sqrt(K) max|a_i.| max|b_j.| (the
    digit slicing keeps 54 bits of each row relative to its largest entry)."""
    import torch
    rng = np.random.default_rng(M * 1000 + N + K)
    A = _rows(rng, M, K, 30)
    B = _rows(rng, N, K, 30)
    C = binding.lc_gemm_f64_tc(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    ref = (A.astype(np.longdouble) @ B.astype(np.longdouble).T)
    err = np.abs(C.astype(np.longdouble) - ref).astype(np.float64)
    bound = 2.0 ** -48 * np.sqrt(K) * np.outer(np.abs(A).max(axis=1), np.abs(B).max(axis=1))
    assert np.all(err <= bound + 1e-300)
    if M > 2:
        assert np.all(C[0] == 0.0)


def test_gemm_f64_tc_exact_on_small_integers():
    """Integer entries small enough for every product and sum to be exact
    give the exact product."""
    import torch
    rng = np.random.default_rng(3)
    A = rng.integers(-1000, 1000, size=(257, 777)).astype(np.float64)
    B = rng.integers(-1000, 1000, size=(129, 777)).astype(np.float64)
    C = binding.lc_gemm_f64_tc(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    assert np.array_equal(C, A @ B.T)


def _random_su_state(d, n0, seed):
    """n0 orthonormal elements of su(d): orthonormal mixes (QR of a Gaussian
    matrix) of the d^2 - 1 non-identity Pauli strings."""
    n = int(np.log2(d))
    rng = np.random.default_rng(seed)
    labels = ["".join("IXYZ"[(s >> (2 * q)) & 3] for q in range(n)) for s in range(1, 4 ** n)]
    P = inputs.generators_from_labels(labels)
    Q, _ = np.linalg.qr(rng.standard_normal((d * d - 1, n0)))
    flat = P.reshape(d * d - 1, d * d)
    return (Q.T @ flat.real + 1j * (Q.T @ flat.imag)).reshape(n0, d, d)


def test_closure_with_tc_projections_matches_fp64_gemms_and_oracle():
    """Resumed from a dense 2000-element orthonormal state at d = 64 (rows of
    4096 components) at the pair (1500, 0), 300 candidates, mixed mode: the
    flagged rows' projections run on the tensor-core FP64 GEMM (reported);
    every accepted element equals the oracle's and the FP64-SIMT-GEMM run's."""
    d, n0 = 64, 2000
    V0 = _random_su_state(d, n0, seed=64)
    g = inputs.random_set(d, 2, seed=1)
    state = oc.Alg4Result(V=np.concatenate([V0, np.zeros((400, d, d), np.complex128)]), dim=n0, l=1500, m=0,
                          max_dim=4095)
    ref = oc.alg4_orthonormalization(g, 1e-8, resume=state, max_candidates=300)
    a = binding.lie_closure_resume(V0, (1500, 0), 1e-8, precision="mixed", max_candidates=300, max_dim=2400,
                                   ortho_check=1)
    assert a.report["accept_tc_gemms"] > 0
    assert a.dim == ref.dim > n0
    np.testing.assert_allclose(a.basis, ref.basis, atol=1e-11, rtol=0)
    assert a.report["ortho_defect"] < 1e-12
    b = binding.lie_closure_resume(V0, (1500, 0), 1e-8, precision="mixed", max_candidates=300, max_dim=2400,
                                   accept_gemm=1)
    assert b.report["accept_tc_gemms"] == 0
    assert b.dim == a.dim
    np.testing.assert_allclose(a.basis, b.basis, atol=1e-11, rtol=0)


def test_su64_chain_and_su128_growth_with_tc_projections():
    """Full su(64) chain closure (4095) and the su(128) random pair to its
    saturation exit (16383), both with the tensor-core projections: closed-form
    dimensions and FP64-level orthonormality (device Gram)."""
    g, _ = inputs.workload_generators("su64_chain_d64")
    r = binding.lie_closure(g, 1e-8, precision="mixed", ortho_check=1)
    assert r.dim == 4095 and r.report["ortho_defect"] < 1e-12
    g, _ = inputs.workload_generators("su128_random2_d128")
    r = binding.lie_closure(g, 1e-8, precision="mixed", saturation_exit=1, ortho_check=1, return_basis=False)
    assert r.dim == 16383
    assert r.report["accept_tc_gemms"] > 0
    assert r.report["ortho_defect"] < 1e-12


def test_su128_prefix_panel_projections_match_fp64_gemms():
    """su(128) random pair, first 12000 candidates (growth blocks of 1024 with
    hundreds of accepts each, decided in panels of 128 rows): with the
    tensor-core projections, including those of each panel's accepts out of
    the later rows, the basis equals the FP64-SIMT-GEMM run's."""
    g, _ = inputs.workload_generators("su128_random2_d128")
    a = binding.lie_closure(g, 1e-8, precision="mixed", max_candidates=12000, max_dim=16384)
    b = binding.lie_closure(g, 1e-8, precision="mixed", max_candidates=12000, max_dim=16384, accept_gemm=1)
    assert a.report["accept_tc_gemms"] > 0 and b.report["accept_tc_gemms"] == 0
    assert a.dim == b.dim > 1000
    np.testing.assert_allclose(a.basis, b.basis, atol=1e-11, rtol=0)
