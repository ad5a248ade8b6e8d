"""Random generator sets whose closure is a proper subalgebra of su(d).

so(d) (two random real antisymmetric generators) and su(d/2) + su(d/2) (two
random block-diagonal generators) close far below d^2 - 1, so the saturation
exit never fires and every candidate goes through the screen: a screen that
rejected an independent candidate it should have flagged would lose a
dimension or change the span.  At d = 16 the GPU bases are compared with the
oracle's element by element; at d = 64 (tensor-core brackets) the dimension
is compared with the closed forms d(d-1)/2 and 2((d/2)^2 - 1), the span with
the canonical basis of the subalgebra (sin of the largest principal angle
<= 1e-6, the mixed-precision bar), and a candidate prefix with the oracle.
"""
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


def _so_basis(d):
    """Orthonormal basis of so(d) under tr(a^dagger b)/d: sqrt(d/2) (E_jk - E_kj)."""
    out = []
    for j in range(d):
        for k in range(j + 1, d):
            a = np.zeros((d, d), dtype=np.complex128)
            a[j, k], a[k, j] = 1.0, -1.0
            out.append(np.sqrt(d / 2.0) * a)
    return np.stack(out)


def _block_su_basis(d):
    """Orthonormal basis of su(d/2) + su(d/2): sqrt(2) i P_s in each diagonal
    block for the non-identity Pauli strings P_s on log2(d/2) qubits."""
    h = d // 2
    n = int(np.log2(h))
    labels = ["".join("IXYZ"[(s >> (2 * q)) & 3] for q in range(n)) for s in range(1, 4 ** n)]
    P = inputs.generators_from_labels(labels)
    out = []
    for blk in range(2):
        for p in P:
            a = np.zeros((d, d), dtype=np.complex128)
            a[blk * h:(blk + 1) * h, blk * h:(blk + 1) * h] = np.sqrt(2.0) * p
            out.append(a)
    return np.stack(out)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kind,dim", [("so", 120), ("block", 126)])
def test_subalgebra_d16_matches_oracle(prec, kind, dim):
    g = inputs.random_subalgebra_set(kind, 16, 2, seed=5)
    ref = oc.alg4_orthonormalization(g, 1e-8)
    res = binding.lie_closure(g, 1e-8, precision=prec)
    assert res.dim == ref.dim == dim
    np.testing.assert_allclose(res.basis, ref.basis, atol=1e-11, rtol=0)


@pytest.mark.parametrize("kind", ["so", "block"])
def test_subalgebra_d64_closed_form_and_span(kind):
    d = 64
    g = inputs.random_subalgebra_set(kind, d, 2, seed=64)
    res = binding.lie_closure(g, 1e-8, precision="mixed", ortho_check=1)
    want = d * (d - 1) // 2 if kind == "so" else 2 * ((d // 2) ** 2 - 1)
    assert res.dim == want
    rep = res.report
    assert rep["brackets_checked"] == want * (want - 1) // 2
    assert rep["ortho_defect"] < 1e-12
    U = _so_basis(d) if kind == "so" else _block_su_basis(d)
    assert oc.span_distance(res.basis, U) < 1e-6
    assert rep["min_acc_screen_rel_res"] > rep["tau_screen"]
    # the same sets on a candidate prefix, element by element with the oracle
    ref = oc.alg4_orthonormalization(g, 1e-8, max_candidates=600)
    pre = binding.lie_closure(g, 1e-8, precision="mixed", max_candidates=600, max_dim=1024)
    assert pre.dim == ref.dim
    np.testing.assert_allclose(pre.basis, ref.basis, atol=1e-11, rtol=0)


@pytest.mark.parametrize("kind,d,ncand", [("so", 128, 200), ("block", 128, 200), ("so", 256, 60)])
def test_subalgebra_prefix_large_d(kind, d, ncand):
    """Subalgebra sets at d = 128 (k_bracket_tc<128>) and d = 256
    (k_bracket_big): a candidate prefix element by element with the oracle
    (their full closures, 8128 and more elements, are beyond the oracle)."""
    g = inputs.random_subalgebra_set(kind, d, 2, seed=d + 1)
    ref = oc.alg4_orthonormalization(g, 1e-8, max_candidates=ncand)
    res = binding.lie_closure(g, 1e-8, precision="mixed", max_candidates=ncand, max_dim=512)
    assert res.dim == ref.dim
    np.testing.assert_allclose(res.basis, ref.basis, atol=1e-11, rtol=0)
    if kind == "so":                      # every element real antisymmetric (inside so(d))
        assert np.max(np.abs(res.basis.imag)) < 1e-12
