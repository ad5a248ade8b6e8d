"""Element-by-element oracle parity of the tensor-core bracket kernels.

The mixed path forms brackets on the tensor cores for d = 32
(k_bracket_tc<32>), d = 64 (k_bracket_q64), d = 128 (k_bracket_tc<128>) and
d >= 256 (k_bracket_big).  Full closures at
those sizes are out of the oracle's reach, so these tests stop both sides
after the same number of bracket candidates (the pair order is the same, so
the two runs check the same candidates) and compare the bases element by
element within 1e-11: every accepted element is an FP64 result on the GPU,
so the screen must pass every candidate the oracle accepts and reject only
candidates the oracle rejects.  A second form resumes both sides from one
orthonormal state built here (a random orthonormal mix of Pauli strings) to
check a window deep into a large basis.
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


def _prefix_case(g, tol, ncand, max_dim):
    ref = oc.alg4_orthonormalization(g, tol, max_candidates=ncand)
    res = binding.lie_closure(g, tol, precision="mixed", max_candidates=ncand, max_dim=max_dim)
    assert res.report["brackets_checked"] == ncand
    assert (res.report["cursor_l"], res.report["cursor_m"]) == (ref.l, ref.m)
    assert res.dim == ref.dim
    np.testing.assert_allclose(res.basis, ref.basis, atol=1e-11, rtol=0)
    assert oc.ortho_defect(res.basis) < 1e-12
    return res, ref


def test_random_pair_d32_to_saturation():
    """k_bracket_tc<32> (M = 64 shape, half its rows used): a random traceless
    pair at d = 32 to su(32) (1023) with the saturation exit on both sides,
    every element compared."""
    g = inputs.random_set(32, 2, seed=32)
    ref = oc.alg4_orthonormalization(g, 1e-8, saturation_exit=True)
    res = binding.lie_closure(g, 1e-8, precision="mixed", saturation_exit=1)
    assert res.dim == ref.dim == 1023
    np.testing.assert_allclose(res.basis, ref.basis, atol=1e-11, rtol=0)


def test_prefix_su32_chain_d32():
    """k_bracket_tc<32> on the Pauli chain (zero and duplicate brackets)."""
    g = inputs.generators_from_labels(inputs.su2n_chain_labels(5))
    _prefix_case(g, 1e-8, 4000, 1023)


def test_prefix_random_pair_d64():
    """k_bracket_q64: a random traceless pair at d = 64 for 700 candidates
    (every accepted element checked against the oracle's)."""
    g = inputs.random_set(64, 2, seed=77)
    res, ref = _prefix_case(g, 1e-8, 700, 1024)
    assert res.dim > 500          # growth phase: nearly every bracket independent
    assert res.report["n_flagged"] >= res.dim - 2


def test_prefix_su64_chain_d64():
    """k_bracket_q64 on the Pauli chain: zero brackets (commuting strings) and
    duplicates mixed with new strings."""
    g, _ = inputs.workload_generators("su64_chain_d64")
    res, ref = _prefix_case(g, 1e-8, 3000, 4095)
    assert res.report["n_nonzero"] < res.report["brackets_checked"]


def test_prefix_random_pair_d128():
    """k_bracket_tc<128> on the su(128) workload's generators (seed 2506)."""
    g, _ = inputs.workload_generators("su128_random2_d128")
    res, ref = _prefix_case(g, 1e-8, 250, 512)
    assert res.dim > 150


def test_prefix_so16_chain_d256():
    """k_bracket_big at d = 256: the so(16) chain, first 900 candidates."""
    g = inputs.generators_from_labels(inputs.so2n_chain_labels(8))
    _prefix_case(g, 1e-8, 900, 160)


def test_prefix_random_pair_d256():
    """k_bracket_big with dense operands (random traceless pair, d = 256)."""
    g = inputs.random_set(256, 2, seed=256)
    res, _ = _prefix_case(g, 1e-8, 60, 128)
    assert res.dim > 40


def test_prefix_so20_chain_d1024():
    """k_bracket_big at d = 1024 (the so(20) workload), first 80 candidates."""
    g, _ = inputs.workload_generators("so20_chain_d1024")
    _prefix_case(g, 1e-8, 80, 190)


def _random_su_state(d, n0, seed):
    """n0 orthonormal elements of su(d): a random mix of the d^2 - 1 non-identity
    Pauli strings with orthonormal mixing rows (QR of a Gaussian matrix), so
    the elements are dense and orthonormal under <a, b> = tr(a^dagger b)/d."""
    n = int(np.log2(d))
    rng = np.random.default_rng(seed)
    labels = ["".join("IXYZ"[(s >> (2 * q)) & 3] for q in range(n)) for s in range(1, 4 ** n)]
    P = inputs.generators_from_labels(labels)                  # i * string, (d^2 - 1, d, d)
    Q, _ = np.linalg.qr(rng.standard_normal((d * d - 1, n0)))
    flat = P.reshape(d * d - 1, d * d)
    return (Q.T @ flat.real + 1j * (Q.T @ flat.imag)).reshape(n0, d, d)


def test_resumed_window_deep_in_su64():
    """Both sides resume from the same 2000-element orthonormal state (not a
    subalgebra, so brackets leave its span) at the pair (1500, 0) and check
    the next 80 candidates: screening GEMMs over a 2000-row basis, eight
    256-wide N tiles, and every accept compared element by element."""
    d, n0 = 64, 2000
    V0 = _random_su_state(d, n0, seed=64)
    assert oc.ortho_defect(V0) < 1e-13
    g = inputs.random_set(d, 2, seed=1)               # only the saturation bound reads these
    state = oc.Alg4Result(V=np.concatenate([V0, np.zeros((200, d, d), np.complex128)]), dim=n0, l=1500, m=0,
                          max_dim=4095)
    ref = oc.alg4_orthonormalization(g, 1e-8, resume=state, max_candidates=80)
    res = binding.lie_closure_resume(V0, (1500, 0), 1e-8, precision="mixed", max_candidates=80, max_dim=2200)
    assert res.dim == ref.dim > n0
    np.testing.assert_allclose(res.basis, ref.basis, atol=1e-11, rtol=0)
