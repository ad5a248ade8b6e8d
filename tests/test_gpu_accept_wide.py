"""GPU parity of the accept path's alternatives against the oracle, through
the C ABI: the row-sliced in-block accept kernel (k_accept_wide, option
accept_kernel = 2) and the first projection taken from the screening GEMM's
coefficients (default in mixed mode, off with fp64_first_pass).

The sliced kernel takes the in-block decisions of Algorithm 4 in the same
order as the one-CTA-per-row kernel; only the order of the FP64 partial sums
of its dot products differs.  Forced on small cases (many accepts per panel
of 128 rows, several groups of 8 rows, ragged last group) it must return the
oracle's basis element by element, in both precisions and for Algorithm 3; its
bounded grid barrier must report a timeout without losing the device; the
capacity stop must keep the oracle's first max_dim elements; and at d = 1024
the default choice must take it.
"""
import numpy as np
import pytest

import oracle.closure as oc
from paper_2506_01120_gb300 import binding, inputs
from paper_2506_01120_gb300.build import build

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "mixed"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build()


def _case(name):
    """(generators, tol, candidate prefix or None for the whole sweep), sized so
    the oracle finishes in seconds"""
    if name == "so6":
        return inputs.generators_from_labels(inputs.so2n_chain_labels(3)), 1e-10, None
    if name == "su32_prefix":
        return inputs.generators_from_labels(inputs.su2n_chain_labels(5)), 1e-10, 1500
    if name == "rand_d8":
        return inputs.random_set(8, 2, seed=6), 1e-8, None
    if name == "rand_d16_prefix":
        return inputs.random_set(16, 2, seed=6), 1e-8, 3000
    return inputs.random_set(6, 3, seed=13), 1e-8, None


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["so6", "su32_prefix", "rand_d8", "rand_d16_prefix", "rand_d6_k3"])
def test_sliced_accept_matches_oracle(prec, name):
    g, tol, ncand = _case(name)
    kw = {} if ncand is None else {"max_candidates": ncand}
    ref = oc.alg4_orthonormalization(g, tol, **kw)
    w = binding.lie_closure(g, tol, precision=prec, accept_kernel=2, **kw)
    assert w.report["accept_wide_launches"] > 0
    assert w.dim == ref.dim
    np.testing.assert_allclose(w.basis, ref.basis, atol=1e-11, rtol=0)
    assert oc.ortho_defect(w.basis) < 1e-12
    # the two kernels sum the dot products in other orders: elements accepted
    # with a small residual near saturation amplify that rounding (1e-13 seen)
    r = binding.lie_closure(g, tol, precision=prec, accept_kernel=1, **kw)
    assert r.report["accept_wide_launches"] == 0
    assert r.dim == w.dim
    np.testing.assert_allclose(w.basis, r.basis, atol=1e-11, rtol=0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["su8", "rand_d6_k3"])
def test_sliced_accept_alg3_matches_oracle(prec, name):
    if name == "su8":
        g, tol = inputs.generators_from_labels(inputs.su2n_chain_labels(3)), 1e-10
    else:
        g, tol, _ = _case(name)
    ref = oc.alg3_orthonormalization(g, tol)
    B, V, st, rep = binding.lie_closure_alg3(g, tol, precision=prec, accept_kernel=2)
    assert st == binding.LC_OK and B.shape[0] == V.shape[0] == ref.dim
    assert rep["accept_wide_launches"] > 0
    scale = np.max(np.abs(ref.B), axis=(1, 2), keepdims=True)
    np.testing.assert_array_less(np.abs(B - ref.B) / scale, 1e-12)
    np.testing.assert_allclose(V, ref.V, atol=1e-11)


def test_sliced_accept_capacity_stop():
    g = inputs.random_set(4, 2, seed=5)
    ref = oc.alg4_orthonormalization(g, 1e-8)
    for prec in PRECS:
        r = binding.lie_closure(g, 1e-8, max_dim=10, check=False, precision=prec, accept_kernel=2)
        assert r.status == binding.LC_ERR_CAPACITY
        assert r.dim == 10
        np.testing.assert_allclose(r.basis, ref.basis[:10], atol=1e-12)


def test_sliced_accept_timeout_is_reported_and_device_stays_usable():
    """The first grid barrier is told to expect one arrival more than there
    are CTAs; the bounded wait runs out, LC_ERR_TIMEOUT comes back, and the
    next call works."""
    g = inputs.generators_from_labels(inputs.su2n_chain_labels(3))
    for prec in PRECS:
        r = binding.lie_closure(g, 1e-10, precision=prec, fault_inject=1, spin_cap=50_000_000, check=False,
                                accept_kernel=2)
        assert r.status == binding.LC_ERR_TIMEOUT
        ok = binding.lie_closure(g, 1e-10, precision=prec, accept_kernel=2)
        assert ok.status == binding.LC_OK and ok.dim == 63


def test_bad_accept_kernel_is_an_argument_error():
    g = inputs.generators_from_labels(inputs.su2n_chain_labels(2))
    r = binding.lie_closure(g, 1e-10, accept_kernel=4, check=False)
    assert r.status == binding.LC_ERR_ARG


def test_default_takes_sliced_kernel_for_long_rows():
    """so(20) at d = 1024 (rows of 2^20 doubles): the default choice runs the
    sliced kernel, and an 80-candidate prefix equals the one-CTA-per-row run
    and the oracle's prefix."""
    g, _ = inputs.workload_generators("so20_chain_d1024")
    a = binding.lie_closure(g, 1e-8, precision="mixed", max_candidates=80, max_dim=190)
    assert a.report["accept_wide_launches"] > 0
    b = binding.lie_closure(g, 1e-8, precision="mixed", max_candidates=80, max_dim=190, accept_kernel=1)
    assert b.report["accept_wide_launches"] == 0
    assert a.dim == b.dim
    np.testing.assert_allclose(a.basis, b.basis, atol=1e-11, rtol=0)
    ref = oc.alg4_orthonormalization(g, 1e-8, max_candidates=80)
    assert a.dim == ref.dim
    np.testing.assert_allclose(a.basis, ref.basis, atol=1e-11, rtol=0)


def test_sliced_accept_dense_d256_prefix():
    """Dense rows of 2^16 doubles, most candidates accepted (random traceless
    pair at d = 256, first 60 candidates): the forced sliced kernel against
    the oracle's prefix."""
    g = inputs.random_set(256, 2, seed=256)
    ref = oc.alg4_orthonormalization(g, 1e-8, max_candidates=60)
    a = binding.lie_closure(g, 1e-8, precision="mixed", max_candidates=60, max_dim=128, accept_kernel=2)
    assert a.report["accept_wide_launches"] > 0
    assert a.dim == ref.dim > 40
    np.testing.assert_allclose(a.basis, ref.basis, atol=1e-11, rtol=0)


# ------------------------------------------------ first projection from the screen
@pytest.mark.parametrize("name", ["rand_d8", "rand_d16_prefix", "rand_d6_k3"])
def test_screen_coefficient_first_pass_matches_oracle(name):
    """Mixed mode, blocks whose flagged rows need a second Gram-Schmidt pass
    (screened rho^2 < 1/2, i.e. more than half of the space spanned) take
    the screening GEMM's coefficients as the first projection and one FP64
    pass after it; the basis is the oracle's element by element and the same
    as with the FP64 first pass (option fp64_first_pass).  (Pauli-string sets
    never take it: their flagged rows have rho = 1.)"""
    g, tol, ncand = _case(name)
    kw = {} if ncand is None else {"max_candidates": ncand}
    ref = oc.alg4_orthonormalization(g, tol, **kw)
    a = binding.lie_closure(g, tol, precision="mixed", ortho_check=1, **kw)
    assert a.report["screen_pass1_blocks"] > 0
    assert a.dim == ref.dim
    np.testing.assert_allclose(a.basis, ref.basis, atol=1e-11, rtol=0)
    assert a.report["ortho_defect"] < 1e-12
    b = binding.lie_closure(g, tol, precision="mixed", fp64_first_pass=1, **kw)
    assert b.report["screen_pass1_blocks"] == 0
    assert b.dim == a.dim
    np.testing.assert_allclose(a.basis, b.basis, atol=1e-11, rtol=0)


def test_fp64_mode_never_takes_screen_coefficients():
    g, tol, ncand = _case("rand_d16_prefix")
    r = binding.lie_closure(g, tol, precision="fp64", max_candidates=ncand)
    assert r.report["screen_pass1_blocks"] == 0


# ------------------------------------------------ rows held in shared memory
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["so6", "rand_d8", "rand_d16_prefix", "rand_d6_k3"])
def test_rowsmem_accept_identical_to_row_per_cta(prec, name):
    """accept_kernel = 3 (each later row kept in its CTA's shared memory,
    fused sweeps) computes k_accept_seq's values in k_accept_seq's order:
    the basis is bit-identical to accept_kernel = 1's and equals the
    oracle's."""
    g, tol, ncand = _case(name)
    kw = {} if ncand is None else {"max_candidates": ncand}
    a = binding.lie_closure(g, tol, precision=prec, accept_kernel=3, **kw)
    b = binding.lie_closure(g, tol, precision=prec, accept_kernel=1, **kw)
    assert a.dim == b.dim
    np.testing.assert_array_equal(a.basis, b.basis)
    ref = oc.alg4_orthonormalization(g, tol, **kw)
    assert a.dim == ref.dim
    np.testing.assert_allclose(a.basis, ref.basis, atol=1e-11, rtol=0)


def test_rowsmem_accept_alg3_capacity_and_timeout():
    g, tol = inputs.generators_from_labels(inputs.su2n_chain_labels(3)), 1e-10
    ref = oc.alg3_orthonormalization(g, tol)
    B, V, st, rep = binding.lie_closure_alg3(g, tol, precision="mixed", accept_kernel=3)
    assert st == binding.LC_OK and B.shape[0] == ref.dim
    np.testing.assert_allclose(V, ref.V, atol=1e-11)
    g4 = inputs.random_set(4, 2, seed=5)
    ref4 = oc.alg4_orthonormalization(g4, 1e-8)
    r = binding.lie_closure(g4, 1e-8, max_dim=10, check=False, precision="mixed", accept_kernel=3)
    assert r.status == binding.LC_ERR_CAPACITY and r.dim == 10
    np.testing.assert_allclose(r.basis, ref4.basis[:10], atol=1e-12)
    r = binding.lie_closure(g, 1e-10, precision="mixed", fault_inject=1, spin_cap=50_000_000, check=False,
                            accept_kernel=3)
    assert r.status == binding.LC_ERR_TIMEOUT
    ok = binding.lie_closure(g, 1e-10, precision="mixed", accept_kernel=3)
    assert ok.status == binding.LC_OK and ok.dim == 63
