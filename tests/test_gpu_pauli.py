"""GPU parity of the sparse Pauli-sum path (``lie_closure_pauli``) against the
CPU oracle.

The oracle runs Algorithm 4 on the dense d x d matrices of the same
generators; the GPU path never forms a matrix.  Bars:
* dimension: exact;
* elements: each GPU element, turned into its matrix, equals the oracle's
  element of the same index within 1e-11 (same pair order, same FP64 test);
* single-string sets: every element is one string with coefficient exactly
  +-1, and the set of strings equals the exact Pauli closure (O3);
* the basis is orthonormal in the coefficient inner product within 1e-12.
"""
import json
import os

import numpy as np
import pytest

import oracle.closure as oc
from paper_2506_01120_gb300 import binding, inputs
from paper_2506_01120_gb300.build import build

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_dims.json")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    build()
    return binding.lib()


def run(ops, n, tol, **kw):
    s, c, o = inputs.pauli_sum_terms(ops)
    return binding.lie_closure_pauli(s, c, o, n, tol, **kw)


def matrices(res, n):
    out = []
    for i in range(res.dim):
        op = [(binding.pauli_label(s, n), c) for s, c in res.element(i)]
        out.append(inputs.pauli_sum_matrix(op, n))
    return np.stack(out) if out else np.zeros((0, 2 ** n, 2 ** n), dtype=np.complex128)


def dense(ops, n):
    return np.stack([inputs.pauli_sum_matrix(op, n) for op in ops])


def coeff_gram(res):
    D = res.dim
    rows = [dict(res.element(i)) for i in range(D)]
    G = np.zeros((D, D))
    for i in range(D):
        for j in range(i + 1):
            common = rows[i].keys() & rows[j].keys()
            G[i, j] = G[j, i] = sum(rows[i][s] * rows[j][s] for s in common)
    return G


def check_elementwise(res, ops, n, tol, **okw):
    ref = oc.alg4_orthonormalization(dense(ops, n), tol, **okw)
    # parity is only defined where no FP64 decision sits near tol (the oracle's
    # margin report); near-commuting pairs of random sums can put one there
    m = oc.margin_report(ref)
    assert m["min_acc_rel_res"] > 10 * tol and m["max_rej_rel_res"] < tol / 10, m
    assert res.dim == ref.dim
    if res.dim:
        np.testing.assert_allclose(matrices(res, n), ref.basis, atol=1e-11, rtol=0)
        assert np.abs(coeff_gram(res) - np.eye(res.dim)).max() < 1e-12
    return ref


def labels_ops(labels):
    return [[(l, 1.0)] for l in labels]


# ------------------------------------------------------------ elementwise parity
@pytest.mark.parametrize("n", [2, 3])
def test_hea_chain_matches_oracle_elementwise(n):
    ops = labels_ops(inputs.su2n_chain_labels(n))
    res = run(ops, n, 1e-10)
    check_elementwise(res, ops, n, 1e-10)
    assert res.dim == 4 ** n - 1
    D = res.dim
    assert res.report["brackets_checked"] == D * (D - 1) // 2


@pytest.mark.parametrize("n", [3, 4])
def test_so2n_chain_matches_oracle_elementwise(n):
    ops = labels_ops(inputs.so2n_chain_labels(n))
    res = run(ops, n, 1e-10)
    check_elementwise(res, ops, n, 1e-10)
    assert res.dim == n * (2 * n - 1)          # Jordan-Wigner: so(2n)


@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_tfim_sums_match_oracle_elementwise(n):
    """Multi-term generators: sum_j X_j and sum_j Z_j Z_{j+1}."""
    ops = inputs.tfim_ops(n)
    res = run(ops, n, 1e-10)
    check_elementwise(res, ops, n, 1e-10)


@pytest.mark.parametrize("n,k,terms,seed,sat", [(3, 2, 3, 5, False), (3, 3, 2, 2, False), (4, 2, 2, 7, False),
                                                (4, 3, 2, 8, False), (5, 3, 2, 10, False), (3, 2, 4, 6, True),
                                                (4, 2, 4, 13, True), (4, 2, 6, 15, True)])
def test_random_sums_match_oracle_elementwise(n, k, terms, seed, sat):
    """Random sums on both sides with the oracle's documented floor for Pauli
    sums (oc.ETA_ABS_PAULI_SUMS = 1e-9): chains of accepts with small relative
    residuals amplify the dense oracle's rounding, and a bracket that is zero
    can come out near 1e-11 there."""
    ops = inputs.random_pauli_sums(n, k, terms, seed)
    eta = oc.ETA_ABS_PAULI_SUMS
    res = run(ops, n, 1e-8, saturation_exit=int(sat), eta_abs=eta)
    check_elementwise(res, ops, n, 1e-8, saturation_exit=sat, eta_abs=eta)


def test_structural_zero_brackets_stay_zero():
    """Random 3-term sums on 4 qubits (seed 14) close to a 36-dimensional
    algebra.  The dense FP64 oracle at its default floor eta_abs = 1e-12 forms
    the zero bracket of elements 35 and 0 as ~1.7e-11 (rounding compounded
    through accepts with relative residuals ~1e-3) and accepts it, after which
    noise fills su(16) (dim 255).  The sparse path multiplies only the strings
    present, gets that bracket below the floor and keeps dim 36, which is what
    the oracle returns once its floor (1e-9) clears the compounded rounding."""
    ops = inputs.random_pauli_sums(4, 2, 3, 14)
    res = run(ops, 4, 1e-8, saturation_exit=1)
    assert res.dim == 36
    ref = oc.alg4_orthonormalization(dense(ops, 4), 1e-8, eta_abs=oc.ETA_ABS_PAULI_SUMS, saturation_exit=True)
    assert ref.dim == 36
    # the oracle's later elements carry that compounded rounding (~2e-11)
    np.testing.assert_allclose(matrices(res, 4), ref.basis, atol=1e-9, rtol=0)


def test_regrown_tables_give_the_same_basis():
    """The accept warp's tables start at their smallest size (test hook) and
    regrow; the result equals the default run's."""
    ops = inputs.random_pauli_sums(4, 2, 6, 15)
    a = run(ops, 4, 1e-8, saturation_exit=1)
    b = run(ops, 4, 1e-8, saturation_exit=1, fault_inject=2)
    assert a.dim == b.dim == 136
    np.testing.assert_array_equal(a.offsets, b.offsets)
    np.testing.assert_array_equal(a.strings, b.strings)
    np.testing.assert_allclose(a.coefs, b.coefs, atol=1e-13)


# ------------------------------------------------------------ exact closures
@pytest.mark.parametrize("n,k,seed", [(3, 4, 1), (4, 6, 2), (5, 8, 3), (6, 8, 4), (8, 10, 5), (10, 12, 6),
                                      (12, 12, 7)])
def test_single_string_sets_equal_exact_closure(n, k, seed):
    rng = np.random.default_rng(seed)
    labels = inputs.random_pauli_labels(n, k, rng)
    res = run(labels_ops(labels), n, 1e-8)
    ref = oc.pauli_closure(labels)
    assert res.dim == len(ref)
    np.testing.assert_array_equal(np.diff(res.offsets), 1)
    assert np.all(np.abs(res.coefs) == 1.0)
    got = {binding.pauli_label(s, n) for s in res.strings}
    assert got == set(ref)


@pytest.mark.parametrize("n", [6, 7])
def test_hea_full_size(n):
    """The hardware-efficient-ansatz generators of Table 2 (iX_j, iY_j,
    iZ_jZ_{j+1}): su(2^n), every element one distinct non-identity string with
    coefficient +-1, every pair of the final basis checked."""
    res = run(labels_ops(inputs.su2n_chain_labels(n)), n, 1e-8)
    D = 4 ** n - 1
    with open(GOLDEN) as fh:
        t2 = json.load(fh)["table2_hea_sparse"]
    assert t2["dim"][t2["n"].index(n)] == D          # the dimensions Table 2 prints
    assert res.dim == D
    assert res.status == binding.LC_OK
    assert res.report["brackets_checked"] == D * (D - 1) // 2
    np.testing.assert_array_equal(np.diff(res.offsets), 1)
    assert np.all(np.abs(res.coefs) == 1.0)
    assert len(set(res.strings.tolist())) == D and 0 not in set(res.strings.tolist())


@pytest.mark.parametrize("n", [6, 10, 20])
def test_so2n_chain_dimension(n):
    res = run(labels_ops(inputs.so2n_chain_labels(n)), n, 1e-10, max_dim=1024)
    assert res.dim == n * (2 * n - 1)


# ------------------------------------------------------------ edge cases
def test_degenerate_generator_sets():
    z = run([[("XY", 0.0)], [("ZZ", 0.0)]], 2, 1e-8)
    assert z.dim == 0 and z.status == binding.LC_OK
    one = run([[("XY", 2.5)]], 2, 1e-8)
    assert one.dim == 1 and one.element(0) == [(inputs.pauli_string("XY"), 1.0)]
    comm = run(labels_ops(["ZII", "IZI", "ZZI", "IIZ"]), 3, 1e-8)
    assert comm.dim == 4
    dup = run([[("XI", 1.0)], [("XI", -2.5)], [("IZ", 1.0)]], 2, 1e-8)
    assert dup.dim == 2
    summed = run([[("XX", 1.0), ("XX", 1.0)]], 2, 1e-8)      # repeated string inside one generator
    assert summed.dim == 1 and summed.element(0) == [(inputs.pauli_string("XX"), 1.0)]
    ident = run([[("II", 1.0)], [("XI", 1.0)], [("YI", 1.0)]], 2, 1e-8)
    assert ident.dim == 4                                     # u(1) + su(2) on qubit 1


def test_errors():
    s, c, o = inputs.pauli_sum_terms([[("XY", 1.0)], [("ZZ", 1.0)]])
    bad = s.copy()
    bad[0] |= np.uint64(1 << 5)                               # a qubit outside n = 2
    assert binding.lie_closure_pauli(bad, c, o, 2, 1e-8, check=False).status == binding.LC_ERR_ARG
    nan = c.copy()
    nan[1] = np.nan
    assert binding.lie_closure_pauli(s, nan, o, 2, 1e-8, check=False).status == binding.LC_ERR_NONFINITE


def test_capacity_keeps_the_prefix():
    ops = labels_ops(inputs.su2n_chain_labels(3))
    full = run(ops, 3, 1e-10)
    part = run(ops, 3, 1e-10, max_dim=10, check=False)
    assert part.status == binding.LC_ERR_CAPACITY and part.dim == 10
    np.testing.assert_array_equal(part.strings, full.strings[:10])
    tcap = run(inputs.tfim_ops(4), 4, 1e-10, term_capacity=12, check=False)
    assert tcap.status == binding.LC_ERR_CAPACITY
    ref = run(inputs.tfim_ops(4), 4, 1e-10)
    assert tcap.dim >= 1 and tcap.offsets[-1] <= 12
    np.testing.assert_array_equal(tcap.offsets, ref.offsets[:tcap.dim + 1])


def test_max_candidates_cursor_matches_oracle():
    ops = labels_ops(inputs.su2n_chain_labels(3))
    ref = oc.alg4_orthonormalization(dense(ops, 3), 1e-10, max_candidates=500)
    res = run(ops, 3, 1e-10, max_candidates=500, block_k=64)
    assert res.report["brackets_checked"] == 500
    assert (res.report["cursor_l"], res.report["cursor_m"]) == (ref.l, ref.m)
    assert res.dim == ref.dim
    np.testing.assert_allclose(matrices(res, 3), ref.basis, atol=1e-12)


def test_block_size_does_not_change_the_result():
    ops = inputs.random_pauli_sums(4, 3, 2, 8)
    a = run(ops, 4, 1e-8, block_k=7)
    b = run(ops, 4, 1e-8)
    assert a.dim == b.dim
    np.testing.assert_array_equal(a.strings, b.strings)
    np.testing.assert_allclose(a.coefs, b.coefs, atol=1e-13)


def test_dev_api_matches_host_api():
    import torch
    ops = inputs.tfim_ops(5)
    host = run(ops, 5, 1e-10)
    s, c, o = inputs.pauli_sum_terms(ops)
    ds = torch.from_numpy(s.view(np.int64)).cuda()
    dc = torch.from_numpy(c).cuda()
    do = torch.from_numpy(o).cuda()
    cap, tcap = 64, 4096
    bs = torch.zeros(tcap, dtype=torch.int64, device="cuda")
    bc = torch.zeros(tcap, dtype=torch.float64, device="cuda")
    bo = torch.zeros(cap + 1, dtype=torch.int64, device="cuda")
    r = binding.lie_closure_pauli_dev(ds, dc, do, 5, 1e-10, cap, tcap, bs, bc, bo)
    assert r.dim == host.dim
    off = bo[:r.dim + 1].cpu().numpy()
    np.testing.assert_array_equal(off, host.offsets)
    np.testing.assert_array_equal(bs[:off[-1]].cpu().numpy().view(np.uint64), host.strings)
    np.testing.assert_allclose(bc[:off[-1]].cpu().numpy(), host.coefs, atol=1e-13)
