"""GPU parity at full workload sizes, through properties that hold at any
size plus sampled checks the oracle computes one by one."""
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


def _pauli_label_of(v, n):
    """The Pauli string P with v = c i P, c = +-1, or None."""
    d = v.shape[0]
    H = -1j * v
    # a Pauli string has exactly one nonzero per row, all of modulus 1
    nz = np.abs(H) > 1e-9
    if not np.all(nz.sum(axis=1) == 1) or not np.allclose(np.abs(H[nz]), 1.0, atol=1e-12):
        return None
    best = None
    for lab in _candidate_labels(H, n):
        P = inputs.pauli_matrix(lab)
        c = np.vdot(P, H) / d
        if abs(abs(c) - 1) < 1e-12 and np.allclose(H, c * P, atol=1e-12):
            best = lab
    return best


def _candidate_labels(H, n):
    # x bits from the permutation pattern of row 0; z bits from the phases
    d = H.shape[0]
    col = int(np.argmax(np.abs(H[0])))
    x = col
    labels = []
    for z in range(d):
        lab = []
        for q in range(n):
            xb = (x >> (n - 1 - q)) & 1
            zb = (z >> (n - 1 - q)) & 1
            lab.append("IXZY"[xb + 2 * zb])
        labels.append("".join(lab))
    return labels


@pytest.mark.parametrize("prec", ["mixed"])
def test_su64_chain_full(prec):
    g, labels = inputs.workload_generators("su64_chain_d64")
    r = binding.lie_closure(g, 1e-8, precision=prec)
    assert r.dim == 4095
    D = r.dim
    assert r.report["brackets_checked"] == D * (D - 1) // 2
    V = r.basis
    assert oc.ortho_defect(V) < 1e-12
    rng = np.random.default_rng(7)
    pairs = [tuple(sorted(rng.choice(D, size=2, replace=False), reverse=True)) for _ in range(300)]
    assert oc.closure_residual(V, pairs=pairs) < 1e-7
    # every element is +-i times one Pauli string, and the strings are exactly
    # the exact integer closure of the generator strings
    want = set(oc.pauli_closure(labels))
    rows = rng.choice(D, size=200, replace=False)
    for i in rows:
        lab = _pauli_label_of(V[i], 6)
        assert lab in want
    traces = np.einsum("nii->n", V)
    assert np.max(np.abs(traces)) < 1e-12


def test_su128_random_growth_mixed():
    """Two random generators at d = 128 reach su(128) (dim 16383); the run stops
    at saturation, the exact dimension argument for anti-Hermitian inputs.
    The returned basis: orthonormal (the device's FP64 Gram over every 4th
    row equals the oracle's metric on the same rows), anti-Hermitian and
    traceless, and the screen's margin is reported."""
    g, _ = inputs.workload_generators("su128_random2_d128")
    r = binding.lie_closure(g, 1e-8, precision="mixed", saturation_exit=1, ortho_check=1)
    assert r.dim == 16383
    rep = r.report
    assert rep["min_acc_rel_res"] > 1e-8
    assert rep["ortho_rows"] == 4096
    V = r.basis
    want = oc.ortho_defect(V[::4])
    # the device's Gram entries are FP64 dot products over P = 16384
    # components (rounding ~ sqrt(P) u each); the host's BLAS sums in
    # another order: the two agree to a few sqrt(P) u
    assert abs(rep["ortho_defect"] - want) <= 4 * np.sqrt(128 * 128) * 2.0 ** -53
    assert rep["ortho_defect"] < 1e-12
    # brackets are traceless; an accepted element's component along the
    # trace direction iI / 1 (|tr v| / d) is FP64 rounding (~1e-16 per
    # term, grown by sqrt(N) ~ 128 over the projection) amplified by
    # ||h|| / ||h_perp|| <= 1 / min_acc (~1e4 here)
    traces = np.einsum("nii->n", V)
    bound = 1e-16 * 128 / rep["min_acc_rel_res"]
    assert np.max(np.abs(traces)) / 128 < bound
    assert np.max(np.abs(traces[:4096])) / 128 < 1e-13          # early elements: large residuals
    rng = np.random.default_rng(11)
    for i in rng.choice(r.dim, size=64, replace=False):
        np.testing.assert_allclose(V[i], -V[i].conj().T, atol=1e-14)
    assert 0.0 < rep["eps_screen"] < rep["tau_screen"] <= 1e-3


def test_random_d64_mixed_matches_fp64_path():
    """Random traceless pair at d = 64 (tensor-core brackets): the mixed path
    accepts the same candidates as the FP64 path (itself pinned to the oracle
    on small sizes), so the bases agree element by element."""
    g = inputs.random_set(64, 2, seed=77)
    a = binding.lie_closure(g, 1e-8, precision="mixed", saturation_exit=1)
    b = binding.lie_closure(g, 1e-8, precision="fp64", saturation_exit=1)
    assert a.dim == b.dim == 4095
    assert oc.ortho_defect(a.basis[:512]) < 1e-12
    np.testing.assert_allclose(a.basis, b.basis, atol=1e-10)
    # the measured threshold sits above the screen's noise (the largest
    # screened residual among the rejects stays below tau / 2), and every
    # accepted candidate screened far above tau
    rep = a.report
    assert rep["max_screen_rej_rel_res"] < 0.5 * rep["tau_screen"]
    assert rep["min_acc_screen_rel_res"] > 10.0 * rep["tau_screen"]


def test_su128_chain_growth_is_pauli():
    """su(128) chain, stopped at saturation: dimension 4^7 - 1 and every sampled
    element is +-i times a single Pauli string (brackets of strings are strings)."""
    labels = inputs.su2n_chain_labels(7)
    g = inputs.generators_from_labels(labels)
    r = binding.lie_closure(g, 1e-8, precision="mixed", saturation_exit=1)
    assert r.dim == 16383
    rng = np.random.default_rng(3)
    for i in rng.choice(r.dim, size=64, replace=False):
        assert _pauli_label_of(r.basis[i], 7) is not None


def test_so16_chain_d256_large_bracket_matches_fp64():
    """d = 256 goes through the large-d tensor-core bracket kernel; the mixed
    basis equals the FP64 path's element by element, and its dimension is
    n(2n-1) = 120 (so(16)), the exact Pauli closure's count."""
    labels = inputs.so2n_chain_labels(8)
    g = inputs.generators_from_labels(labels)
    a = binding.lie_closure(g, 1e-8, max_dim=160, precision="mixed")
    b = binding.lie_closure(g, 1e-8, max_dim=160, precision="fp64")
    assert a.dim == b.dim == 120 == len(oc.pauli_closure(labels))
    np.testing.assert_allclose(a.basis, b.basis, atol=1e-10)


def test_so20_chain_d1024_full():
    """The d = 1024 open chain closes to so(20): dimension 190, every element
    +-i times one of the exact closure's Pauli strings."""
    g, labels = inputs.workload_generators("so20_chain_d1024")
    r = binding.lie_closure(g, 1e-8, max_dim=256, precision="mixed")
    want = set(oc.pauli_closure(labels))
    assert r.dim == 190 == len(want)
    assert r.report["brackets_checked"] == 190 * 189 // 2
    rng = np.random.default_rng(5)
    for i in rng.choice(r.dim, size=12, replace=False):
        assert _pauli_label_of(r.basis[i], 10) in want


def test_batched256_per_set_dims():
    """The 256-set batched workload (saturation exit on): random traceless sets
    reach su(d), Pauli sets reach exactly their string closure."""
    sets = inputs.batched_sets(256, seed=1120)
    dims, stat, _, reps = binding.lie_closure_batched([s["generators"] for s in sets], 1e-8, saturation_exit=1)
    assert all(st == 0 for st in stat)
    for s, dim in zip(sets, dims):
        if s["kind"] == "pauli":
            assert dim == len(oc.pauli_closure(s["labels"])), s["labels"]
        else:
            assert dim == s["d"] ** 2 - 1
