"""Pins for the CPU oracle: closed forms, brute force, exact Pauli closure,
invariants, and planted mistakes that each pin must catch.  No GPU."""
import json
import os

import numpy as np
import pytest

import oracle.closure as oc
from paper_2506_01120_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dim(labels=None, gens=None, tol=1e-10, **kw):
    if gens is None:
        gens = inputs.generators_from_labels(labels)
    return oc.alg4_orthonormalization(gens, tol, **kw)


# ------------------------------------------------------------ primitives
def _sl2():
    E = np.array([[0, 1], [0, 0]], dtype=np.complex128)
    F = np.array([[0, 0], [1, 0]], dtype=np.complex128)
    H = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    return E, F, H


def test_sl2_relations():
    """Textbook sl(2) relations: [E, F] = H, [H, E] = 2E, [H, F] = -2F."""
    E, F, H = _sl2()
    np.testing.assert_array_equal(oc.bracket(E, F), H)
    np.testing.assert_array_equal(oc.bracket(H, E), 2 * E)
    np.testing.assert_array_equal(oc.bracket(H, F), -2 * F)


def test_pauli_algebra_closed_forms():
    """[iX, iY] = -[X, Y] = -2iZ; <iP, iQ> = delta_PQ for Pauli strings."""
    X, Y, Z = (inputs.pauli_matrix(c) for c in "XYZ")
    np.testing.assert_allclose(oc.bracket(1j * X, 1j * Y), -2j * Z, atol=0)
    np.testing.assert_allclose(oc.bracket(1j * Y, 1j * X), 2j * Z, atol=0)
    assert oc.inner(1j * Y, 1j * Y) == pytest.approx(1.0)
    assert abs(oc.inner(1j * X, 1j * Y)) == 0.0
    assert oc.norm(2j * Z) == pytest.approx(2.0)
    # <a, b> is conjugate-linear in a: <i a, b> = -i <a, b>
    a = inputs.random_antihermitian(4, np.random.default_rng(0))
    b = inputs.random_antihermitian(4, np.random.default_rng(1))
    assert oc.inner(1j * a, b) == pytest.approx(-1j * oc.inner(a, b))
    # anti-Hermitian operands give a real inner product
    assert abs(oc.inner(a, b).imag) < 1e-15


def test_project_out_matches_least_squares():
    """h - proj_V h equals the least-squares residual against span(V)."""
    rng = np.random.default_rng(3)
    d = 4
    V = oc.alg4_orthonormalization(np.stack([inputs.random_antihermitian(d, rng) for _ in range(5)]),
                                   1e-10, max_candidates=0).basis
    h = inputs.random_antihermitian(d, rng)
    r = oc.project_out(V, h)
    A = V.reshape(V.shape[0], -1).T
    coef, *_ = np.linalg.lstsq(A, h.reshape(-1), rcond=None)
    np.testing.assert_allclose(r.reshape(-1), h.reshape(-1) - A @ coef, atol=1e-13)


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("n", [2, 3, 4])
def test_so2n_chain(n):
    """Open chain {iX_j, iZ_jZ_{j+1}} maps (Jordan-Wigner) to nearest-neighbour
    Majorana bilinears, which generate so(2n): dimension n(2n-1)."""
    res = _dim(inputs.so2n_chain_labels(n))
    assert res.dim == n * (2 * n - 1)


def test_su2n_chain_matches_paper_table():
    """{iX_j, iY_j, iZ_jZ_{j+1}} is controllable: dimension 4^n - 1, the value
    Table 1(a) prints for each n."""
    table = json.load(open(os.path.join(GOLDEN, "paper_dims.json")))["table1a_hea"]
    printed = dict(zip(table["n"], table["dim"]))
    for n in (2, 3):
        res = _dim(inputs.su2n_chain_labels(n))
        assert res.dim == printed[n] == 4 ** n - 1
    res = _dim(inputs.su2n_chain_labels(4), saturation_exit=True)
    assert res.dim == printed[4] == 255 and res.saturated


def test_table2_basis_matrix_size():
    """Table 2 prints the d^2 x |B| basis-matrix size for dims 4095 and 16383."""
    t = json.load(open(os.path.join(GOLDEN, "paper_dims.json")))["table2_hea_sparse"]
    for n, dim, size in zip(t["n"], t["dim"], t["basis_matrix_size"]):
        assert dim == 4 ** n - 1
        assert abs(4 ** n * dim - size) / size < 0.01


@pytest.mark.parametrize("d", [2, 3, 4, 6])
def test_random_pair_generates_su_or_u(d):
    """A generic traceless pair generates su(d) (d^2 - 1); keeping the trace adds
    the centre direction and gives u(d) (d^2)."""
    rng = np.random.default_rng(10 + d)
    g = np.stack([inputs.random_antihermitian(d, rng) for _ in range(2)])
    assert _dim(gens=g, tol=1e-8).dim == d * d - 1
    g2 = np.stack([inputs.random_antihermitian(d, rng, traceless=False) for _ in range(2)])
    assert _dim(gens=g2, tol=1e-8).dim == d * d


def test_degenerate_sets():
    """Commuting sets give dim k; one generator gives 1; repeats and multiples are
    rejected in the generator pass; the zero operator is never accepted."""
    lab = ["ZII", "IZI", "ZZI", "IIZ"]
    assert _dim(lab).dim == 4
    assert _dim(["XYZ"]).dim == 1
    g = inputs.generators_from_labels(["XI", "XI", "IZ"])
    g[1] *= 3.0
    assert _dim(gens=g).dim == 2
    z = np.zeros((2, 4, 4), dtype=np.complex128)
    assert _dim(gens=z).dim == 0
    # a dependent combination of earlier generators is rejected
    a, b = inputs.generators_from_labels(["XX", "ZZ"])
    assert _dim(gens=np.stack([a, b, 0.3 * a - 2 * b])).dim == 2


# ------------------------------------------------------ brute force (Alg. 1)
@pytest.mark.parametrize("seed", range(12))
def test_alg4_equals_alg1_rank(seed):
    """Algorithm 4 and Algorithm 1 with an SVD rank test give the same dimension
    (Section 3.2: the two methods yield the same algebra)."""
    rng = np.random.default_rng(seed)
    d = int(rng.choice([2, 4, 8]))
    n = int(np.log2(d))
    if seed % 2 == 0:
        labels = inputs.random_pauli_labels(n, int(rng.integers(1, 4)), rng, max_weight=min(3, n))
        g = inputs.generators_from_labels(labels)
    else:
        d = int(rng.choice([2, 3, 4]))
        k = int(rng.integers(1, 3))
        g = np.stack([inputs.random_antihermitian(d, rng) for _ in range(k)])
    r4 = oc.alg4_orthonormalization(g, 1e-10)
    b1 = oc.alg1_rank(g)
    assert r4.dim == b1.shape[0]
    # same span: B from Alg. 1 is not orthonormal, compare spans
    if r4.dim:
        assert oc.span_distance(r4.basis, b1) < 1e-9


# ------------------------------------------------------- exact Pauli closure
def test_pauli_closure_closed_forms():
    assert len(oc.pauli_closure(inputs.so2n_chain_labels(3))) == 15
    assert len(oc.pauli_closure(inputs.so2n_chain_labels(10))) == 190
    assert len(oc.pauli_closure(inputs.su2n_chain_labels(6))) == 4095
    assert len(oc.pauli_closure(["X", "Z"])) == 3
    assert len(oc.pauli_closure(["ZI", "IZ"])) == 2


@pytest.mark.parametrize("seed", range(20))
def test_alg4_equals_pauli_closure(seed):
    """For Pauli-string generators the closure is spanned by the strings reached by
    the bracket, so Algorithm 4 and the exact integer closure agree, string by
    string (each accepted V element is +-i times one string)."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.choice([2, 3, 4]))
    labels = inputs.random_pauli_labels(n, int(rng.integers(2, 6)), rng, max_weight=min(3, n))
    strings = oc.pauli_closure(labels)
    res = oc.alg4_orthonormalization(inputs.generators_from_labels(labels), 1e-10)
    assert res.dim == len(strings)
    U = inputs.generators_from_labels(strings)
    assert oc.span_distance(res.basis, U) < 1e-12


# ------------------------------------------------------------- invariants
@pytest.mark.parametrize("case", ["so6", "random3"])
def test_basis_invariants(case):
    if case == "so6":
        g = inputs.generators_from_labels(inputs.so2n_chain_labels(3))
        tol = 1e-10
    else:
        g = inputs.random_set(3, 2, seed=7)
        tol = 1e-8
    res = oc.alg4_orthonormalization(g, tol)
    V = res.basis
    assert oc.ortho_defect(V) < 1e-12
    assert oc.closure_residual(V) < 10 * tol
    for v in V:
        np.testing.assert_allclose(v, -v.conj().T, atol=1e-14)        # anti-Hermitian
    for i in range(len(V)):
        for j in range(i):
            assert abs(np.trace(oc.bracket(V[i], V[j]))) < 1e-13      # traceless brackets
    assert res.max_imag_beta < 1e-14


def test_span_distance_known_angle():
    """sin of a rotation angle out of the span is recovered exactly."""
    labels = ["XI", "ZI", "IX", "IZ"]
    V = inputs.generators_from_labels(labels)
    W = inputs.generators_from_labels(["YY"])[0]
    for theta in (1e-9, 1e-3, 0.7):
        U = V.copy()
        U[2] = np.cos(theta) * V[2] + np.sin(theta) * W
        assert oc.span_distance(V, U) == pytest.approx(np.sin(theta), rel=1e-6, abs=1e-15)
    assert oc.span_distance(V, V[[1, 0, 3, 2]]) < 1e-15
    assert oc.span_distance(V, V[:3]) == 1.0


def test_resume_matches_single_run():
    """The (V, l, m) cursor state is complete: a run split in two equals one run."""
    g = inputs.generators_from_labels(inputs.su2n_chain_labels(2))
    full = oc.alg4_orthonormalization(g, 1e-10)
    part = oc.alg4_orthonormalization(g, 1e-10, max_candidates=17)
    part = oc.alg4_orthonormalization(g, 1e-10, resume=part)
    assert part.dim == full.dim
    np.testing.assert_allclose(part.basis, full.basis, atol=1e-14)


# ------------------------------------------------------- planted mistakes
def _pins_pass():
    """A compact subset of the pins above; True iff all hold."""
    try:
        if _dim(inputs.so2n_chain_labels(3)).dim != 15:
            return False
        if _dim(inputs.su2n_chain_labels(2)).dim != 15:
            return False
        g = inputs.random_set(3, 2, seed=7)
        res = oc.alg4_orthonormalization(g, 1e-8)
        if res.dim != 8 or oc.ortho_defect(res.basis) > 1e-12:
            return False
        if oc.closure_residual(res.basis) > 1e-7:
            return False
        X, Y, Z = (inputs.pauli_matrix(c) for c in "XYZ")
        if not np.allclose(oc.bracket(1j * X, 1j * Y), -2j * Z):
            return False
        E, F, H = _sl2()
        if not (np.allclose(oc.bracket(E, F), H) and np.allclose(oc.bracket(H, E), 2 * E)):
            return False
        return True
    except Exception:
        return False


def test_pins_pass_unpatched():
    assert _pins_pass()


@pytest.mark.parametrize("mistake", ["anticommutator", "no_conjugate", "transposed_operand",
                                     "dropped_projection_term", "wrong_inner_scale"])
def test_planted_mistake_is_caught(monkeypatch, mistake):
    """Each plausible slip in the oracle's arithmetic makes a pin fail."""
    if mistake == "anticommutator":
        monkeypatch.setattr(oc, "bracket", lambda a, b: a @ b + b @ a)
    elif mistake == "no_conjugate":
        monkeypatch.setattr(oc, "coefficients",
                            lambda V, h: np.einsum("ljk,jk->l", V, h) / h.shape[0])
        monkeypatch.setattr(oc, "inner", lambda a, b: np.trace(a.T @ b) / a.shape[0])
    elif mistake == "transposed_operand":
        monkeypatch.setattr(oc, "bracket", lambda a, b: a.T @ b - b @ a.T)
    elif mistake == "dropped_projection_term":
        orig = oc.project_out
        monkeypatch.setattr(oc, "project_out", lambda V, h: orig(V[:-1], h) if len(V) > 1 else orig(V, h))
    elif mistake == "wrong_inner_scale":
        monkeypatch.setattr(oc, "coefficients",
                            lambda V, h: np.einsum("ljk,jk->l", V.conj(), h))
    assert not _pins_pass()


# ------------------------------------------------------------- Algorithm 3
@pytest.mark.parametrize("case", ["so6", "su8", "rand_d4", "pauli"])
def test_alg3_same_algebra_as_alg4(case):
    """Algorithm 3 keeps the generators and nested brackets B; the paper notes
    that it yields the same algebra as Algorithm 4 (Section 3.2).  Pins: equal
    dimension, span(B) = span(V) = the Algorithm 4 span, V orthonormal, and every
    kept element after the generators is literally the bracket of its parents."""
    if case == "so6":
        g = inputs.generators_from_labels(inputs.so2n_chain_labels(3)); expect = 15
    elif case == "su8":
        g = inputs.generators_from_labels(inputs.su2n_chain_labels(3)); expect = 63
    elif case == "rand_d4":
        g = inputs.random_set(4, 2, seed=3); expect = 15
    else:
        rng = np.random.default_rng(9)
        labels = inputs.random_pauli_labels(3, 4, rng)
        g = inputs.generators_from_labels(labels); expect = len(oc.pauli_closure(labels))
    r3 = oc.alg3_orthonormalization(g, 1e-10)
    r4 = oc.alg4_orthonormalization(g, 1e-10)
    assert r3.dim == r4.dim == expect
    assert oc.ortho_defect(r3.V) < 1e-12
    assert oc.span_distance(r3.V, r4.basis) < 1e-9
    assert oc.span_distance(r3.B, r3.V) < 1e-9
    for i, par in enumerate(r3.parents):
        if par is None:
            assert any(np.array_equal(r3.B[i], x) for x in g)
        else:
            l, m = par
            np.testing.assert_array_equal(r3.B[i], oc.bracket(r3.B[l], r3.B[m]))


# ------------------------------------------------------------- Algorithm 2
@pytest.mark.parametrize("case", ["so6", "su8", "rand_d4", "pauli", "dependent"])
def test_alg2_same_algebra(case):
    """The matrix-inversion method (Theorem 1: h is dependent iff
    h - B A^-1 beta = 0) finds the same algebra as Algorithm 4; B is unit-norm,
    its Gram matrix times the stored inverse is the identity, and B's elements
    after the generators are normalised brackets of earlier ones."""
    if case == "so6":
        g = inputs.generators_from_labels(inputs.so2n_chain_labels(3)); expect = 15
    elif case == "su8":
        g = inputs.generators_from_labels(inputs.su2n_chain_labels(3)); expect = 63
    elif case == "rand_d4":
        g = inputs.random_set(4, 2, seed=3); expect = 15
    elif case == "pauli":
        rng = np.random.default_rng(9)
        labels = inputs.random_pauli_labels(3, 4, rng)
        g = inputs.generators_from_labels(labels); expect = len(oc.pauli_closure(labels))
    else:
        a, b = inputs.generators_from_labels(["XX", "ZZ"])
        g = np.stack([a, b, 0.3 * a - 2 * b]); expect = 2      # commuting, third dependent
    r2 = oc.alg2_matrix_inversion(g, 1e-10)
    r4 = oc.alg4_orthonormalization(g, 1e-10)
    assert r2.dim == r4.dim == expect
    assert oc.span_distance(r4.basis, r2.B) < 1e-9
    for b in r2.B:
        assert oc.norm(b) == pytest.approx(1.0, abs=1e-13)
    G = oc.gram(r2.B)
    assert np.max(np.abs(G @ r2.A_inv - np.eye(r2.dim))) < 1e-8


def test_packed_pauli_strings_follow_the_oracle_bit_convention():
    """The Pauli-sum entry point's packed strings (x | z << 32) carry the same
    (x, z) bits as the oracle's symplectic encoding, and a product string is the
    XOR of the two (up to phase), checked on matrices."""
    import itertools
    from paper_2506_01120_gb300 import inputs
    for label in ["X", "Y", "Z", "XYZ", "IZY", "YYIX"]:
        x, z = oc.pauli_to_bits(label)
        assert inputs.pauli_string(label) == x | (z << 32)
    for a, b in itertools.product(["XY", "ZI", "YZ", "XX"], repeat=2):
        pa, pb = inputs.pauli_string(a), inputs.pauli_string(b)
        prod = inputs.pauli_matrix(a) @ inputs.pauli_matrix(b)
        x, z = (pa ^ pb) & 0xFFFFFFFF, (pa ^ pb) >> 32
        ref = inputs.pauli_matrix(oc.bits_to_pauli(x, z, 2))
        ratio = prod[np.nonzero(ref)] / ref[np.nonzero(ref)]
        assert np.allclose(ratio, ratio[0]) and abs(abs(ratio[0]) - 1) < 1e-15


def test_alg2_goes_unstable_where_alg4_does_not():
    """Section 3.1 warns that the matrix-inversion method may be numerically
    unstable.  On a random traceless pair at d = 16 and tol = 1e-8 Algorithm 4
    returns su(16) (255, the closed form) while Algorithm 2's inverse Gram
    matrix lets rounding through and its basis grows past any possible
    dimension (capacity 2 d^2 reached)."""
    from paper_2506_01120_gb300 import inputs
    g = inputs.random_set(16, 2, seed=116)
    assert oc.alg4_orthonormalization(g, 1e-8, saturation_exit=True).dim == 255
    with pytest.raises(oc.CapacityError):
        oc.alg2_matrix_inversion(g, 1e-8)


# -------------------------------------------- pins of the comparison metrics
# The tests of the GPU path lean on ortho_defect, closure_residual and
# margin_report as upper-bound gates, so each must recover a value planted in
# its input; a metric that always returns 0 (or drops a term) fails here.
def _tilted_su2(phi):
    """{iXI, iYI, i(cos phi ZI + sin phi IX)}: orthonormal.  [iXI, iYI] = -2i ZI
    has the component -2 cos(phi) along the third element, so its residual is
    2 |sin phi| out of a norm of 2; the other two brackets are multiples of iYI
    and iXI (in the span).  Closure residual: |sin phi| exactly."""
    a, b, z, x = inputs.generators_from_labels(["XI", "YI", "ZI", "IX"])
    return np.stack([a, b, np.cos(phi) * z + np.sin(phi) * x])


def _overlap_basis(eps, phase, delta):
    """Four orthonormal Pauli elements with element 1 tilted to overlap
    eps * e^{i phase} with element 0 (still unit norm) and element 3 scaled by
    (1 + delta): defect max(eps, 2 delta + delta^2)."""
    V = inputs.generators_from_labels(["XI", "ZI", "IY", "ZZ"]).copy()
    V[1] = np.sqrt(1 - eps ** 2) * V[1] + eps * np.exp(1j * phase) * V[0]
    V[3] = (1 + delta) * V[3]
    return V


def _metric_pins_pass():
    try:
        for eps, phase, delta in [(1e-3, 0.0, 0.0), (2e-7, 1.1, 0.0), (1e-9, 2.5, 3e-6), (0.25, -0.4, 1e-4)]:
            want = max(eps, 2 * delta + delta ** 2)
            if abs(oc.ortho_defect(_overlap_basis(eps, phase, delta)) - want) > 1e-15 + 1e-9 * want:
                return False
        if oc.ortho_defect(inputs.generators_from_labels(oc.pauli_closure(["XY", "ZI"]))) > 1e-15:
            return False
        for phi in (0.3, 1e-4, 1.2):
            if abs(oc.closure_residual(_tilted_su2(phi)) - abs(np.sin(phi))) > 1e-12:
                return False
        if oc.closure_residual(_tilted_su2(0.0)) > 1e-15:
            return False
        labels = oc.pauli_closure(inputs.so2n_chain_labels(3))
        V = inputs.generators_from_labels(labels)
        if oc.closure_residual(V) > 1e-15:          # so(6) is closed
            return False
        # so(6) minus one element: some pair brackets exactly onto the missing string
        if abs(oc.closure_residual(V[:-1]) - 1.0) > 1e-12:
            return False
        # margins of a hand-built result
        r = oc.Alg4Result(V=V, dim=3, accepted_rel=[0.5, 1e-3, 0.9], rejected_rel=[1e-14, 3e-12, 2e-13])
        m = oc.margin_report(r)
        if (m["min_acc_rel_res"], m["max_rej_rel_res"], m["n_acc"], m["n_rej_nonzero"]) != (1e-3, 3e-12, 3, 3):
            return False
        m0 = oc.margin_report(oc.Alg4Result(V=V, dim=0))
        if not (m0["min_acc_rel_res"] == np.inf and m0["max_rej_rel_res"] == 0.0):
            return False
        # margins of a real run: the second generator iXI + eps iZZ has relative
        # residual eps / sqrt(1 + eps^2) against the first
        eps = 1e-3
        a, zz = inputs.generators_from_labels(["XI", "ZZ"])
        res = oc.alg4_orthonormalization(np.stack([a, a + eps * zz]), 1e-8)
        mr = oc.margin_report(res)
        if abs(mr["min_acc_rel_res"] - eps / np.sqrt(1 + eps ** 2)) > 1e-12:
            return False
        if mr["n_acc"] != res.dim or mr["max_rej_rel_res"] > 1e-12:
            return False
        return True
    except Exception:
        return False


def test_metric_pins_pass_unpatched():
    assert _metric_pins_pass()


def test_ortho_defect_recovers_planted_overlap():
    for eps in (1e-12, 1e-6, 0.1):
        assert oc.ortho_defect(_overlap_basis(eps, 0.7, 0.0)) == pytest.approx(eps, rel=1e-9, abs=1e-16)
    assert oc.ortho_defect(_overlap_basis(0.0, 0.0, 1e-5)) == pytest.approx(2e-5 + 1e-10, rel=1e-9)


def test_closure_residual_recovers_planted_tilt():
    for phi in (1e-6, 0.3, np.pi / 2):
        assert oc.closure_residual(_tilted_su2(phi)) == pytest.approx(abs(np.sin(phi)), rel=1e-10, abs=1e-15)
    # the pair list restricts the maximum: only (1, 0) leaves the span
    V = _tilted_su2(0.5)
    assert oc.closure_residual(V, pairs=[(2, 0), (2, 1)]) < 1e-15
    assert oc.closure_residual(V, pairs=[(1, 0)]) == pytest.approx(np.sin(0.5), rel=1e-12)


def test_margin_report_of_a_near_dependent_generator():
    for eps in (1e-2, 1e-5):
        a, zz = inputs.generators_from_labels(["XI", "ZZ"])
        res = oc.alg4_orthonormalization(np.stack([a, a + eps * zz]), 1e-8)
        m = oc.margin_report(res)
        assert m["min_acc_rel_res"] == pytest.approx(eps / np.sqrt(1 + eps ** 2), rel=1e-10)
        assert m["n_acc"] == res.dim


@pytest.mark.parametrize("mistake", ["defect_zero", "defect_signed", "defect_no_identity", "residual_unscaled",
                                     "residual_anticommutator", "residual_no_projection", "margin_swapped",
                                     "margin_first_accept"])
def test_planted_metric_mistake_is_caught(monkeypatch, mistake):
    """Each plausible slip in a comparison metric makes a metric pin fail."""
    if mistake == "defect_zero":
        monkeypatch.setattr(oc, "ortho_defect", lambda V: 0.0)
    elif mistake == "defect_signed":
        monkeypatch.setattr(oc, "ortho_defect",
                            lambda V: float(np.max((oc.gram(V) - np.eye(V.shape[0])).real)) if len(V) else 0.0)
    elif mistake == "defect_no_identity":
        monkeypatch.setattr(oc, "ortho_defect",
                            lambda V: float(np.max(np.abs(oc.gram(V) - np.diag(np.diag(oc.gram(V)))))))
    elif mistake == "residual_unscaled":
        def unscaled(V, pairs=None, eta_abs=1e-12):
            N = V.shape[0]
            pairs = pairs or [(i, j) for i in range(N) for j in range(i)]
            return max([oc.norm(oc.project_out(V, oc.bracket(V[i], V[j]))) for i, j in pairs] or [0.0])
        monkeypatch.setattr(oc, "closure_residual", unscaled)
    elif mistake == "residual_anticommutator":
        monkeypatch.setattr(oc, "bracket", lambda a, b: a @ b + b @ a)
    elif mistake == "residual_no_projection":
        monkeypatch.setattr(oc, "project_out", lambda V, h: h.copy())
    elif mistake == "margin_swapped":
        orig = oc.margin_report
        def swapped(res):
            m = orig(res)
            m["min_acc_rel_res"], m["max_rej_rel_res"] = m["max_rej_rel_res"], m["min_acc_rel_res"]
            return m
        monkeypatch.setattr(oc, "margin_report", swapped)
    elif mistake == "margin_first_accept":
        orig = oc.margin_report
        def first(res):
            m = orig(res)
            m["min_acc_rel_res"] = res.accepted_rel[0] if res.accepted_rel else np.inf
            return m
        monkeypatch.setattr(oc, "margin_report", first)
    assert not _metric_pins_pass()


def test_absolute_and_relative_tolerance_readings():
    """g2 = 1e4 iXI + 1e-3 iZZ has orthogonal part 1e-3 iZZ against g1 = iXI:
    relative residual ~1e-7, absolute residual 1e-3.  At tol = 1e-6 the
    relative reading rejects it (dimension 1: no pair to bracket), the absolute
    one accepts it, and {XI, ZZ} bracket to YZ, closing to dimension 3."""
    a, zz = inputs.generators_from_labels(["XI", "ZZ"])
    g = np.stack([a, 1e4 * a + 1e-3 * zz])
    assert oc.alg4_orthonormalization(g, 1e-6).dim == 1
    r = oc.alg4_orthonormalization(g, 1e-6, tol_mode="absolute")
    assert r.dim == 3
    assert r.accepted_rel[1] == pytest.approx(1e-3 / np.linalg.norm([1e4, 1e-3]), rel=1e-6)
    # a residual of 1e-3 at tol 1e-2 is rejected in both readings
    assert oc.alg4_orthonormalization(g, 1e-2, tol_mode="absolute").dim == 1
