"""Input builders and the label <-> packed-string conversions of the Pauli-sum
entry point (CPU only)."""
import numpy as np

from paper_2506_01120_gb300 import binding, inputs


def test_packed_string_round_trip():
    rng = np.random.default_rng(7)
    for n in (1, 3, 8, 31):
        for _ in range(50):
            label = "".join("IXYZ"[int(v)] for v in rng.integers(0, 4, size=n))
            assert binding.pauli_label(inputs.pauli_string(label), n) == label


def test_pauli_sum_terms_layout():
    ops = [[("XI", 1.0), ("ZZ", -0.5)], [], [("YY", 2.0)]]
    s, c, o = inputs.pauli_sum_terms(ops)
    assert s.dtype == np.uint64 and c.dtype == np.float64 and o.dtype == np.int64
    assert o.tolist() == [0, 2, 2, 3]
    assert [binding.pauli_label(x, 2) for x in s] == ["XI", "ZZ", "YY"]
    assert c.tolist() == [1.0, -0.5, 2.0]


def test_pauli_sum_matrix_is_anti_hermitian_and_linear():
    op = [("XZ", 0.3), ("YI", -1.2), ("XZ", 0.7)]
    M = inputs.pauli_sum_matrix(op, 2)
    np.testing.assert_allclose(M, -M.conj().T, atol=1e-15)
    ref = 1j * (1.0 * inputs.pauli_matrix("XZ") - 1.2 * inputs.pauli_matrix("YI"))
    np.testing.assert_allclose(M, ref, atol=1e-15)


def test_random_pauli_sums_are_seeded_and_never_identity():
    a = inputs.random_pauli_sums(5, 3, 4, seed=11)
    b = inputs.random_pauli_sums(5, 3, 4, seed=11)
    assert a == b
    assert len(a) == 3 and all(len(op) == 4 for op in a)
    assert all(set(label) != {"I"} for op in a for label, _ in op)
    assert a != inputs.random_pauli_sums(5, 3, 4, seed=12)


def test_tfim_ops():
    xs, zz = inputs.tfim_ops(4)
    assert [l for l, _ in xs] == ["XIII", "IXII", "IIXI", "IIIX"]
    assert [l for l, _ in zz] == ["ZZII", "IZZI", "IIZZ"]
    assert all(c == 1.0 for _, c in xs + zz)


def test_random_subalgebra_sets_have_the_stated_structure():
    import numpy as np
    from paper_2506_01120_gb300 import inputs
    g = inputs.random_subalgebra_set("so", 8, 3, seed=1)
    assert g.shape == (3, 8, 8)
    assert np.all(g.imag == 0) and np.allclose(g, -np.transpose(g, (0, 2, 1)))
    b = inputs.random_subalgebra_set("block", 8, 2, seed=2)
    assert np.all(b[:, :4, 4:] == 0) and np.all(b[:, 4:, :4] == 0)
    for a in b:
        np.testing.assert_allclose(a, -a.conj().T, atol=1e-15)
        assert abs(np.trace(a[:4, :4])) < 1e-14 and abs(np.trace(a[4:, 4:])) < 1e-14
    assert np.allclose([np.sum(np.abs(a) ** 2) for a in np.concatenate([g, b])], 1.0)
