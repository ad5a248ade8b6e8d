"""Seeded synthetic generator sets for the Lie-closure workloads.

This module builds inputs only: Pauli-string matrices, open-chain generator
sets and seeded random anti-Hermitian matrices.  It contains none of the
closure arithmetic (no brackets, inner products or projections), so both the
CUDA path and the CPU oracle can draw their inputs from it.

Conventions
-----------
* Pauli matrices X=[[0,1],[1,0]], Y=[[0,-i],[i,0]], Z=diag(1,-1); qubit 1 is
  the leftmost Kronecker factor, so label "XZI" is X (x) Z (x) I.
* A generator is the anti-Hermitian matrix i*P for a Pauli string P, or i*H for
  a random Hermitian H (the paper works in su(d), Section 2.1).
* Random Hermitian draw: a d x d real block then a d x d imaginary block, both
  row-major standard normals scaled by sqrt(1/2) (so E|G_jk|^2 = 1), from
  ``numpy.random.default_rng(seed)`` (PCG64); H = (G + G^dagger)/2; by default
  the trace part (tr H / d) I is removed so that a generic pair generates
  su(d) of dimension d^2 - 1; the result i*H is scaled to unit Frobenius norm.
* Generator order inside a chain set: all iX_j, then all iY_j, then all
  iZ_jZ_{j+1}, each by ascending j.
"""
from __future__ import annotations

import numpy as np

_PAULI = {
    "I": np.array([[1, 0], [0, 1]], dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def pauli_matrix(label: str) -> np.ndarray:
    """Dense 2^n x 2^n matrix of the Pauli string ``label`` (qubit 1 leftmost)."""
    out = np.ones((1, 1), dtype=np.complex128)
    for ch in label:
        out = np.kron(out, _PAULI[ch])
    return out


def chain_labels(n: int, singles=("X",), zz: bool = True) -> list[str]:
    """Open-chain labels: every letter of ``singles`` on each qubit, then Z_jZ_{j+1}."""
    labels = []
    for letter in singles:
        for j in range(n):
            labels.append("I" * j + letter + "I" * (n - j - 1))
    if zz:
        for j in range(n - 1):
            labels.append("I" * j + "ZZ" + "I" * (n - j - 2))
    return labels


def generators_from_labels(labels) -> np.ndarray:
    """Stack of i*P for each Pauli string label, shape (k, d, d), complex128."""
    return np.stack([1j * pauli_matrix(s) for s in labels]).astype(np.complex128)


def pauli_string(label: str) -> int:
    """Packed string x | (z << 32) of a Pauli label: bit q of x (z) is set when
    qubit q+1 carries X or Y (Z or Y)."""
    x = z = 0
    for q, ch in enumerate(label):
        if ch in "XY":
            x |= 1 << q
        if ch in "ZY":
            z |= 1 << q
    return x | (z << 32)


def pauli_sum_terms(ops):
    """Sparse generator arrays for the Pauli-sum entry point.  ``ops`` is a list
    of operators, each a list of (label, coefficient) pairs standing for
    i * sum coefficient * P(label).  Returns (strings uint64, coefs float64,
    offsets int64)."""
    strings, coefs, offsets = [], [], [0]
    for op in ops:
        for label, c in op:
            strings.append(pauli_string(label))
            coefs.append(float(c))
        offsets.append(len(strings))
    return (np.array(strings, dtype=np.uint64), np.array(coefs, dtype=np.float64),
            np.array(offsets, dtype=np.int64))


def pauli_sum_matrix(op, n: int) -> np.ndarray:
    """Dense i * sum c P(label) of one Pauli-sum operator."""
    out = np.zeros((2 ** n, 2 ** n), dtype=np.complex128)
    for label, c in op:
        out += 1j * c * pauli_matrix(label)
    return out


def tfim_ops(n: int) -> list:
    """Transverse-field Ising generators on an open chain: sum_j X_j and
    sum_j Z_j Z_{j+1}, unit coefficients."""
    xs = [("I" * j + "X" + "I" * (n - j - 1), 1.0) for j in range(n)]
    zz = [("I" * j + "ZZ" + "I" * (n - j - 2), 1.0) for j in range(n - 1)]
    return [xs, zz]


def random_pauli_sums(n: int, k: int, terms: int, seed: int) -> list:
    """k operators of ``terms`` random non-identity strings each (letters
    uniform over I, X, Y, Z per qubit, redrawn if all I) with N(0, 1)
    coefficients, from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    ops = []
    for _ in range(k):
        op = []
        while len(op) < terms:
            label = "".join("IXYZ"[int(v)] for v in rng.integers(0, 4, size=n))
            if set(label) == {"I"}:
                continue
            op.append((label, float(rng.standard_normal())))
        ops.append(op)
    return ops


def so2n_chain_labels(n: int) -> list[str]:
    """{X_j} and {Z_jZ_{j+1}} on an open chain of n qubits."""
    return chain_labels(n, singles=("X",), zz=True)


def su2n_chain_labels(n: int) -> list[str]:
    """{X_j}, {Y_j} and {Z_jZ_{j+1}} on an open chain of n qubits."""
    return chain_labels(n, singles=("X", "Y"), zz=True)


def random_hermitian_block(d: int, rng: np.random.Generator) -> np.ndarray:
    """G with i.i.d. complex N(0,1) entries (real block, then imaginary block)."""
    re = rng.standard_normal((d, d))
    im = rng.standard_normal((d, d))
    return (re + 1j * im) * np.sqrt(0.5)


def random_antihermitian(d: int, rng: np.random.Generator, traceless: bool = True,
                         unit_frobenius: bool = True) -> np.ndarray:
    """i*H with H = (G + G^dagger)/2 as described in the module docstring."""
    g = random_hermitian_block(d, rng)
    h = (g + g.conj().T) / 2
    if traceless:
        h = h - (np.trace(h).real / d) * np.eye(d)
    a = 1j * h
    if unit_frobenius:
        a = a / np.sqrt(np.sum(np.abs(a) ** 2))
    return a.astype(np.complex128)


def random_pauli_labels(n: int, k: int, rng: np.random.Generator, max_weight: int = 3) -> list[str]:
    """k random Pauli strings on n qubits with support size uniform in 1..max_weight,
    support qubits uniform without replacement and each support letter uniform in XYZ."""
    labels = []
    for _ in range(k):
        w = int(rng.integers(1, max_weight + 1))
        qubits = rng.choice(n, size=w, replace=False)
        letters = rng.integers(0, 3, size=w)
        s = ["I"] * n
        for q, c in zip(qubits, letters):
            s[int(q)] = "XYZ"[int(c)]
        labels.append("".join(s))
    return labels


def batched_sets(nsets: int = 256, seed: int = 1120, dims=(8, 16, 32, 64)):
    """The batched workload: ``nsets`` independent generator sets.

    Per set, in draw order: d uniform over ``dims``; k uniform over 2..6; kind
    uniform over {random, pauli}; then the k generators.  Returns a list of dicts
    with keys d, k, kind, generators (k, d, d) and labels (Pauli sets only)."""
    rng = np.random.default_rng(seed)
    sets = []
    for _ in range(nsets):
        d = int(rng.choice(np.asarray(dims)))
        k = int(rng.integers(2, 7))
        kind = "pauli" if int(rng.integers(0, 2)) == 1 else "random"
        if kind == "random":
            gens = np.stack([random_antihermitian(d, rng) for _ in range(k)])
            labels = None
        else:
            n = int(np.log2(d))
            labels = random_pauli_labels(n, k, rng)
            gens = generators_from_labels(labels)
        sets.append({"d": d, "k": k, "kind": kind, "generators": gens, "labels": labels})
    return sets


def random_subalgebra_set(kind: str, d: int, k: int, seed: int) -> np.ndarray:
    """k seeded random generators inside a proper subalgebra of su(d), unit
    Frobenius norm:
      "so"    -- real antisymmetric matrices (i.i.d. N(0, 1) above the
                 diagonal), which are anti-Hermitian and span so(d);
      "block" -- block-diagonal diag(a, b) of two independent random traceless
                 anti-Hermitian (d/2) x (d/2) blocks, inside su(d/2) + su(d/2)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        if kind == "so":
            x = np.triu(rng.standard_normal((d, d)), 1)
            a = (x - x.T).astype(np.complex128)
        elif kind == "block":
            h = d // 2
            a = np.zeros((d, d), dtype=np.complex128)
            a[:h, :h] = random_antihermitian(h, rng, unit_frobenius=False)
            a[h:, h:] = random_antihermitian(h, rng, unit_frobenius=False)
        else:
            raise ValueError(kind)
        out.append(a / np.sqrt(np.sum(np.abs(a) ** 2)))
    return np.stack(out)


def random_set(d: int, k: int, seed: int, traceless: bool = True) -> np.ndarray:
    """k seeded random anti-Hermitian generators of size d (unit Frobenius norm)."""
    rng = np.random.default_rng(seed)
    return np.stack([random_antihermitian(d, rng, traceless=traceless) for _ in range(k)])


# The five workloads.  ``expected_dim`` is the textbook closed form for the set.
WORKLOADS = {
    "so6_chain_d8": dict(n=3, d=8, tol=1e-10, expected_dim=15,
                         doc="iX_j (j=1..3), iZ_jZ_{j+1} (j=1..2), open chain; so(6)"),
    "su64_chain_d64": dict(n=6, d=64, tol=1e-8, expected_dim=4095,
                           doc="iX_j, iY_j (j=1..6), iZ_jZ_{j+1} (j=1..5); su(64)"),
    "so20_chain_d1024": dict(n=10, d=1024, tol=1e-8, expected_dim=190,
                             doc="iX_j (j=1..10), iZ_jZ_{j+1} (j=1..9); so(20)"),
    "batched256_d8to64": dict(nsets=256, seed=1120, tol=1e-8, expected_dim=None,
                              doc="256 random or Pauli sets, d in {8,16,32,64}"),
    "su128_random2_d128": dict(n=7, d=128, tol=1e-8, seed=2506, expected_dim=16383,
                               doc="two seeded traceless random iH, unit Frobenius; su(128)"),
}


def workload_generators(name: str):
    """Generators (k, d, d) complex128 and Pauli labels (or None) of a single-set workload."""
    w = WORKLOADS[name]
    if name == "so6_chain_d8" or name == "so20_chain_d1024":
        labels = so2n_chain_labels(w["n"])
        return generators_from_labels(labels), labels
    if name == "su64_chain_d64":
        labels = su2n_chain_labels(w["n"])
        return generators_from_labels(labels), labels
    if name == "su128_random2_d128":
        return random_set(w["d"], 2, w["seed"]), None
    raise KeyError(name)
