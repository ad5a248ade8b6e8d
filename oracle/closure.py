"""CPU oracle for the Lie closure (test infrastructure, not product code).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA path and
never touches a GPU.  Everything is plain NumPy in complex128 (FP64), written
from the paper's definitions, one candidate at a time, so that each step can be
checked against the paper by eye.

Functions and the passage each follows
--------------------------------------
* ``bracket``      -- the Lie bracket [a, b] = ab - ba (Section 2.2, the
                      matrix-commutator definition).
* ``inner``        -- <a, b> = tr(a^dagger b) / d (Section 2.2).
* ``norm``         -- ||a|| = sqrt(<a, a>) (Section 2.2).
* ``project_out``  -- h - proj_V h = h - sum_l <V[l], h> V[l] (Section 3.2,
                      the Corollary and the equation after it).
* ``alg4_orthonormalization`` -- Algorithm 4 (dimension-only orthonormalisation
                      method), O1.
* ``alg2_matrix_inversion`` -- Algorithm 2 (the matrix-inversion method of
                      Section 3.1: unit-norm B, Gram matrix A and its inverse).
* ``alg3_orthonormalization`` -- Algorithm 3 (orthonormalisation keeping the
                      generators and nested brackets B beside V).
* ``alg1_rank``    -- Algorithm 1 with the independence test done by matrix rank
                      via SVD (Section 3, the rank method), O2.
* ``pauli_closure`` -- exact closure of a set of Pauli strings by set
                      membership (Section 3, the Pauli-string containment idea
                      the paper cites as prior art), O3.
* ``span_distance``, ``ortho_defect``, ``closure_residual`` -- comparison
                      metrics (sin of the largest principal angle; max
                      |<v_i,v_j> - delta_ij|; relative residual of brackets).

Readings of the paper taken here (the paper leaves them open):
* Each pair (l, m), 0 <= m < l, is formed once, l ascending then m ascending;
  the loop ends when l reaches |V| (Algorithm 4 re-forms some pairs; re-checking
  is idempotent).
* "h_perp != 0" is decided as ||h|| > eta_abs and ||h_perp|| > tol * ||h||,
  with h_perp from two classical Gram-Schmidt passes ("twice is enough").
* ``tol_mode="absolute"`` reads the test as ||h_perp|| > tol instead (the
  elements of V have unit norm, so this thresholds the orthogonal part
  itself); the relative form is the default.
* Optional saturation exit: for anti-Hermitian inputs the closure lies in
  su(d) plus at most one trace direction, so once |V| reaches that bound every
  remaining candidate is dependent.  Off by default.
* The absolute floor eta_abs (default 1e-12) is for brackets of orthonormal
  elements whose exact value is zero (commuting pairs).  For operators that
  are sums of many Pauli strings with random coefficients, a zero bracket
  formed from elements that were themselves accepted with relative residuals
  near 1e-3 carries rounding amplified by those accepts and can reach ~1e-11,
  above 1e-12; accepting it fills the algebra with noise (the inflated
  dimensions of Table 1(d) are that failure).  For such inputs the floor is
  ``ETA_ABS_PAULI_SUMS`` = 1e-9, still far below any genuine bracket of unit
  elements at the sizes used, and a run is trusted only when its margin report
  shows min_acc > 10 tol and max_rej < tol / 10.

Parity status: every public function here is pinned by ``tests/test_oracle.py``
(closed-form dimensions, brute-force rank agreement, exact Pauli closure,
invariants, and planted-mistake checks); the comparison metrics
``ortho_defect``, ``closure_residual`` and ``margin_report`` by planted values
they must recover (an overlap of known size, a su(2) subalgebra tilted out of
its span by a known angle, a candidate with a known relative residual).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np


# Absolute floor on ||h|| for generators that are sums of many Pauli strings
# with random coefficients (see the readings above).
ETA_ABS_PAULI_SUMS = 1e-9


# ---------------------------------------------------------------- primitives
def bracket(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """[a, b] = ab - ba (Section 2.2)."""
    return a @ b - b @ a


def inner(a: np.ndarray, b: np.ndarray) -> complex:
    """<a, b> = tr(a^dagger b) / d (Section 2.2)."""
    d = a.shape[0]
    return np.trace(a.conj().T @ b) / d


def norm(a: np.ndarray) -> float:
    """||a|| = sqrt(<a, a>) (Section 2.2)."""
    return float(np.sqrt(max(inner(a, a).real, 0.0)))


def coefficients(V: np.ndarray, h: np.ndarray) -> np.ndarray:
    """beta_l = <V[l], h> for every stored element (Theorem 1's beta vector)."""
    d = h.shape[0]
    # tr(V[l]^dagger h) = sum_jk conj(V[l]_jk) h_jk
    return np.einsum("ljk,jk->l", V.conj(), h) / d


def project_out(V: np.ndarray, h: np.ndarray) -> np.ndarray:
    """h - proj_V h = h - sum_l <V[l], h> V[l] for orthonormal V (Section 3.2)."""
    if V.shape[0] == 0:
        return h.copy()
    beta = coefficients(V, h)
    return h - np.einsum("l,ljk->jk", beta, V)


# ------------------------------------------------------------- Algorithm 4
class CapacityError(RuntimeError):
    """More independent elements than the space can hold (or than requested)."""


@dataclass
class Alg4Result:
    V: np.ndarray                      # (dim, d, d) orthonormal basis
    dim: int
    candidates: int = 0                # generators + brackets tested
    accepted_rel: list = field(default_factory=list)   # rel. residuals of accepts
    rejected_rel: list = field(default_factory=list)   # rel. residuals of nonzero rejects
    max_imag_beta: float = 0.0         # diagnostic: beta is real for anti-Hermitian V, h
    l: int = 1                         # pair cursor (resumable state)
    m: int = 0
    saturated: bool = False
    t_total: float = 0.0
    t_last_accept: float = 0.0
    max_dim: int = 0

    @property
    def basis(self) -> np.ndarray:
        """The accepted orthonormal elements, (dim, d, d)."""
        return self.V[: self.dim]


def _test_and_append(n: int, h: np.ndarray, tol: float, eta_abs: float,
                     res: Alg4Result, tol_mode: str = "relative") -> int:
    """One independence check of Algorithm 4; returns the new |V| (res.V grows).

    "h_perp != 0" is read as ||h_perp|| > tol * ||h|| (tol_mode "relative",
    the default) or as ||h_perp|| > tol ("absolute": V has unit-norm elements,
    so the threshold is on the orthogonal part itself)."""
    V = res.V
    hn = norm(h)
    res.candidates += 1
    if hn <= eta_abs:
        return n
    Vn = V[:n]
    if n:
        beta = coefficients(Vn, h)
        res.max_imag_beta = max(res.max_imag_beta, float(np.max(np.abs(beta.imag))))
    r = project_out(Vn, h)          # first classical Gram-Schmidt pass
    r = project_out(Vn, r)          # second pass
    rn = norm(r)
    rel = rn / hn
    if (rn > tol) if tol_mode == "absolute" else (rel > tol):
        if n >= res.max_dim:
            raise CapacityError(f"closure dimension would exceed {res.max_dim}")
        if n == V.shape[0]:
            grown = np.zeros((max(4, 2 * n),) + V.shape[1:], dtype=np.complex128)
            grown[:n] = V[:n]
            res.V = V = grown
        V[n] = r / rn
        res.accepted_rel.append(rel)
        return n + 1
    if rel > 0.0:
        res.rejected_rel.append(rel)
    return n


def max_dim_bound(generators: np.ndarray) -> int:
    """Largest possible closure dimension for anti-Hermitian d x d generators:
    brackets are traceless, so the closure lies in su(d) plus the span of the
    generators' trace parts (at most one direction)."""
    d = generators.shape[1]
    has_trace = any(abs(np.trace(g)) > 1e-12 * max(1.0, np.abs(g).max()) for g in generators)
    return d * d - 1 + (1 if has_trace else 0)


def alg4_orthonormalization(generators: np.ndarray, tol: float, eta_abs: float = 1e-12,
                            saturation_exit: bool = False, max_candidates: int | None = None,
                            capacity: int | None = None, resume: Alg4Result | None = None,
                            max_dim: int | None = None, tol_mode: str = "relative") -> Alg4Result:
    """Algorithm 4: the dimension-only orthonormalisation method.

    generators: (k, d, d) complex array, taken in the given order.
    tol: residual tolerance, relative to ||h|| (tol_mode "relative") or
    absolute ("absolute"); eta_abs: absolute floor on ||h||.
    max_candidates: stop after this many candidate checks (timing samples);
    the returned result then carries the cursor (l, m) and can be resumed.
    max_dim: raise CapacityError rather than grow past this many elements.
    """
    t0 = time.perf_counter()
    k, d, _ = generators.shape
    if resume is None:
        cap = capacity if capacity is not None else min(d * d + 1, 64)
        # d x d complex matrices span a real space of dimension 2 d^2, so more
        # accepts than that means the arithmetic is broken
        res = Alg4Result(V=np.zeros((cap, d, d), dtype=np.complex128), dim=0,
                         max_dim=max_dim if max_dim is not None else 2 * d * d)
        n = 0
        # generator pass
        for g in generators:
            n = _test_and_append(n, np.asarray(g, dtype=np.complex128), tol, eta_abs, res, tol_mode)
            res.t_last_accept = time.perf_counter() - t0
        l, m = 1, 0
    else:
        res = resume
        n = res.dim
        l, m = res.l, res.m
    bound = max_dim_bound(generators) if saturation_exit else None
    budget = max_candidates
    # pair sweep: (l, m) with m < l, l ascending, m ascending; l < |V| re-read each step
    while l < n:
        if bound is not None and n >= bound:
            res.saturated = True
            break
        if budget is not None and budget <= 0:
            break
        h = bracket(res.V[l], res.V[m])
        n_before = n
        n = _test_and_append(n, h, tol, eta_abs, res, tol_mode)
        if n > n_before:
            res.t_last_accept = time.perf_counter() - t0
        if budget is not None:
            budget -= 1
        m += 1
        if m == l:
            l += 1
            m = 0
    res.dim = n
    res.l, res.m = l, m
    res.t_total += time.perf_counter() - t0
    return res


# ------------------------------------------------------------- Algorithm 2
@dataclass
class Alg2Result:
    B: np.ndarray          # (dim, d, d): unit-norm generators and nested brackets
    A_inv: np.ndarray      # (dim, dim): inverse of the Gram matrix A_ij = <B_i, B_j>
    dim: int
    candidates: int = 0
    residuals: list = field(default_factory=list)   # ||h - B (A^-1 beta)|| of accepts


def alg2_matrix_inversion(generators: np.ndarray, tol: float, eta_abs: float = 1e-12,
                          saturation_exit: bool = False) -> Alg2Result:
    """Algorithm 2: the matrix-inversion method (Section 3.1, Theorem 1).

    Operators enter B unit-normalised.  A candidate h (normalised) with
    beta_i = <B_i, h> is independent iff h - sum_i B_i (A^-1 beta)_i != 0, read
    as: its norm exceeds tol (h has unit norm, so this is the relative test);
    brackets with ||[B_l, B_m]|| <= eta_abs are zero.  On accept A grows by the
    row beta (A_{i,new} = beta_i, A_{new,i} = conj(beta_i), A_{new,new} = 1) and
    A^-1 is recomputed.  Brackets are formed from B.
    """
    k, d, _ = generators.shape
    cap = 2 * d * d
    B = np.zeros((min(cap, 64), d, d), dtype=np.complex128)
    A = np.zeros((0, 0), dtype=np.complex128)
    A_inv = np.zeros((0, 0), dtype=np.complex128)
    n = 0
    res = Alg2Result(B=B, A_inv=A_inv, dim=0)

    def try_append(h):
        nonlocal B, A, A_inv, n
        res.candidates += 1
        hn = norm(h)
        if hn <= eta_abs:
            return
        hb = h / hn
        beta = coefficients(B[:n], hb) if n else np.zeros(0, dtype=np.complex128)
        x = A_inv @ beta
        r = hb - np.einsum("l,ljk->jk", x, B[:n]) if n else hb
        rn = norm(r)
        if rn <= tol:
            return
        if n >= cap:
            raise CapacityError("closure dimension would exceed 2 d^2")
        if n == B.shape[0]:
            grown = np.zeros((max(4, 2 * n), d, d), dtype=np.complex128)
            grown[:n] = B[:n]
            B = grown
        B[n] = hb
        A_new = np.zeros((n + 1, n + 1), dtype=np.complex128)
        A_new[:n, :n] = A
        A_new[:n, n] = beta
        A_new[n, :n] = beta.conj()
        A_new[n, n] = 1.0
        A = A_new
        A_inv = np.linalg.inv(A)
        res.residuals.append(rn)
        n += 1

    for g in generators:
        try_append(np.asarray(g, dtype=np.complex128))
    bound = max_dim_bound(generators) if saturation_exit else None
    l, m = 1, 0
    while l < n:
        if bound is not None and n >= bound:
            break
        try_append(bracket(B[l], B[m]))
        m += 1
        if m == l:
            l += 1
            m = 0
    res.B, res.A_inv, res.dim = B[:n], A_inv, n
    return res


# ------------------------------------------------------------- Algorithm 3
@dataclass
class Alg3Result:
    B: np.ndarray          # (dim, d, d): the generators and nested brackets kept
    V: np.ndarray          # (dim, d, d): orthonormal basis of the same span
    dim: int
    parents: list          # per element of B: None (a generator) or (l, m)
    candidates: int = 0


def alg3_orthonormalization(generators: np.ndarray, tol: float, eta_abs: float = 1e-12,
                            saturation_exit: bool = False) -> Alg3Result:
    """Algorithm 3: the orthonormalisation method keeping the original basis.

    Two tuples grow together: B holds the accepted generators and nested
    brackets themselves, V their orthonormalised versions.  Brackets are formed
    from B; each is tested against V with the same rule as Algorithm 4
    (two classical Gram-Schmidt passes, relative tolerance, absolute floor).
    """
    k, d, _ = generators.shape
    cap = 2 * d * d
    B = np.zeros((min(cap, 64), d, d), dtype=np.complex128)
    V = np.zeros_like(B)
    parents: list = []
    n = 0
    count = 0

    def grow(arr, n):
        out = np.zeros((max(4, 2 * n),) + arr.shape[1:], dtype=np.complex128)
        out[:n] = arr[:n]
        return out

    def test(h):
        hn = norm(h)
        if hn <= eta_abs:
            return None
        r = project_out(V[:n], h)
        r = project_out(V[:n], r)
        rn = norm(r)
        return r / rn if rn > tol * hn else None

    for g in generators:
        g = np.asarray(g, dtype=np.complex128)
        count += 1
        v = test(g)
        if v is not None:
            if n >= cap:
                raise CapacityError("closure dimension would exceed 2 d^2")
            if n == B.shape[0]:
                B, V = grow(B, n), grow(V, n)
            B[n], V[n] = g, v
            parents.append(None)
            n += 1
    bound = max_dim_bound(generators) if saturation_exit else None
    l, m = 1, 0
    while l < n:
        if bound is not None and n >= bound:
            break
        h = bracket(B[l], B[m])
        count += 1
        v = test(h)
        if v is not None:
            if n >= cap:
                raise CapacityError("closure dimension would exceed 2 d^2")
            if n == B.shape[0]:
                B, V = grow(B, n), grow(V, n)
            B[n], V[n] = h, v
            parents.append((l, m))
            n += 1
        m += 1
        if m == l:
            l += 1
            m = 0
    return Alg3Result(B=B[:n], V=V[:n], dim=n, parents=parents, candidates=count)


# ------------------------------------------------------------- Algorithm 1
def alg1_rank(generators: np.ndarray, rank_tol: float | None = None) -> np.ndarray:
    """Algorithm 1 with the rank test: append h iff rank([B | h]) > rank(B).

    Operators are unit-normalised before they enter B (the paper reports that
    normalisation is needed for stability, Section 3.1).  Rank is the number of
    singular values above ``rank_tol * sigma_max`` (default max(rows, cols) *
    machine epsilon, the NumPy convention).  Returns B as (dim, d, d).
    Only for tiny inputs: each test is an SVD of a d^2 x (|B|+1) matrix.
    """
    k, d, _ = generators.shape
    B: list[np.ndarray] = []

    def independent(h: np.ndarray) -> bool:
        hn = norm(h)
        if hn <= 1e-12:
            return False
        cols = [b.reshape(-1) for b in B] + [(h / hn).reshape(-1)]
        M = np.stack(cols, axis=1)
        s = np.linalg.svd(M, compute_uv=False)
        tol_r = (rank_tol if rank_tol is not None else max(M.shape) * np.finfo(float).eps) * s[0]
        return int(np.sum(s > tol_r)) > len(B)

    for g in generators:
        if independent(g):
            B.append(g / norm(g))
    l, m = 1, 0
    while l < len(B):
        h = bracket(B[l], B[m])
        if independent(h):
            B.append(h / norm(h))
        m += 1
        if m == l:
            l += 1
            m = 0
    return np.stack(B) if B else np.zeros((0, d, d), dtype=np.complex128)


# ------------------------------------------------------- exact Pauli closure
def pauli_to_bits(label: str) -> tuple[int, int]:
    """Symplectic (x, z) bit vectors of a Pauli string (bit j = qubit j+1)."""
    x = z = 0
    for j, ch in enumerate(label):
        if ch in "XY":
            x |= 1 << j
        if ch in "ZY":
            z |= 1 << j
    return x, z


def bits_to_pauli(x: int, z: int, n: int) -> str:
    out = []
    for j in range(n):
        xb, zb = (x >> j) & 1, (z >> j) & 1
        out.append("IXZY"[xb + 2 * zb])
    return "".join(out)


def anticommute(p: tuple[int, int], q: tuple[int, int]) -> bool:
    """Two Pauli strings anticommute iff their symplectic form is odd."""
    return (bin((p[0] & q[1]) ^ (p[1] & q[0])).count("1") & 1) == 1


def pauli_closure(labels) -> list[str]:
    """Exact closure of {i P_s}: the bracket of two anticommuting strings is
    proportional to their product string (x and z XORed); of commuting strings
    it is zero.  Distinct strings are orthonormal under <a,b> = tr(a^dagger b)/d,
    so the closure dimension is the number of distinct strings reached.
    Returns the strings in discovery order (breadth first)."""
    n = len(labels[0])
    seen: dict[tuple[int, int], int] = {}
    order: list[tuple[int, int]] = []
    for s in labels:
        b = pauli_to_bits(s)
        if b == (0, 0):
            continue        # i*I is a valid generator but commutes with all
        if b not in seen:
            seen[b] = len(order)
            order.append(b)
    # the identity direction is handled separately: it never brackets to anything
    i = 0
    while i < len(order):
        p = order[i]
        for j in range(i):
            q = order[j]
            if anticommute(p, q):
                r = (p[0] ^ q[0], p[1] ^ q[1])
                if r not in seen:
                    seen[r] = len(order)
                    order.append(r)
        i += 1
    out = [bits_to_pauli(x, z, n) for x, z in order]
    if any(pauli_to_bits(s) == (0, 0) for s in labels):
        out.append("I" * n)
    return out


# ------------------------------------------------------------------ metrics
def _isometric_rows(V: np.ndarray) -> np.ndarray:
    """Rows vec(V[l]) / sqrt(d): the paper's inner product becomes the plain
    complex dot product of these rows."""
    N, d, _ = V.shape
    return V.reshape(N, d * d) / np.sqrt(d)


def gram(V: np.ndarray) -> np.ndarray:
    X = _isometric_rows(V)
    return X.conj() @ X.T


def ortho_defect(V: np.ndarray) -> float:
    """max |<v_i, v_j> - delta_ij| over the basis."""
    if V.shape[0] == 0:
        return 0.0
    G = gram(V)
    return float(np.max(np.abs(G - np.eye(G.shape[0]))))


def span_distance(V: np.ndarray, U: np.ndarray) -> float:
    """sin of the largest principal angle between span(U) and span(V):
    the spectral norm of (I - P_V) Q_U, with Q_U an orthonormal basis of span(U)
    (projector-residual form; accurate at small angles).  Both bases must have
    the same size, otherwise the distance is 1."""
    if V.shape[0] != U.shape[0]:
        return 1.0
    if V.shape[0] == 0:
        return 0.0
    X = _isometric_rows(V)
    Y = _isometric_rows(U)
    # orthonormal bases of both row spaces (QR is the library step)
    Qx, _ = np.linalg.qr(X.T)
    Qy, _ = np.linalg.qr(Y.T)
    E = Qy - Qx @ (Qx.conj().T @ Qy)
    return float(np.linalg.norm(E, 2))


def closure_residual(V: np.ndarray, pairs=None, eta_abs: float = 1e-12) -> float:
    """max over pairs (i, j) of ||[v_i, v_j] - proj_V [v_i, v_j]|| / ||[v_i, v_j]||,
    for orthonormal V.  All pairs i < j when ``pairs`` is None."""
    N = V.shape[0]
    if pairs is None:
        pairs = [(i, j) for i in range(N) for j in range(i)]
    worst = 0.0
    for i, j in pairs:
        h = bracket(V[i], V[j])
        hn = norm(h)
        if hn <= eta_abs:
            continue
        r = project_out(V, h)
        worst = max(worst, norm(r) / hn)
    return worst


def margin_report(res: Alg4Result) -> dict:
    """Smallest relative residual among accepts and largest among nonzero rejects."""
    acc = np.asarray(res.accepted_rel) if res.accepted_rel else np.asarray([np.inf])
    rej = np.asarray(res.rejected_rel) if res.rejected_rel else np.asarray([0.0])
    return {"min_acc_rel_res": float(acc.min()), "max_rej_rel_res": float(rej.max()),
            "n_acc": len(res.accepted_rel), "n_rej_nonzero": len(res.rejected_rel)}
