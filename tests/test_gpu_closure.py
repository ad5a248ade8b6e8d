"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars (written here, derived from the arithmetic):
* dimension: exact integer match;
* FP64 mode: every accepted element is an FP64 CGS2 result, so the basis
  matches the oracle's element by element within 1e-11 when the same
  candidates are accepted in the same order (same pair order, same test), and
  its span within 1e-9;
* mixed mode: accepted elements are recomputed in FP64 too, so the same bars
  hold whenever the screen passes every candidate the FP64 test accepts; the
  span bar of 1e-6 is the one stated for mixed precision;
* orthonormality defect <= 1e-12; closure residual <= 10 tol.
"""
import ctypes

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
    return binding.lib()


PRECS = ["fp64", "mixed"]


def _compare(res, ref, tol, prec, elementwise=True):
    assert res.dim == ref.dim
    V = res.basis
    assert oc.ortho_defect(V) < 1e-12
    assert oc.span_distance(V, ref.basis) < (1e-9 if prec == "fp64" else 1e-6)
    if elementwise:
        np.testing.assert_allclose(V, ref.basis, atol=1e-11, rtol=0)
    for v in V[: min(len(V), 64)]:
        np.testing.assert_allclose(v, -v.conj().T, atol=1e-14)


# ------------------------------------------------------------ split GEMM
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 300, 500), (64, 33, 17), (1000, 257, 4096), (7, 1, 3000)])
def test_split_gemm_matches_fp64(M, N, K):
    import torch
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g, dtype=torch.float32)
    B = torch.randn(N, K, generator=g, dtype=torch.float32)
    D = binding.lc_split_gemm_f32(A.cuda(), B.cuda()).cpu().double()
    ref = A.double() @ B.double().T
    # three-term BF16 split: ~3 * 2^-16 per product, plus FP32 accumulation
    bound = (3 * 2.0 ** -16 + K * 2.0 ** -24) * (A.double().abs() @ B.double().abs().T)
    assert torch.all((D - ref).abs() <= bound + 1e-30)
    assert ((D - ref).norm() / ref.norm()).item() < 2e-5


# ------------------------------------------------------------ full runs
@pytest.mark.parametrize("prec", PRECS)
def test_so6_chain_d8(prec):
    g, _ = inputs.workload_generators("so6_chain_d8")
    ref = oc.alg4_orthonormalization(g, 1e-10)
    res = binding.lie_closure(g, 1e-10, precision=prec)
    assert res.dim == 15
    _compare(res, ref, 1e-10, prec)
    assert res.report["brackets_checked"] == 15 * 14 // 2
    assert res.report["generators_checked"] == 5


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["su8_chain", "so8_chain_d16", "so10_chain_d32", "rand_d4", "rand_d8",
                                  "rand_d3_k3", "rand_d6_trace", "pauli_d8"])
def test_small_closures(prec, case):
    tol = 1e-8
    if case == "su8_chain":
        g = inputs.generators_from_labels(inputs.su2n_chain_labels(3)); tol = 1e-10
    elif case == "so8_chain_d16":
        g = inputs.generators_from_labels(inputs.so2n_chain_labels(4)); tol = 1e-10
    elif case == "so10_chain_d32":
        g = inputs.generators_from_labels(inputs.so2n_chain_labels(5)); tol = 1e-10
    elif case == "rand_d4":
        g = inputs.random_set(4, 2, seed=21)
    elif case == "rand_d8":
        g = inputs.random_set(8, 2, seed=22)
    elif case == "rand_d3_k3":
        g = inputs.random_set(3, 3, seed=23)
    elif case == "rand_d6_trace":
        g = inputs.random_set(6, 2, seed=24, traceless=False)
    else:
        rng = np.random.default_rng(25)
        g = inputs.generators_from_labels(inputs.random_pauli_labels(3, 4, rng))
    ref = oc.alg4_orthonormalization(g, tol)
    res = binding.lie_closure(g, tol, precision=prec)
    _compare(res, ref, tol, prec)
    assert oc.closure_residual(res.basis, pairs=[(i, j) for i in range(res.dim) for j in range(i)][:3000]) < 10 * tol


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["su16_chain", "rand_d16", "rand_d12_k3", "rand_d24"])
def test_growth_phase_d12_to_24(prec, case):
    """Ragged and multi-tile sizes; both sides stop at saturation (exact)."""
    tol = 1e-8
    if case == "su16_chain":
        g = inputs.generators_from_labels(inputs.su2n_chain_labels(4)); tol = 1e-10
    elif case == "rand_d16":
        g = inputs.random_set(16, 2, seed=6)
    elif case == "rand_d12_k3":
        g = inputs.random_set(12, 3, seed=9)
    else:
        g = inputs.random_set(24, 2, seed=31)
    ref = oc.alg4_orthonormalization(g, tol, saturation_exit=True)
    res = binding.lie_closure(g, tol, precision=prec, saturation_exit=1)
    assert res.dim == g.shape[1] ** 2 - 1
    _compare(res, ref, tol, prec)


def test_block_size_does_not_change_the_result():
    """Blocks are contiguous runs of the pair order: any block size gives the same V."""
    g = inputs.random_set(8, 2, seed=41)
    a = binding.lie_closure(g, 1e-8, precision="mixed", block_k=7)
    b = binding.lie_closure(g, 1e-8, precision="mixed", block_k=4096)
    c = binding.lie_closure(g, 1e-8, precision="fp64", block_k=1)
    assert a.dim == b.dim == c.dim == 63
    np.testing.assert_allclose(a.basis, b.basis, atol=1e-12)
    np.testing.assert_allclose(a.basis, c.basis, atol=1e-12)


# ------------------------------------------------------------ device API
def test_dev_api_matches_host_api():
    import torch
    g = inputs.random_set(8, 3, seed=51)
    host = binding.lie_closure(g, 1e-8)
    gd = torch.from_numpy(g).cuda()
    out = torch.zeros((64, 8, 8), dtype=torch.complex128, device="cuda")
    s = torch.cuda.Stream()
    dev = binding.lie_closure_dev(gd, 1e-8, max_dim=64, basis_out=out, stream=s)
    assert dev.dim == host.dim == 63
    np.testing.assert_allclose(out[:63].cpu().numpy(), host.basis, atol=1e-13)


# ------------------------------------------------------------ edge cases
def test_errors_and_capacity():
    g = inputs.random_set(4, 2, seed=61)
    bad = g.copy()
    bad[0, 0, 1] += 0.1
    r = binding.lie_closure(bad, 1e-8, check=False)
    assert r.status == binding.LC_ERR_NOT_ANTIHERMITIAN
    nan = g.copy()
    nan[1, 2, 2] = np.nan
    assert binding.lie_closure(nan, 1e-8, check=False).status == binding.LC_ERR_NONFINITE
    ref = oc.alg4_orthonormalization(g, 1e-8)
    for prec in PRECS:
        r = binding.lie_closure(g, 1e-8, max_dim=10, check=False, precision=prec)
        assert r.status == binding.LC_ERR_CAPACITY
        assert r.dim == 10
        np.testing.assert_allclose(r.basis, ref.basis[:10], atol=1e-12)


def test_degenerate_inputs():
    z = np.zeros((2, 4, 4), dtype=np.complex128)
    for prec in PRECS:
        assert binding.lie_closure(z, 1e-8, precision=prec).dim == 0
        one = inputs.generators_from_labels(["XY"])
        assert binding.lie_closure(one, 1e-8, precision=prec).dim == 1
        comm = inputs.generators_from_labels(["ZII", "IZI", "ZZI", "IIZ"])
        assert binding.lie_closure(comm, 1e-8, precision=prec).dim == 4
        dup = inputs.generators_from_labels(["XI", "XI", "IZ"])
        dup[1] *= -2.5
        assert binding.lie_closure(dup, 1e-8, precision=prec).dim == 2


def test_max_candidates_prefix_and_cursor():
    g = inputs.generators_from_labels(inputs.su2n_chain_labels(3))
    ref = oc.alg4_orthonormalization(g, 1e-10, max_candidates=500)
    r = binding.lie_closure(g, 1e-10, precision="mixed", max_candidates=500)
    assert r.report["brackets_checked"] == 500
    assert (r.report["cursor_l"], r.report["cursor_m"]) == (ref.l, ref.m)
    assert r.dim == ref.dim
    np.testing.assert_allclose(r.basis, ref.basis, atol=1e-12)


# ------------------------------------------------------------ batched
def test_batched_small_sets():
    sets = [s for s in inputs.batched_sets(64, seed=1120, dims=(8, 16)) if s["d"] == 8][:6]
    sets += [s for s in inputs.batched_sets(64, seed=1120, dims=(8, 16)) if s["kind"] == "pauli"][:4]
    dims, stat, bases, reps = binding.lie_closure_batched([s["generators"] for s in sets], 1e-8,
                                                          return_basis=True, saturation_exit=1)
    for s, dim, st, B in zip(sets, dims, stat, bases):
        assert st == 0
        if s["kind"] == "pauli":
            assert dim == len(oc.pauli_closure(s["labels"]))
        else:
            ref = oc.alg4_orthonormalization(s["generators"], 1e-8, saturation_exit=True)
            assert dim == ref.dim
            assert oc.span_distance(B, ref.basis) < 1e-6


# ------------------------------------------------------------ failure detection
def test_forced_wait_timeout_is_reported_and_device_stays_usable():
    """The accept kernel's grid barrier is told to expect one arrival more than
    there are CTAs (a flag nothing sets); its bounded wait runs out after
    spin_cap ns, the kernel records LC_ERR_TIMEOUT and returns, and the next
    call on the same device works."""
    g = inputs.generators_from_labels(inputs.su2n_chain_labels(3))
    for prec in PRECS:
        r = binding.lie_closure(g, 1e-10, precision=prec, fault_inject=1, spin_cap=50_000_000, check=False)
        assert r.status == binding.LC_ERR_TIMEOUT
        ok = binding.lie_closure(g, 1e-10, precision=prec)
        assert ok.status == binding.LC_OK and ok.dim == 63


# ------------------------------------------------------------ checkpoint / resume
@pytest.mark.parametrize("prec", PRECS)
def test_resume_equals_uninterrupted_run(prec):
    """Algorithm 4's state is (V, l, m): a run stopped after a prefix of the
    sweep and resumed from its returned basis and cursor gives the same basis as
    one run, and matches the oracle's resumed run."""
    for g, tol, cut in [(inputs.generators_from_labels(inputs.su2n_chain_labels(3)), 1e-10, 700),
                        (inputs.random_set(8, 2, seed=71), 1e-8, 150)]:
        full = binding.lie_closure(g, tol, precision=prec)
        part = binding.lie_closure(g, tol, precision=prec, max_candidates=cut)
        cur = (part.report["cursor_l"], part.report["cursor_m"])
        rest = binding.lie_closure_resume(part.basis, cur, tol, precision=prec)
        assert rest.dim == full.dim
        np.testing.assert_allclose(rest.basis, full.basis, atol=1e-12)
        ref = oc.alg4_orthonormalization(g, tol, max_candidates=cut)
        assert (ref.l, ref.m) == cur
        np.testing.assert_allclose(rest.basis, oc.alg4_orthonormalization(g, tol, resume=ref).basis, atol=1e-11)
