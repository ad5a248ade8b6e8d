"""GPU tests of the boundary's report fields and options (through the C ABI):
the device-computed orthonormality defect against the oracle's, the measured
screen threshold and gray count, the absolute tolerance reading against the
oracle, the autotuner (same basis as fixed parameters, cached choice), and
the device-pointer batched call against the host one."""
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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["so6", "su32_chain", "rand_d16"])
def test_report_ortho_defect_matches_oracle(prec, case):
    """rep.ortho_defect (FP64 Gram on the device, all rows since |V| <= 4096)
    equals the oracle's max |<v_i, v_j> - delta_ij| on the returned basis."""
    if case == "so6":
        g, _ = inputs.workload_generators("so6_chain_d8")
    elif case == "su32_chain":
        g = inputs.generators_from_labels(inputs.su2n_chain_labels(5))
    else:
        g = inputs.random_set(16, 2, seed=6)
    r = binding.lie_closure(g, 1e-8, precision=prec, ortho_check=1, saturation_exit=1)
    assert r.report["ortho_rows"] == r.dim
    want = oc.ortho_defect(r.basis)
    assert abs(r.report["ortho_defect"] - want) <= 1e-14
    assert r.report["ortho_defect"] < 1e-12


def test_report_ortho_defect_off_is_minus_one():
    g, _ = inputs.workload_generators("so6_chain_d8")
    r = binding.lie_closure(g, 1e-10, precision="mixed")
    assert r.report["ortho_defect"] == -1.0 and r.report["ortho_rows"] == 0


def test_measured_screen_threshold_is_reported_and_harmless():
    """The default (measured) tau_screen is kappa * eps_screen clamped to
    [2^-21, 1e-3]; the basis equals the oracle's and the fixed-threshold run's."""
    g = inputs.generators_from_labels(inputs.su2n_chain_labels(4))
    ref = oc.alg4_orthonormalization(g, 1e-10)
    r = binding.lie_closure(g, 1e-10, precision="mixed")
    rep = r.report
    assert 0.0 < rep["eps_screen"] < 1e-4
    assert 2.0 ** -21 <= rep["tau_screen"] <= 1e-3
    assert rep["tau_screen"] <= max(10.0 * rep["eps_screen"] * 1.0001, 2.0 ** -21)
    assert rep["n_gray"] >= 0
    assert rep["min_acc_screen_rel_res"] > rep["tau_screen"]
    np.testing.assert_allclose(r.basis, ref.basis, atol=1e-11, rtol=0)
    f = binding.lie_closure(g, 1e-10, precision="mixed", tau_screen=1e-3)
    assert f.report["tau_screen"] == 1e-3
    # another threshold flags another set, so the FP64 GEMMs see other row
    # counts (other split-K plans): equal to rounding
    np.testing.assert_allclose(r.basis, f.basis, atol=1e-13, rtol=0)


def test_fp64_mode_reports_no_screen_noise():
    g = inputs.random_set(8, 2, seed=3)
    r = binding.lie_closure(g, 1e-8, precision="fp64")
    assert r.report["eps_screen"] == 0.0 and r.report["n_gray"] == 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_absolute_tolerance_matches_oracle(prec):
    """g2 = 1e4 iXI + 1e-3 iZZ: rejected by the relative reading at tol 1e-6,
    accepted by the absolute one (the oracle's tol_mode pin), element by
    element; plus a random set where both readings agree."""
    a, zz = inputs.generators_from_labels(["XI", "ZZ"])
    g = np.stack([a, 1e4 * a + 1e-3 * zz])
    for mode, dim in (("relative", 1), ("absolute", 3)):
        ref = oc.alg4_orthonormalization(g, 1e-6, tol_mode=mode)
        r = binding.lie_closure(g, 1e-6, precision=prec, tol_mode=mode)
        assert r.dim == ref.dim == dim
        np.testing.assert_allclose(r.basis, ref.basis, atol=1e-11, rtol=0)
    g = inputs.random_set(6, 3, seed=12)
    ref = oc.alg4_orthonormalization(g, 1e-8, tol_mode="absolute")
    r = binding.lie_closure(g, 1e-8, precision=prec, tol_mode="absolute")
    assert r.dim == ref.dim == 35
    np.testing.assert_allclose(r.basis, ref.basis, atol=1e-11, rtol=0)


def test_bad_tol_mode_is_an_argument_error():
    g, _ = inputs.workload_generators("so6_chain_d8")
    r = binding.lie_closure(g, 1e-10, precision="mixed", tol_mode=7, check=False)
    assert r.status == binding.LC_ERR_ARG


def test_autotune_gives_the_same_basis_and_caches_its_choice():
    """su(64) chain, mixed: the autotuned call tries the three screening-GEMM
    tiles with four block sizes on its saturated-phase blocks (real
    candidates, each screened by the tile under trial) and returns the
    fixed-parameter basis (blocking and tiles change no decision; a trial
    block that falls in a pause of the growth groups the in-block FP64
    Gram-Schmidt differently, so equality is to FP64 rounding); the next call
    takes the cached choice without trials and returns the same basis."""
    g, _ = inputs.workload_generators("su64_chain_d64")
    fixed = binding.lie_closure(g, 1e-8, precision="mixed")
    a = binding.lie_closure(g, 1e-8, precision="mixed", autotune=1)
    assert a.dim == fixed.dim == 4095
    assert a.report["autotuned"] == 1 and a.report["autotune_trials"] == 12
    assert a.report["gemm_tile_n"] in (128, 256) and a.report["gemm_tile_k"] in (32, 64)
    assert a.report["block_k_used"] in (4096, 8192, 16384, 32768)
    np.testing.assert_allclose(a.basis, fixed.basis, atol=1e-13, rtol=0)
    b = binding.lie_closure(g, 1e-8, precision="mixed", autotune=1)
    assert b.report["autotuned"] == 1 and b.report["autotune_trials"] == 0
    assert (b.report["block_k_used"], b.report["gemm_tile_n"], b.report["gemm_tile_k"]) == \
        (a.report["block_k_used"], a.report["gemm_tile_n"], a.report["gemm_tile_k"])
    np.testing.assert_allclose(b.basis, fixed.basis, atol=1e-13, rtol=0)


def test_batched_dev_equals_batched_host():
    """lie_closure_batched_dev on device tensors returns the dimensions,
    statuses and bases of lie_closure_batched on the same sets."""
    import torch
    sets = inputs.batched_sets(24, seed=7)
    gens = [s["generators"] for s in sets]
    dims_h, st_h, bases_h, _ = binding.lie_closure_batched(gens, 1e-8, return_basis=True, saturation_exit=1)
    dg = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in gens]
    caps = [x.shape[1] ** 2 for x in gens]
    outs = [torch.zeros((c, x.shape[1], x.shape[1]), dtype=torch.complex128, device="cuda") for c, x in zip(caps, gens)]
    torch.cuda.synchronize()
    dims_d, st_d, reps = binding.lie_closure_batched_dev(dg, 1e-8, bases=outs, saturation_exit=1)
    assert st_d == st_h == [0] * len(sets)
    assert dims_d == dims_h
    for i, s in enumerate(sets):
        if s["kind"] == "pauli":
            assert dims_d[i] == len(oc.pauli_closure(s["labels"]))
        else:
            assert dims_d[i] == s["d"] ** 2 - 1
        np.testing.assert_allclose(outs[i][: dims_d[i]].cpu().numpy(), bases_h[i], atol=1e-13, rtol=0)
    # dimensions only (no output buffers)
    dims_n, st_n, _ = binding.lie_closure_batched_dev(dg, 1e-8, saturation_exit=1)
    assert dims_n == dims_h and st_n == st_h
