"""GPU parity for Algorithm 3 (generators and nested brackets kept beside V)
against the oracle's Algorithm 3, through the C ABI."""
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


def _case(name):
    if name == "so6":
        return inputs.generators_from_labels(inputs.so2n_chain_labels(3)), 1e-10
    if name == "su8":
        return inputs.generators_from_labels(inputs.su2n_chain_labels(3)), 1e-10
    if name == "rand_d4":
        return inputs.random_set(4, 2, seed=3), 1e-8
    if name == "rand_d6_k3":
        return inputs.random_set(6, 3, seed=13), 1e-8
    rng = np.random.default_rng(9)
    return inputs.generators_from_labels(inputs.random_pauli_labels(3, 4, rng)), 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["so6", "su8", "rand_d4", "rand_d6_k3", "pauli"])
def test_alg3_matches_oracle(prec, name):
    g, tol = _case(name)
    ref = oc.alg3_orthonormalization(g, tol)
    B, V, st, rep = binding.lie_closure_alg3(g, tol, precision=prec)
    assert st == binding.LC_OK and B.shape[0] == V.shape[0] == ref.dim
    scale = np.max(np.abs(ref.B), axis=(1, 2), keepdims=True)
    np.testing.assert_array_less(np.abs(B - ref.B) / scale, 1e-12)
    np.testing.assert_allclose(V, ref.V, atol=1e-11)
    assert oc.ortho_defect(V) < 1e-12
    assert oc.span_distance(B, V) < 1e-9


def test_alg3_su64_chain_tensor_path():
    """d = 64 (tensor-core brackets of B): su(64); the kept elements are
    generators or nested brackets of Pauli strings, i.e. powers of two times
    +-i times a Pauli string."""
    labels = inputs.su2n_chain_labels(6)
    g = inputs.generators_from_labels(labels)
    B, V, st, rep = binding.lie_closure_alg3(g, 1e-8, precision="mixed", saturation_exit=1)
    assert st == binding.LC_OK and B.shape[0] == 4095
    rng = np.random.default_rng(4)
    for i in rng.choice(4095, size=40, replace=False):
        b = B[i]
        nz = np.abs(b) > 1e-9
        assert np.all(nz.sum(axis=1) == 1)          # one nonzero per row, like a Pauli string
        mag = np.abs(b[nz])
        assert np.allclose(mag, mag[0]) and np.isclose(np.log2(mag[0]), round(np.log2(mag[0])))
    assert oc.ortho_defect(V[:512]) < 1e-12
