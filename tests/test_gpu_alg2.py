"""GPU parity for Algorithm 2 (the matrix-inversion method) against the
oracle's Algorithm 2, through the C ABI.  Bars: equal dimension, B (unit-norm
generators and normalised brackets) equal element by element within 1e-10,
and the same span as Algorithm 4."""
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


@pytest.mark.parametrize("name", ["so6", "su8", "rand_d4", "rand_d3_k3", "pauli", "dependent"])
def test_alg2_matches_oracle(name):
    tol = 1e-10
    if name == "so6":
        g = inputs.generators_from_labels(inputs.so2n_chain_labels(3))
    elif name == "su8":
        g = inputs.generators_from_labels(inputs.su2n_chain_labels(3))
    elif name == "rand_d4":
        g = inputs.random_set(4, 2, seed=3); tol = 1e-8
    elif name == "rand_d3_k3":
        g = inputs.random_set(3, 3, seed=23); tol = 1e-8
    elif name == "pauli":
        rng = np.random.default_rng(9)
        g = inputs.generators_from_labels(inputs.random_pauli_labels(3, 4, rng))
    else:
        a, b = inputs.generators_from_labels(["XX", "ZZ"])
        g = np.stack([a, b, 0.3 * a - 2 * b])
    ref = oc.alg2_matrix_inversion(g, tol)
    r = binding.lie_closure_alg2(g, tol)
    assert r.dim == ref.dim
    np.testing.assert_allclose(r.basis, ref.B, atol=1e-10)
    r4 = oc.alg4_orthonormalization(g, tol)
    assert oc.span_distance(r4.basis, r.basis) < 1e-9


def test_alg2_su16_chain_saturation():
    g = inputs.generators_from_labels(inputs.su2n_chain_labels(4))
    r = binding.lie_closure_alg2(g, 1e-10, saturation_exit=1)
    assert r.dim == 255
    G = oc.gram(r.basis)
    assert np.max(np.abs(G - np.eye(255))) < 1e-12      # Pauli strings: B is orthonormal already
