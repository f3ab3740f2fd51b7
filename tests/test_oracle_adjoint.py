"""Pins for oracle.adjoint: analytic gradients against central finite differences (FP64)."""
import numpy as np
import pytest

from oracle import adjoint as A



@pytest.fixture(scope="module")
def field():
    rng = np.random.default_rng(17)
    n, box = 16, 200.0
    mesh = rng.standard_normal((n, n, n))
    return mesh, n, box


def test_power_gradient_fd(field):
    mesh, n, box = field
    kb, ells = (0.02, 0.04, 5), (0, 2, 4)
    rng = np.random.default_rng(1)
    dldp = {l: rng.standard_normal(kb[2]) for l in ells}

    def loss(m):
        p = A.power_from_mesh(m, box, 3, kb, ells, 2.5, 0.3, los=(0, 0, 1))
        return sum(np.dot(dldp[l], p[l]) for l in ells)

    grad = A.power_mesh_grad(mesh, box, 3, kb, ells, 2.5, dldp, los=(0, 0, 1))
    eps = 1e-4
    for c in rng.integers(0, n, size=(12, 3)):
        e = np.zeros_like(mesh)
        e[tuple(c)] = eps
        fd = (loss(mesh + e) - loss(mesh - e)) / (2 * eps)
        assert fd == pytest.approx(grad[tuple(c)], rel=1e-6, abs=1e-9 * np.max(np.abs(grad)))


def test_bispec0_gradient_fd(field):
    mesh, n, box = field
    kb = (0.03, 0.03, 3)    # k_max = 0.12 < k_N/2 = 0.1257
    rng = np.random.default_rng(2)
    dldb = rng.standard_normal(kb[2])

    def loss(m):
        return np.dot(dldb, A.bispec0_equilateral(m, box, 3, kb, 1.7))

    grad = A.bispec0_mesh_grad(mesh, box, 3, kb, 1.7, dldb)
    eps = 1e-4
    for c in rng.integers(0, n, size=(10, 3)):
        e = np.zeros_like(mesh)
        e[tuple(c)] = eps
        fd = (loss(mesh + e) - loss(mesh - e)) / (2 * eps)
        assert fd == pytest.approx(grad[tuple(c)], rel=1e-6, abs=1e-9 * np.max(np.abs(grad)))


def test_tsc_adjoint_fd():
    rng = np.random.default_rng(3)
    n = 12
    s = rng.random((40, 3)) * n
    w = 0.5 + rng.random(40)
    G = rng.standard_normal((n, n, n))

    def loss(ss):
        return np.sum(G * A.paint_tsc(ss, w, n))

    grad = A.tsc_adjoint(s, w, G)
    eps = 1e-6
    for p in range(0, 40, 7):
        for a in range(3):
            e = np.zeros_like(s)
            e[p, a] = eps
            fd = (loss(s + e) - loss(s - e)) / (2 * eps)
            assert fd == pytest.approx(grad[p, a], rel=1e-6, abs=1e-8)


def test_gradient_is_linear_in_dldp(field):
    mesh, n, box = field
    kb, ells = (0.0, 0.05, 4), (0, 2)
    g1 = {0: np.ones(4), 2: np.zeros(4)}
    g2 = {0: np.zeros(4), 2: np.ones(4)}
    g12 = {0: np.ones(4), 2: np.ones(4)}
    a = A.power_mesh_grad(mesh, box, 2, kb, ells, 1.0, g1)
    b = A.power_mesh_grad(mesh, box, 2, kb, ells, 1.0, g2)
    c = A.power_mesh_grad(mesh, box, 2, kb, ells, 1.0, g12)
    np.testing.assert_allclose(a + b, c, atol=1e-12 * np.max(np.abs(c)))

