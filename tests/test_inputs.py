"""Checks of the seeded workload generators (CPU only)."""
import json
import math
import os

import numpy as np

from paper_1707_04333_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def test_constants_reproduce_paper_bernstein_numbers():
    """Sec. III.C(b): omega_c = eB/m for 5 T, n = omega_p^2 eps0 m / e^2, lambda_D = v_th/omega_p
    with k_B T = m c^2/eta, eta = 20."""
    g = json.load(open(GOLDEN))["bernstein"]
    wc = inputs.Q_E * g["B0"] / inputs.M_E
    np.testing.assert_allclose(wc, g["omega_c"], rtol=1e-4)
    n = g["omega_p"] ** 2 * inputs.EPS0 * inputs.M_E / inputs.Q_E ** 2
    np.testing.assert_allclose(n, g["n"], rtol=1e-4)
    lam_d = inputs.C_LIGHT * math.sqrt(1.0 / g["eta"]) / g["omega_p"]
    np.testing.assert_allclose(lam_d, g["lambda_D"], rtol=1e-2)
    np.testing.assert_allclose(g["omega_p"] / g["omega_c"], 3.0, rtol=1e-4)


def test_maxwell_juttner_2d_mean_gamma():
    """pdf(gamma) ~ gamma exp(-eta gamma) on [1, inf): E[gamma] = 1 + (eta+2)/(eta(eta+1))."""
    rng = np.random.default_rng(0)
    for eta in (10.0, 2.0):
        u = inputs.maxwell_juttner_2d(400_000, eta, rng)
        g = np.sqrt(1 + (u ** 2).sum(1) / inputs.C_LIGHT ** 2)
        want = 1 + (eta + 2) / (eta * (eta + 1))
        assert abs(g.mean() - want) < 4 * g.std() / math.sqrt(len(g))
        # isotropy
        assert abs(u[:, 0].mean()) < 5 * u[:, 0].std() / math.sqrt(len(u))


def test_mesh_covers_rectangle_and_is_seeded():
    m1 = inputs.jittered_delaunay(20, 14, 2.0, 1.0, 0.3, seed=3)
    m2 = inputs.jittered_delaunay(20, 14, 2.0, 1.0, 0.3, seed=3)
    assert np.array_equal(m1.triangles, m2.triangles) and np.array_equal(m1.nodes, m2.nodes)
    p, t = m1.nodes, m1.triangles
    a = 0.5 * ((p[t[:, 1], 0] - p[t[:, 0], 0]) * (p[t[:, 2], 1] - p[t[:, 0], 1])
               - (p[t[:, 2], 0] - p[t[:, 0], 0]) * (p[t[:, 1], 1] - p[t[:, 0], 1]))
    assert (a > 0).all()
    np.testing.assert_allclose(a.sum(), 2.0, rtol=1e-13)
    assert len(t) == 2 * 20 * 14


def test_pair_plasma_shape():
    w = inputs.pair_plasma(10, 4, seed=9)
    e, p = w.species
    assert len(e.x) == len(w.mesh.triangles) * 4
    np.testing.assert_array_equal(e.x, p.x)
    np.testing.assert_array_equal(e.u, -p.u)
    assert e.q == -p.q and e.m == p.m
