"""Pins of the oracle's topology, Whitney forms and Hodge/SPAI setup (CPU only).

Each test checks the oracle against something fixed by the paper or by
mathematics, not against a retyped copy of its own formulas.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1707_04333_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


@pytest.fixture(scope="module")
def mesh(oracle_mod):
    m = inputs.jittered_delaunay(12, 10, 1.3, 0.9, 0.3, seed=7)
    return m, oracle_mod.OracleMesh(m.nodes, m.triangles)


def test_euler_and_paper_mesh_counts(mesh):
    """V - E + F = 1 for a triangulated disk; the paper's Bernstein mesh (Sec. III.C(b)) obeys it too."""
    g = json.load(open(GOLDEN))["bernstein_mesh"]
    assert g["nodes"] - g["edges"] + g["faces"] == 1
    _, om = mesh
    assert om.nn - om.ne + om.nf == 1
    # every interior edge has two faces, boundary edges one: 3F = 2E - E_b
    assert 3 * om.nf == 2 * om.ne - int(om.edge_bnd.sum())


def test_incidence_div_curl_zero(mesh):
    """S~ C^T = 0 exactly (integers in {-1,0,1}, Sec. II.A): the dual divergence of a curl vanishes."""
    _, om = mesh
    Cm = om.curl()
    S = om.div_dual()
    assert set(np.unique(Cm.data)) <= {-1.0, 1.0}
    Z = (S @ Cm.T).tocoo()
    assert np.all(Z.data == 0.0)
    # each face sees 3 edges, each edge 1 or 2 faces with opposite circulation signs
    colsum = np.asarray(abs(Cm).sum(axis=0)).ravel()
    assert set(np.unique(colsum)) <= {1.0, 2.0}
    interior = om.edge_bnd == 0
    assert np.all(np.asarray(Cm.sum(axis=0)).ravel()[interior] == 0.0)


def test_orientation_and_neighbours(mesh):
    _, om = mesh
    assert np.all(om.d2A > 0)
    for f in range(om.nf):
        for m in range(3):
            nb = om.tri_nb[f, m]
            if nb < 0:
                assert om.edge_bnd[om.tri_edge[f, m]] == 1
                continue
            m2 = list(om.tri_edge[nb]).index(om.tri_edge[f, m])
            assert om.tri_nb[nb, m2] == f
            # opposite circulation across a shared edge
            assert om.tri_sign[f, m] == -om.tri_sign[nb, m2]


def _barycentric_numpy(nodes, tri, pts):
    """Independent barycentrics: solve [x0 x1 x2; y0 y1 y2; 1 1 1] l = [x; y; 1]."""
    T = np.stack([nodes[tri, 0], nodes[tri, 1], np.ones(3)])
    return np.linalg.solve(T, np.vstack([pts.T, np.ones(len(pts))])).T


def test_lambdas_match_linear_solve(mesh):
    m, om = mesh
    rng = np.random.default_rng(0)
    for f in rng.integers(0, om.nf, 20):
        w = rng.dirichlet([1, 1, 1], 5)
        pts = w @ m.nodes[om.tri[f]]
        lam = om.lambdas(np.full(5, f), pts[:, 0], pts[:, 1])
        ref = _barycentric_numpy(m.nodes, om.tri[f], pts)
        np.testing.assert_allclose(lam, ref, atol=1e-13)
        np.testing.assert_allclose(lam.sum(1), 1.0, atol=1e-14)


def test_hodge_uniform_field_energy(mesh):
    """e.[*eps].e = eps0 |E0|^2 * area for a uniform field projected on all edges (Whitney exactness)."""
    m, om = mesh
    eps0 = 8.8541878128e-12
    H = om.hodge_eps(eps0)
    assert abs(H - H.T).max() < 1e-25
    E0 = np.array([3.0, -2.0])
    t = m.nodes[om.edge[:, 1]] - m.nodes[om.edge[:, 0]]
    e = t @ E0
    area = 0.5 * om.d2A.sum()
    np.testing.assert_allclose(area, m.lx * m.ly, rtol=1e-13)
    np.testing.assert_allclose(e @ (H @ e), eps0 * (E0 @ E0) * area, rtol=1e-12)
    # SPD on free edges
    Af = H[om.free][:, om.free].toarray()
    assert np.linalg.eigvalsh(Af).min() > 0


def test_spai_converges_to_dense_inverse(oracle_mod):
    """Level-k SPAI: Frobenius residual decreases with k and reaches the exact inverse (Sec. II.A)."""
    m = inputs.jittered_delaunay(5, 4, 1.0, 1.0, 0.3, seed=3)
    om = oracle_mod.OracleMesh(m.nodes, m.triangles)
    A = om.hodge_eps(1.0)[om.free][:, om.free].tocsr()
    n = A.shape[0]
    Ainv = np.linalg.inv(A.toarray())
    res = []
    for k in range(1, 12):
        M = oracle_mod.spai(A, k)
        res.append(np.linalg.norm(np.eye(n) - A @ M.toarray()))
    assert all(res[i + 1] <= res[i] * (1 + 1e-12) for i in range(len(res) - 1))
    assert res[0] > 1e-3
    M = oracle_mod.spai(A, 40)
    np.testing.assert_allclose(M.toarray(), Ainv, rtol=0, atol=1e-12 * np.abs(Ainv).max())


def test_spai_level1_pattern(oracle_mod):
    m = inputs.jittered_delaunay(6, 6, 1.0, 1.0, 0.3, seed=4)
    om = oracle_mod.OracleMesh(m.nodes, m.triangles)
    A = om.hodge_eps(1.0)[om.free][:, om.free].tocsr()
    M = oracle_mod.spai(A, 1)
    pa = (A != 0).astype(int)
    pm = (M != 0).astype(int)
    assert (pm - pa).nnz == 0 or ((pm - pa) > 0).nnz == 0
    # symmetric
    assert abs(M - M.T).max() < 1e-12 * abs(M).max()


def test_field_at_reproduces_uniform_field(mesh):
    """Whitney 1-forms span the constant fields: edge unknowns e_ij = E0 . (r_j - r_i) of a uniform
    E0 give back E0 at any point of any triangle (Sec. II.B), to round-off."""
    m, om = mesh
    E0 = np.array([0.37, -1.21])
    r = m.nodes
    e = (r[om.edge[:, 1]] - r[om.edge[:, 0]]) @ E0
    rng = np.random.default_rng(3)
    pts = inputs.sample_in_triangles(m, np.arange(len(m.triangles)).repeat(3), rng)
    got = om.field_at(e, pts[:, 0], pts[:, 1])
    np.testing.assert_allclose(got, np.broadcast_to(E0, got.shape), rtol=0, atol=1e-13)


def test_field_at_edge_circulation_and_tangential_continuity(mesh):
    """For arbitrary edge unknowns, the field's tangential component is constant along each edge and
    its line integral is the edge unknown (the defining property of the Whitney 1-form basis), so at
    an edge midpoint E . (r_j - r_i) = e_ij from either neighbouring triangle."""
    _, om = mesh
    rng = np.random.default_rng(5)
    e = rng.normal(size=om.ne)
    r = np.asarray(om.xy)
    checked = 0
    for f in range(om.nf):
        for k in range(3):
            g = om.tri_edge[f, k]
            i, j = om.edge[g]
            for t in (0.5, 0.2):
                p = r[i] + t * (r[j] - r[i])
                E = om.field_at(e, [p[0]], [p[1]], cell=[f])[0]
                assert abs(E @ (r[j] - r[i]) - e[g]) < 1e-12 * (1 + abs(e[g]))
                checked += 1
    assert checked == 6 * om.nf
