"""Pins of the oracle's periodic walls (CPU only): the identified mesh is a cylinder, fields are
single-valued across the identified edges, free flight wraps by the period, and the discrete
continuity equation holds through the wall.  The paper's Bernstein strip is periodic top and bottom
(Sec. III.C); particles leaving one wall re-enter at the corresponding point of the other with the
same momentum."""
import numpy as np

from paper_1707_04333_gb300 import inputs

C = inputs.C_LIGHT
QE, ME = inputs.Q_E, inputs.M_E


def _mesh(nx=10, ny=6, lx=1.3, ly=0.7, seed=9):
    return inputs.jittered_delaunay(nx, ny, lx, ly, 0.3, seed, periodic_y=True)


def test_identified_mesh_is_a_cylinder(oracle_mod):
    """Euler characteristic 0 (an annulus) once each top node is the bottom node below it; only the
    left and right walls remain boundary; S~ C^T = 0; each identified edge is crossed with opposite
    shifts from its two triangles."""
    m = _mesh()
    pairs, (tx, ty) = m.periodic
    om = oracle_mod.OracleMesh(m.nodes, m.triangles, m.periodic)
    nv = om.nn - len(pairs)
    assert nv - om.ne + om.nf == 0
    nb = int(om.edge_bnd.sum())
    assert nb == 2 * 6                                   # two walls of ny edges
    assert 3 * om.nf == 2 * om.ne - nb
    Z = (om.div_dual() @ om.curl().T).tocoo()
    assert np.all(Z.data == 0)
    sh = om.tri_shift
    assert (sh != 0).sum() == 2 * 10                     # nx periodic edges, seen from both sides
    for f, k in zip(*np.nonzero(sh)):
        g = om.tri_nb[f, k]
        k2 = list(om.tri_edge[g]).index(om.tri_edge[f, k])
        assert sh[g, k2] == -sh[f, k]
    # the top copy of a periodic edge moves down by one period
    ytop = om.ny[np.nonzero(sh == -1)[0]].max(axis=1)
    assert np.allclose(ytop, m.ly)


def test_fields_single_valued_across_the_wall(oracle_mod):
    """A uniform field loaded as e = E0 . (r_j - r_i) is reproduced everywhere (edge vectors read off
    either copy agree); for arbitrary e, the tangential component at the midpoint of each copy of an
    identified edge integrates to its single unknown."""
    m = _mesh(seed=11)
    om = oracle_mod.OracleMesh(m.nodes, m.triangles, m.periodic)
    E0 = np.array([-0.8, 0.45])
    e = om.edge_vectors() @ E0
    rng = np.random.default_rng(2)
    pts = inputs.sample_in_triangles(m, np.arange(len(m.triangles)).repeat(2), rng)
    np.testing.assert_allclose(om.field_at(e, pts[:, 0], pts[:, 1]), np.broadcast_to(E0, (len(pts), 2)),
                               rtol=0, atol=1e-13)
    e = rng.normal(size=om.ne)
    for f, k in zip(*np.nonzero(om.tri_shift)):
        a, b = (k + 1) % 3, (k + 2) % 3
        pa = np.array([om.nx[f, a], om.ny[f, a]])
        pb = np.array([om.nx[f, b], om.ny[f, b]])
        mid = 0.5 * (pa + pb)
        E = om.field_at(e, [mid[0]], [mid[1]], cell=[f])[0]
        g = om.tri_edge[f, k]
        assert abs(E @ (pb - pa) * om.tri_sign[f, k] - e[g]) < 1e-12 * (1 + abs(e[g]))


def _free_flight(oracle_mod, m, x0, d, dt=1e-7):
    sim = oracle_mod.OracleSim(m.nodes, m.triangles, dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                               spai_level=1, periodic=m.periodic)
    v = d / dt
    v2 = (v * v).sum(1) / (C * C)
    assert v2.max() < 1
    sim.load(QE, ME, x0, v / np.sqrt(1 - v2)[:, None])
    recs = sim.step("boris", record=64, only_particles=True)
    s = sim.species[0]
    return np.stack([s["x"], s["y"]], 1), recs[0], sim


def test_free_flight_wraps_by_the_period(oracle_mod):
    """E = B = 0: the end point is x0 + d with y taken modulo the period, also for paths that wrap
    more than once in one step; crossings of the periodic wall are recorded as edge crossings, not
    wall reflections."""
    m = _mesh(seed=13)
    rng = np.random.default_rng(4)
    n = 200
    x0 = np.stack([rng.uniform(0.2, 1.1, n), rng.uniform(0.0, m.ly, n)], 1)
    d = np.stack([rng.uniform(-0.05, 0.05, n), rng.uniform(-2.3, 2.3, n) * m.ly], 1)
    got, (cnt, rec), sim = _free_flight(oracle_mod, m, x0, d)
    want_y = np.mod(x0[:, 1] + d[:, 1], m.ly)
    np.testing.assert_allclose(got[:, 0], x0[:, 0] + d[:, 0], rtol=0, atol=1e-12)
    dy = np.abs(got[:, 1] - want_y)
    dy = np.minimum(dy, m.ly - dy)                        # a point on the wall may sit on either copy
    assert dy.max() < 1e-12
    assert (got[:, 1] >= 0).all() and (got[:, 1] <= m.ly).all()
    om = sim.mesh
    wraps = np.floor((x0[:, 1] + d[:, 1]) / m.ly).astype(int)
    assert (wraps != 0).sum() > 100
    periodic_edges = set(om.tri_edge[np.nonzero(om.tri_shift)])
    for p in np.nonzero(wraps != 0)[0]:
        crossed = [e for e in rec[p, :cnt[p]] if e >= 0]
        assert (rec[p, :cnt[p]] >= 0).all()               # no reflections in x range [0.15, 1.15]
        assert sum(e in periodic_edges for e in crossed) == abs(wraps[p])


def test_continuity_through_the_periodic_wall(oracle_mod):
    """DCE (Eq. full.dis.cont) at round-off every step on a periodic strip, with many particles
    crossing the identified wall."""
    w = inputs.pair_plasma(8, 6, kT=0.3, wc_over_wp=0.5, seed=33, pusher="vay", ny=4, periodic_y=True)
    m = w.mesh
    sim = oracle_mod.OracleSim(m.nodes, m.triangles, w.dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                               spai_level=1, b0=w.b0, periodic=m.periodic)
    rng = np.random.default_rng(33)
    for k, s in enumerate(w.species):
        x = s.x.copy()
        if k == 1:                                        # unpair so the charge density is nonzero
            x[:, 0] = np.clip(x[:, 0] + rng.normal(0, 0.05 * m.lx, len(x)), 1e-9, m.lx * (1 - 1e-9))
            x[:, 1] = np.mod(x[:, 1] + rng.normal(0, 0.3 * m.ly, len(x)), m.ly)
            sim.load(s.q, s.m, x, s.u, None)
        else:
            sim.load(s.q, s.m, x, s.u, s.hint)
    om = sim.mesh
    S = om.div_dual()
    periodic_edges = set(om.tri_edge[np.nonzero(om.tri_shift)])
    q0 = sim.charge()
    through = 0
    for n in range(40):
        recs = sim.step("vay", record=8)
        for cnt, rec in recs:
            for p in np.nonzero(cnt)[0]:
                through += sum(int(e) in periodic_edges for e in rec[p, :cnt[p]])
        q1 = sim.charge()
        res = (q1 - q0) + sim.dt * (S @ sim.i)
        scale = abs(S) @ sim.i_abs * sim.dt
        touched = scale > 0
        assert (np.abs(res[touched]) / scale[touched]).max() < 1e-12, n
        assert np.abs(res[~touched]).max() == 0.0
        q0 = q1
    assert through > 20
