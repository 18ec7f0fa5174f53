"""Pins of the oracle's walk, current deposit and conservation laws (CPU only)."""
import math

import numpy as np
import pytest

from paper_1707_04333_gb300 import inputs

C = inputs.C_LIGHT
QE, ME = inputs.Q_E, inputs.M_E


def _bary(nodes, tri, pts):
    T = np.stack([nodes[tri, 0], nodes[tri, 1], np.ones(3)])
    return np.linalg.solve(T, np.vstack([pts.T, np.ones(len(pts))])).T


def brute_force_cells(nodes, tris, p0, p1, eps=1e-12):
    """All triangles whose interior the segment p0->p1 crosses with positive length,
    ordered by entry parameter: clip [0,1] against each triangle's three half-planes."""
    out = []
    for f, t in enumerate(tris):
        l0 = _bary(nodes, t, p0[None])[0]
        l1 = _bary(nodes, t, p1[None])[0]
        lo, hi = 0.0, 1.0
        for k in range(3):
            a, b = l0[k], l1[k]
            if a < 0 and b < 0:
                lo, hi = 1.0, 0.0
                break
            if a < 0 <= b:
                lo = max(lo, a / (a - b))
            elif b < 0 <= a:
                hi = min(hi, a / (a - b))
        if hi - lo > eps:
            out.append((lo, hi, f))
    out.sort()
    return out


def _free_flight(oracle_mod, m, x0, x1, hint=None, dt=1e-7, record=64):
    """Move particles from x0 to x1 in one step with E = B = 0 (the push leaves u unchanged)."""
    sim = oracle_mod.OracleSim(m.nodes, m.triangles, dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                               spai_level=1)
    d = (x1 - x0) / dt                      # = v; u = gamma v
    v2 = (d * d).sum(1) / (C * C)
    assert v2.max() < 1
    u = d / np.sqrt(1 - v2)[:, None]
    cell0 = sim.load(QE, ME, x0, u, hint).copy()
    recs = sim.step("boris", record=record, only_particles=True)
    s = sim.species[0]
    return sim, cell0, recs[0], np.stack([s["x"], s["y"]], 1)


def _cells_from_record(om, c0, cnt, rec):
    cells = [c0]
    for k in range(cnt):
        e = rec[k]
        f = cells[-1]
        if e < 0:
            continue
        m = list(om.tri_edge[f]).index(e)
        cells.append(om.tri_nb[f, m])
    return cells


def test_walk_matches_brute_force(oracle_mod):
    """Ordered cell list of the walk = brute-force line/triangle clipping, for random segments
    spanning several cells (Sec. II.D needs the path split per triangle)."""
    m = inputs.jittered_delaunay(5, 5, 1.0, 1.0, 0.3, seed=21)   # 50 triangles
    rng = np.random.default_rng(0)
    n = 3000
    x0 = rng.uniform(0.02, 0.98, (n, 2))
    x1 = np.clip(x0 + rng.normal(0, 0.3, (n, 2)), 0.01, 0.99)
    sim, cell0, (cnt, rec), xend = _free_flight(oracle_mod, m, x0, x1)
    om = sim.mesh
    for p in range(n):
        bf = brute_force_cells(m.nodes, om.tri, x0[p], xend[p])
        walk = _cells_from_record(om, cell0[p], cnt[p], rec[p])
        # collapse zero-length visits the brute force cannot see
        bf_cells = [f for _, _, f in bf]
        assert bf_cells == walk or [c for c in walk if c in bf_cells] == bf_cells, (p, bf, walk)
        assert walk[-1] == sim.species[0]["cell"][p]
        assert set(bf_cells) <= set(walk)


def test_walk_through_vertices_and_along_edges(oracle_mod):
    """Degenerate segments: aimed exactly at vertices and lying on edges.  The walk must end in a
    triangle containing the end point, visit neighbours only, and telescope the charge exactly."""
    m = inputs.jittered_delaunay(5, 5, 1.0, 1.0, 0.3, seed=22)
    om = oracle_mod.OracleMesh(m.nodes, m.triangles)
    interior = np.array([k for k in range(om.nn)
                         if 0 < m.nodes[k, 0] < 1 and 0 < m.nodes[k, 1] < 1])
    rng = np.random.default_rng(1)
    x0, x1 = [], []
    for _ in range(400):
        v = m.nodes[rng.choice(interior)]
        s = rng.uniform(0.1, 0.9, 2)
        x0.append(s)
        x1.append(s + (v - s) * rng.choice([1.0, 1.5, 2.0]))   # ends on, or passes through, the vertex
    for e in rng.integers(0, om.ne, 200):                        # along an interior edge
        a, b = m.nodes[om.edge[e]]
        x0.append(a + 0.25 * (b - a))
        x1.append(a + 0.75 * (b - a))
    x0 = np.array(x0)
    x1 = np.clip(np.array(x1), 0.0, 1.0)
    sim, cell0, (cnt, rec), xend = _free_flight(oracle_mod, m, x0, x1)
    om = sim.mesh
    lam = om.lambdas(sim.species[0]["cell"], xend[:, 0], xend[:, 1])
    assert lam.min() > -1e-13
    assert sim.status == 0
    for p in range(len(x0)):
        cells = _cells_from_record(om, cell0[p], cnt[p], rec[p])
        for a, b in zip(cells[:-1], cells[1:]):
            assert b in om.tri_nb[a]


def test_deposit_equals_whitney_line_integral(oracle_mod):
    """i_e = (Q/dt) int_path W1_e . dl (Eq. I.assign), checked against Gauss-Legendre quadrature
    of W1_e = l_a grad l_b - l_b grad l_a on each brute-force piece of the path."""
    m = inputs.jittered_delaunay(5, 5, 1.0, 1.0, 0.3, seed=23)
    rng = np.random.default_rng(2)
    x0 = rng.uniform(0.05, 0.95, (1, 2))
    x1 = np.clip(x0 + np.array([[0.45, -0.3]]), 0.02, 0.98)
    dt = 1e-7
    sim, cell0, _, xend = _free_flight(oracle_mod, m, x0, x1, dt=dt)
    om = sim.mesh
    gl_x, gl_w = np.polynomial.legendre.leggauss(1000)
    ref = np.zeros(om.ne)
    p0, p1 = x0[0], xend[0]
    for lo, hi, f in brute_force_cells(m.nodes, om.tri, p0, p1, eps=0):
        t = lo + (hi - lo) * (gl_x + 1) / 2
        pts = p0[None] + t[:, None] * (p1 - p0)[None]
        lam = _bary(m.nodes, om.tri[f], pts)
        T = np.stack([m.nodes[om.tri[f], 0], m.nodes[om.tri[f], 1], np.ones(3)])
        G = np.linalg.inv(T)[:, :2]        # rows: grad lambda_k
        dl = (p1 - p0) * (hi - lo) / 2
        for mm in range(3):
            a, b = (mm + 1) % 3, (mm + 2) % 3
            W = lam[:, a:a + 1] * G[b][None] - lam[:, b:b + 1] * G[a][None]
            val = (gl_w * (W @ dl)).sum()
            e = om.tri_edge[f, mm]
            ref[e] += om.tri_sign[f, mm] * (QE / dt) * val
    np.testing.assert_allclose(sim.i, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    assert np.abs(ref).max() > 0


def _plasma_sim(oracle_mod, pusher="vay", nside=6, ppc=6, seed=31, spai_level=1, exact=False):
    w = inputs.pair_plasma(nside, ppc, kT=0.3, wc_over_wp=0.5, seed=seed, pusher=pusher)
    m = w.mesh
    sim = oracle_mod.OracleSim(m.nodes, m.triangles, w.dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                               spai_level=spai_level, exact_inverse=exact, b0=w.b0)
    # break the pairing a little so the net charge density is nonzero
    for k, s in enumerate(w.species):
        x = s.x.copy()
        if k == 1:
            x = np.clip(x + rng_shift(len(x), seed, m.lx), 1e-9, m.lx * (1 - 1e-9))
            sim.load(s.q, s.m, x, s.u, None)
        else:
            sim.load(s.q, s.m, x, s.u, s.hint)
    return sim


def rng_shift(n, seed, L):
    return np.random.default_rng(seed).normal(0, 0.3 * L / 6, (n, 2))


def test_discrete_continuity_round_off(oracle_mod):
    """DCE (Eq. full.dis.cont): q^{n+1} - q^n + dt S~ i^{n+1/2} = 0 per node, normalised by the
    sum of the absolute contributions, at round-off every step (crossings and wall reflections)."""
    sim = _plasma_sim(oracle_mod)
    S = sim.mesh.div_dual()
    q0 = sim.charge()
    crossings = 0
    for n in range(40):
        recs = sim.step("vay", record=8)
        crossings += sum(int(c.sum()) for c, _ in recs)
        q1 = sim.charge()
        res = (q1 - q0) + sim.dt * (S @ sim.i)
        scale = abs(S) @ sim.i_abs * sim.dt + 1e-300
        touched = scale > 0
        nr = np.abs(res[touched]) / scale[touched]
        assert nr.max() < 1e-12, (n, nr.max())
        q0 = q1
    assert crossings > 50


def test_discrete_gauss_law_d_form(oracle_mod):
    """DGL (Eq. semi.dis.div.2) in the dual-flux form S~ d^n - q^n = S~ d^0 - q^0 at round-off,
    and S~[*eps]e^n = q^n to round-off when the exact inverse replaces the SPAI."""
    for exact in (False, True):
        sim = _plasma_sim(oracle_mod, exact=exact, seed=32)
        S = sim.mesh.div_dual()
        g0 = S @ sim.d - sim.charge()
        qscale = np.abs(sim.charge()).max()
        for _ in range(30):
            sim.step("hc")
        q = sim.charge()
        g = S @ sim.d - q
        dscale = np.abs(S) @ np.abs(sim.d)
        assert np.abs(g - g0).max() < 1e-12 * max(dscale.max(), qscale)
        if exact:
            # the primal form holds on interior nodes (all incident edges free; PEC edges keep e = 0)
            om = sim.mesh
            bnodes = np.unique(om.edge[om.edge_bnd == 1])
            inner = np.setdiff1d(np.arange(om.nn), bnodes)
            s = S @ (sim.star_eps @ sim.e) - q
            assert np.abs((s - g0)[inner]).max() < 1e-11 * max(dscale.max(), qscale)


def test_empty_cavity_uniform_b_is_static(oracle_mod):
    """A uniform B_z in a PEC cavity is a static solution: C^T [*mu^-1] b cancels on every interior
    edge, so e stays at round-off."""
    m = inputs.jittered_delaunay(8, 8, 1.0, 1.0, 0.3, seed=41)
    B0 = 1.0
    sim = oracle_mod.OracleSim(m.nodes, m.triangles, 1e-11, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                               spai_level=2, b0=B0)
    for _ in range(200):
        sim.step()
    e_scale = B0 * C * (1.0 / 8)           # |E| ~ c B times an edge length
    assert np.abs(sim.e).max() < 1e-12 * e_scale
    np.testing.assert_allclose(sim.b, B0 * 0.5 * sim.mesh.d2A, rtol=1e-12)


def test_cavity_mode_energy_bounded(oracle_mod):
    """Leapfrog with the level-2 SPAI at Courant 0.2 is stable: a random initial field keeps a
    bounded discrete energy over 10^4 steps."""
    m = inputs.jittered_delaunay(8, 8, 1.0, 1.0, 0.3, seed=42)
    om = oracle_mod.OracleMesh(m.nodes, m.triangles)
    el = np.linalg.norm(m.nodes[om.edge[:, 1]] - m.nodes[om.edge[:, 0]], axis=1)
    dt = 0.2 * el.min() / C
    sim = oracle_mod.OracleSim(m.nodes, m.triangles, dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                               spai_level=2)
    rng = np.random.default_rng(3)
    sim.b = rng.normal(0, 1e-3, sim.mesh.nf) * 0.5 * sim.mesh.d2A
    sim.b -= sim.b.mean()
    e0 = None
    hist = []
    for n in range(10_000):
        sim.step()
        if n % 50 == 0:
            hist.append(sim.field_energy())
    hist = np.array(hist)
    assert np.isfinite(hist).all()
    assert hist.max() < 3.0 * hist[1:].mean()
    assert hist[-10:].mean() < 2.0 * hist[1:11].mean()
