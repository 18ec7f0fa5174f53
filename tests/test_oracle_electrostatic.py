"""Pins of the oracle's initial electrostatic solve (CPU only): G^T [*eps] G phi = q with phi = 0 on
the PEC walls and e = -G phi, so that the discrete Gauss law (Eq. (semi.dis.div.2)) holds from the
first step rather than relative to it."""
import numpy as np

from paper_1707_04333_gb300 import inputs

C = inputs.C_LIGHT
QE, ME = inputs.Q_E, inputs.M_E


def test_parallel_plates_closed_form(oracle_mod):
    """Structured right-triangle strip, periodic top and bottom, grounded (PEC) plates at x = 0 and
    x = L, charge Q on every node between them.  Linear elements on right triangles give the
    five-point stencil eps0 [(hy/hx)(2 phi_i - phi_{i-1} - phi_{i+1}) + ...] (the diagonals carry
    no weight), and phi depends on x only, so the exact discrete solution is the quadratic
    phi_i = Q hx / (2 eps0 hy) i (N - i), whichever diagonals the triangulation picked."""
    nx, ny, L, H = 12, 5, 1.2, 0.5
    hx, hy = L / nx, H / ny
    m = inputs.jittered_delaunay(nx, ny, L, H, 0.0, seed=1, periodic_y=True)
    ii, jj = np.meshgrid(np.arange(1, nx), np.arange(ny), indexing="ij")
    node = (ii * (ny + 1) + jj).ravel()
    x = m.nodes[node]
    cell = np.array([np.nonzero((m.triangles == n).any(axis=1))[0][0] for n in node], np.int32)
    Q = 1e-12
    sim = oracle_mod.OracleSim(m.nodes, m.triangles, 1e-12, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                               spai_level=1, periodic=m.periodic)
    sim.load(Q, ME, x, np.zeros_like(x), cell=cell)
    phi = sim.electrostatic_solve()
    iall = np.arange(m.nodes.shape[0]) // (ny + 1)
    want = Q * hx / (2 * inputs.EPS0 * hy) * iall * (nx - iall)
    rep = sim.mesh.rep
    own = rep == np.arange(len(rep))                      # image nodes carry no unknown
    np.testing.assert_allclose(phi[own], want[own], rtol=1e-11, atol=1e-12 * want.max())
    # e on every edge is minus the potential difference along it
    v = sim.mesh.edge_vectors()
    horiz = np.abs(v[:, 1]) < 1e-12 * hy
    assert np.abs(sim.e[~horiz & (np.abs(v[:, 0]) < 1e-12 * hx)]).max() < 1e-12 * np.abs(sim.e).max()


def test_gauss_law_holds_and_field_is_curl_free(oracle_mod):
    """Jittered mesh, non-neutral plasma: after the solve S~ [*eps] e = q on every node off the PEC
    walls (to the sparse solver's round-off), C e = 0 (no magnetic field is generated), and e = 0
    on the PEC edges."""
    w = inputs.pair_plasma(10, 4, kT=0.2, wc_over_wp=0.5, seed=41, pusher="vay")
    m = w.mesh
    sim = oracle_mod.OracleSim(m.nodes, m.triangles, w.dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                               spai_level=1, b0=w.b0)
    rng = np.random.default_rng(41)
    sim.load(w.species[0].q, w.species[0].m, w.species[0].x, w.species[0].u, w.species[0].hint)
    xp = np.clip(w.species[1].x + rng.normal(0, 0.1 * m.lx, w.species[1].x.shape), 1e-9, m.lx * (1 - 1e-9))
    sim.load(w.species[1].q, w.species[1].m, xp, w.species[1].u)
    sim.electrostatic_solve()
    om = sim.mesh
    S = om.div_dual()
    q = sim.charge()
    g = S @ (sim.star_eps @ sim.e) - q
    pec_nodes = np.unique(om.edge[om.edge_bnd == 1])
    inner = np.setdiff1d(np.arange(om.nn), pec_nodes)
    scale = (np.abs(S) @ np.abs(sim.star_eps @ sim.e))[inner] + np.abs(q[inner])
    assert (np.abs(g[inner]) <= 1e-12 * scale.max()).all()
    assert np.abs(q[inner]).max() > 1e3 * np.abs(g[inner]).max()   # the field does carry the charge
    ce = om.curl() @ sim.e
    assert np.abs(ce).max() <= 1e-13 * np.abs(sim.e).max() * 3
    assert np.all(sim.e[om.edge_bnd == 1] == 0.0)
    np.testing.assert_allclose(sim.d, sim.star_eps @ sim.e)
