"""Periodic walls on the GPU (the paper's Bernstein strip is periodic top and bottom, Sec. III.C)
against the oracle: the same identified edges and SPAI, bit-identical FP64 steps through the
wall, FP32 within its round-off, and continuity / Gauss residuals at round-off."""
import numpy as np
import pytest

from paper_1707_04333_gb300 import inputs

pytestmark = pytest.mark.gpu

C = inputs.C_LIGHT
QE, ME = inputs.Q_E, inputs.M_E


@pytest.fixture(scope="module")
def fx():
    import torch
    assert torch.cuda.is_available()
    from paper_1707_04333_gb300 import build_lib, fetdpic
    build_lib.build()
    from oracle import oracle
    oracle.build()
    return fetdpic, oracle


def strip_state(seed, nx=20, ny=16, n_e=3077, n_p=1001, dt=3e-10, fast=40, e0=(0.0, 0.0)):
    """Periodic strip 1 x 0.8 m (top and bottom joined), random fields, two species with momenta
    up to gamma ~ 3 (1-2 cells per step), a few gamma = 50 particles crossing many cells and the
    periodic wall several times; PEC left and right."""
    rng = np.random.default_rng(seed)
    m = inputs.jittered_delaunay(nx, ny, 1.0, 0.8, 0.3, seed=seed, periodic_y=True)
    sp = []
    for k, (q, n) in enumerate(((-QE, n_e), (QE, n_p))):
        tri = rng.integers(0, len(m.triangles), n).astype(np.int32)
        x = inputs.sample_in_triangles(m, tri, rng)
        g = 1 + rng.exponential(0.8, n)
        if k == 0:
            g[:fast] = 50.0
        mag = C * np.sqrt(g * g - 1)
        th = rng.uniform(0, 2 * np.pi, n)
        sp.append(inputs.Species(q, ME, x, np.stack([mag * np.cos(th), mag * np.sin(th)], 1), tri))
    return inputs.Workload("strip", m, sp, dt, b0=0.0, e0=e0), rng


def make_pair(fetdpic, oracle, w, precision="fp64", spai_level=1, record=16, sort_interval=-1,
              fields=(None, None), check_interval=0):
    sim = fetdpic.Simulation(w, precision=precision, spai_level=spai_level, record_walk=record,
                             sort_interval=sort_interval, check_interval=check_interval).load()
    ora = oracle.OracleSim(w.mesh.nodes, w.mesh.triangles, w.dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                           spai_level=spai_level, b0=w.b0, e0=w.e0, ext=w.ext, periodic=w.mesh.periodic)
    for s in w.species:
        ora.load(s.q, s.m, s.x, s.u, s.hint)
    e, b = fields
    if e is not None:
        fetdpic.fetdpic_write_fields(sim.h, 0, e, b)
        ora.e = e.copy()
        ora.b = b.copy()
    return sim, ora


def _periodic_edges(om):
    return set(int(e) for e in om.tri_edge[np.nonzero(om.tri_shift)])


def test_periodic_numbering_spai_and_uniform_field(fx):
    """Identified edges numbered as the oracle numbers them, the same SPAI, and a uniform initial E
    projected on the edges the same way (edge vectors read off the triangles, not the stored
    nodes, which a period may separate)."""
    fetdpic, oracle = fx
    w, _ = strip_state(1, e0=(3.0e3, -1.5e3))
    sim, ora = make_pair(fetdpic, oracle, w, spai_level=2)
    om = ora.mesh
    assert np.array_equal(fetdpic.fetdpic_read_edges(sim.h), om.edge)
    assert int(om.edge_bnd.sum()) == 2 * 16                  # only the left and right walls are PEC
    rp, re_, ci, v = fetdpic.fetdpic_read_spai(sim.h)
    import scipy.sparse as sp
    Mg = sp.csr_matrix((v, ci, rp), shape=(len(re_), om.ne))[:, om.free]
    assert np.array_equal(re_, om.free)
    assert abs(Mg - ora.Minv).max() <= 1e-11 * abs(ora.Minv).max()
    np.testing.assert_allclose(sim.read_fields()["e"], ora.e, rtol=0, atol=1e-12 * np.abs(ora.e).max())
    sim.close()


@pytest.mark.parametrize("pusher", ["boris", "boris_tan", "vay", "hc"])
def test_periodic_fp64_single_step_bit_exact(fx, pusher):
    """One FP64 step from random fields: triangles, crossed-edge lists (periodic crossings
    included), positions and momenta bit-identical to the oracle (Boris-tan within 1e-12)."""
    fetdpic, oracle = fx
    w, rng = strip_state(2)
    om = oracle.OracleMesh(w.mesh.nodes, w.mesh.triangles, w.mesh.periodic)
    e = rng.normal(0, 5e4, om.ne) * (om.edge_bnd == 0)
    b = rng.uniform(-0.01, 0.01, om.nf) * 0.5 * om.d2A
    sim, ora = make_pair(fetdpic, oracle, w, fields=(e, b))
    fetdpic.fetdpic_step(sim.h, 1, pusher)
    fetdpic.fetdpic_sync(sim.h)
    recs = ora.step(pusher, record=16)
    assert ora.status == 0
    pe = _periodic_edges(ora.mesh)
    through = 0
    for k, s in enumerate(ora.species):
        g = sim.read_species(k)
        assert np.array_equal(g["cell"], s["cell"])
        if pusher == "boris_tan":
            np.testing.assert_allclose(g["x"][:, 1], s["y"], rtol=0, atol=1e-13)
            continue
        assert np.array_equal(g["x"][:, 0], s["x"]) and np.array_equal(g["x"][:, 1], s["y"])
        assert np.array_equal(g["u"][:, 0], s["ux"]) and np.array_equal(g["u"][:, 1], s["uy"])
        cnt, rec = fetdpic.fetdpic_read_walk(sim.h, k, len(s["x"]), 16)
        assert np.array_equal(cnt, recs[k][0])
        mask = np.arange(16)[None, :] < cnt[:, None]
        assert np.array_equal(np.where(mask, rec, 0), np.where(mask, recs[k][1], 0))
        through += sum(int(x) in pe for x in rec[mask])
    if pusher != "boris_tan":
        assert through > 50
    assert ((ora.species[0]["y"] >= 0) & (ora.species[0]["y"] <= w.mesh.ly)).all()
    f = sim.read_fields()
    assert np.abs(f["j"] - ora.i).max() <= 1e-10 * np.abs(ora.i_abs).max()
    np.testing.assert_allclose(f["e"], ora.e, rtol=0, atol=1e-10 * np.abs(ora.e).max())
    sim.close()


def test_periodic_fp64_multi_step_strip(fx):
    """20 coupled Vay steps of a pair plasma on a periodic strip (sorted every 5 steps): fields
    within 1e-10 of the oracle, every particle in the same triangle, positions within 1e-10."""
    fetdpic, oracle = fx
    w = inputs.pair_plasma(16, 6, kT=0.3, wc_over_wp=0.5, seed=17, pusher="vay", ny=6, periodic_y=True)
    sim, ora = make_pair(fetdpic, oracle, w, spai_level=2, record=0, sort_interval=5)
    fetdpic.fetdpic_step(sim.h, 20, "vay")
    fetdpic.fetdpic_sync(sim.h)
    for _ in range(20):
        ora.step("vay")
    f = sim.read_fields()
    for name, ref in (("e", ora.e), ("b", ora.b), ("j", ora.i)):
        assert np.abs(f[name] - ref).max() <= 1e-10 * max(np.abs(ref).max(), 1e-300), name
    for k, s in enumerate(ora.species):
        g = sim.read_species(k)
        assert np.array_equal(g["cell"], s["cell"])
        np.testing.assert_allclose(g["x"][:, 1], s["y"], rtol=0, atol=1e-10 * w.mesh.ly)
    sim.close()


def test_periodic_fp32_single_step_tolerance(fx):
    """FP32 path vs the FP64 oracle after one step on the periodic strip, with the FP32 bounds of the
    non-periodic case (momenta 2e-5 relative, positions 1e-5 of the cell size, distance taken
    modulo the period for points that end on the wall)."""
    fetdpic, oracle = fx
    w, rng = strip_state(3, fast=0)
    om = oracle.OracleMesh(w.mesh.nodes, w.mesh.triangles, w.mesh.periodic)
    e = rng.normal(0, 5e4, om.ne) * (om.edge_bnd == 0)
    b = rng.uniform(-0.01, 0.01, om.nf) * 0.5 * om.d2A
    sim, ora = make_pair(fetdpic, oracle, w, precision="fp32", fields=(e, b), record=0)
    fetdpic.fetdpic_step(sim.h, 1, "hc")
    fetdpic.fetdpic_sync(sim.h)
    ora.step("hc")
    h = 1.0 / 20
    for k, s in enumerate(ora.species):
        g = sim.read_species(k)
        umag = np.hypot(s["ux"], s["uy"])
        du = np.hypot(g["u"][:, 0] - s["ux"], g["u"][:, 1] - s["uy"])
        assert (du <= 2e-5 * umag + 1e-3).all(), du.max()
        dy = np.abs(g["x"][:, 1] - s["y"])
        dy = np.minimum(dy, w.mesh.ly - dy)
        dx = np.hypot(g["x"][:, 0] - s["x"], dy)
        assert (dx <= 1e-5 * h).all(), dx.max()
        assert (g["cell"] == s["cell"]).mean() > 0.999
    f = sim.read_fields()
    assert np.abs(f["j"] - ora.i).max() <= 1e-4 * np.abs(ora.i_abs).max()
    sim.close()


@pytest.mark.parametrize("precision,tol_dce,tol_dgl", [("fp64", 1e-12, 1e-12), ("fp32", 2e-5, 1e-4)])
def test_periodic_continuity_and_gauss_every_step(fx, precision, tol_dce, tol_dgl):
    fetdpic, _ = fx
    w = inputs.pair_plasma(16, 6, kT=0.3, wc_over_wp=0.5, seed=19, pusher="vay", ny=6, periodic_y=True)
    rng = np.random.default_rng(19)
    p = w.species[1]
    x = p.x.copy()
    x[:, 1] = np.mod(x[:, 1] + rng.normal(0, 0.3 * w.mesh.ly, len(x)), w.mesh.ly)
    w.species[1] = inputs.Species(p.q, p.m, x, p.u, np.full(len(x), -1, np.int32))
    sim = fetdpic.Simulation(w, precision=precision, spai_level=2, sort_interval=4, check_interval=1).load()
    for _ in range(25):
        sim.step(1, "vay").sync()
        c = fetdpic.fetdpic_check(sim.h, 0)
        assert c["dce"] < tol_dce, c
        assert c["dgl"] < tol_dgl, c
    sim.close()
