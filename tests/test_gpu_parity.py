"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

FP64 mode: one step from the same state gives bit-identical triangles,
crossed-edge lists, positions and momenta (Boris-tan within 1e-12: tan is not
correctly rounded); current and fields within 1e-10 of the oracle relative to
their scale (the GPU sums the current exactly in 64-bit fixed point, the
oracle in FP64 particle order, and the two SPAI solvers differ at round-off).
FP32 mode: tolerances derived from FP32 round-off (documented per test).
"""
import math

import numpy as np
import pytest

from paper_1707_04333_gb300 import inputs

pytestmark = pytest.mark.gpu

C = inputs.C_LIGHT
QE, ME = inputs.Q_E, inputs.M_E
PUSHERS = ["boris", "boris_tan", "vay", "hc"]


@pytest.fixture(scope="module")
def fx():
    import torch
    assert torch.cuda.is_available()
    from paper_1707_04333_gb300 import build_lib, fetdpic
    build_lib.build()
    from oracle import oracle
    oracle.build()
    return fetdpic, oracle


def random_state(seed, nx=20, ny=16, n_e=3077, n_p=1001, dt=3e-10, fast=40):
    """Jittered-Delaunay mesh on 1 x 0.8 m, random fields, two species with momenta up to
    gamma ~ 3 (1-2 cells per step), a few gamma = 50 particles crossing many cells, walls hit."""
    rng = np.random.default_rng(seed)
    m = inputs.jittered_delaunay(nx, ny, 1.0, 0.8, 0.3, seed=seed)
    sp = []
    for k, (q, n) in enumerate(((-QE, n_e), (QE, n_p))):
        tri = rng.integers(0, len(m.triangles), n).astype(np.int32)
        x = inputs.sample_in_triangles(m, tri, rng)
        g = 1 + rng.exponential(0.8, n)
        if k == 0:
            g[:fast] = 50.0
        mag = C * np.sqrt(g * g - 1)
        th = rng.uniform(0, 2 * np.pi, n)
        u = np.stack([mag * np.cos(th), mag * np.sin(th)], 1)
        sp.append(inputs.Species(q, ME, x, u, tri))
    w = inputs.Workload("random", m, sp, dt, b0=0.0)
    return w, rng


def random_fields(om, rng, scale_e=5e4, scale_b=0.01):
    e = rng.normal(0, scale_e, om.ne) * (om.edge_bnd == 0)
    b = rng.uniform(-scale_b, scale_b, om.nf) * 0.5 * om.d2A
    return e, b


def make_pair(fetdpic, oracle, w, precision="fp64", spai_level=1, record=16, sort_interval=-1,
              fields=(None, None), max_cross=64, exact=False):
    sim = fetdpic.Simulation(w, precision=precision, spai_level=-1 if exact else spai_level,
                             record_walk=record, sort_interval=sort_interval, max_crossings=max_cross)
    sim.load()
    ora = oracle.OracleSim(w.mesh.nodes, w.mesh.triangles, w.dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                           spai_level=spai_level, exact_inverse=exact, b0=w.b0, e0=w.e0, ext=w.ext,
                           max_cross=max_cross)
    for s in w.species:
        ora.load(s.q, s.m, s.x, s.u, s.hint)
    e, b = fields
    if e is not None:
        fetdpic.fetdpic_write_fields(sim.h, 0, e, b)
        ora.e = e.copy()
        ora.b = b.copy()
    return sim, ora


def test_mesh_numbering_and_spai_match_oracle(fx):
    fetdpic, oracle = fx
    w, _ = random_state(1)
    sim, ora = make_pair(fetdpic, oracle, w, spai_level=2)
    assert np.array_equal(fetdpic.fetdpic_read_edges(sim.h), ora.mesh.edge)
    rp, re_, ci, v = fetdpic.fetdpic_read_spai(sim.h)
    import scipy.sparse as sp
    ne = ora.mesh.ne
    Mg = sp.csr_matrix((v, ci, rp), shape=(len(re_), ne))[:, ora.mesh.free]
    Mo = ora.Minv
    assert np.array_equal(re_, ora.mesh.free)
    d = abs(Mg - Mo).max()
    assert d <= 1e-11 * abs(Mo).max(), d
    sim.close()


@pytest.mark.parametrize("pusher", PUSHERS)
def test_fp64_single_step_bit_exact(fx, pusher):
    fetdpic, oracle = fx
    w, rng = random_state(2)
    om = oracle.OracleMesh(w.mesh.nodes, w.mesh.triangles)
    e, b = random_fields(om, rng)
    sim, ora = make_pair(fetdpic, oracle, w, fields=(e, b))
    fetdpic.fetdpic_step(sim.h, 1, pusher)
    fetdpic.fetdpic_sync(sim.h)
    recs = ora.step(pusher, record=16)
    assert ora.status == 0
    crossings = 0
    for k, s in enumerate(ora.species):
        g = sim.read_species(k)
        assert np.array_equal(g["cell"], s["cell"])
        if pusher == "boris_tan":
            np.testing.assert_allclose(g["u"][:, 0], s["ux"], rtol=1e-12, atol=1e-12 * np.abs(s["ux"]).max())
            np.testing.assert_allclose(g["x"][:, 0], s["x"], rtol=0, atol=1e-13)
        else:
            assert np.array_equal(g["x"][:, 0], s["x"]) and np.array_equal(g["x"][:, 1], s["y"])
            assert np.array_equal(g["u"][:, 0], s["ux"]) and np.array_equal(g["u"][:, 1], s["uy"])
            cnt, rec = fetdpic.fetdpic_read_walk(sim.h, k, len(s["x"]), 16)
            assert np.array_equal(cnt, recs[k][0])
            mask = np.arange(16)[None, :] < cnt[:, None]
            assert np.array_equal(np.where(mask, rec, 0), np.where(mask, recs[k][1], 0))
            crossings += int(cnt.sum())
            assert (rec[mask] < 0).any() or k == 1          # some wall reflections among electrons
    if pusher != "boris_tan":
        assert crossings > 1000
    f = sim.read_fields()
    tol = 1e-10 * np.abs(ora.i_abs).max()
    assert np.abs(f["j"] - ora.i).max() <= tol
    np.testing.assert_allclose(f["b"], ora.b, rtol=1e-13, atol=1e-13 * np.abs(ora.b).max())
    np.testing.assert_allclose(f["e"], ora.e, rtol=0, atol=1e-10 * np.abs(ora.e).max())
    sim.close()


def test_fp64_multi_step_pair_plasma(fx):
    """20 coupled steps (Vay, particles sorted every 5 steps): fields within 1e-10 of the oracle,
    every particle in the same triangle, positions and momenta within 1e-10 relative."""
    fetdpic, oracle = fx
    w = inputs.pair_plasma(14, 6, kT=0.3, wc_over_wp=0.5, seed=7, pusher="vay")
    sim, ora = make_pair(fetdpic, oracle, w, spai_level=2, record=0, sort_interval=5)
    fetdpic.fetdpic_step(sim.h, 20, "vay")
    fetdpic.fetdpic_sync(sim.h)
    for _ in range(20):
        ora.step("vay")
    f = sim.read_fields()
    for name, ref in (("e", ora.e), ("b", ora.b), ("j", ora.i)):
        sc = max(np.abs(ref).max(), 1e-300)
        assert np.abs(f[name] - ref).max() <= 1e-10 * sc, name
    for k, s in enumerate(ora.species):
        g = sim.read_species(k)
        assert np.array_equal(g["cell"], s["cell"])
        np.testing.assert_allclose(g["x"][:, 0], s["x"], rtol=1e-10, atol=1e-10 * w.mesh.lx)
        np.testing.assert_allclose(g["u"][:, 1], s["uy"], rtol=1e-10, atol=1e-10 * np.abs(s["uy"]).max())
    sim.close()


def test_fp64_exact_inverse_mode(fx):
    """spai_level = -1 (dense exact inverse) matches the oracle's exact-inverse mode."""
    fetdpic, oracle = fx
    w = inputs.pair_plasma(6, 4, kT=0.3, seed=8, pusher="hc")
    sim, ora = make_pair(fetdpic, oracle, w, record=0, exact=True)
    fetdpic.fetdpic_step(sim.h, 10, "hc")
    fetdpic.fetdpic_sync(sim.h)
    for _ in range(10):
        ora.step("hc")
    f = sim.read_fields()
    assert np.abs(f["e"] - ora.e).max() <= 1e-10 * np.abs(ora.e).max()
    sim.close()


def test_batched_equals_separate(fx):
    """Two instances packed in one context give bit-identical results to each alone (FP64):
    instances share only the launches, and the integer deposit is order-free."""
    fetdpic, oracle = fx
    w1 = inputs.pair_plasma(10, 5, kT=0.2, seed=11, pusher="boris")
    w2 = inputs.pair_plasma(7, 9, kT=0.05, wc_over_wp=1.0, seed=12, pusher="boris")
    both = fetdpic.Simulation([w1, w2], precision="fp64", spai_level=1, sort_interval=3).load()
    both.step(7, "boris").sync()
    for k, w in enumerate((w1, w2)):
        one = fetdpic.Simulation(w, precision="fp64", spai_level=1, sort_interval=3).load()
        one.step(7, "boris").sync()
        fa, fb = both.read_fields(k), one.read_fields(0)
        for name in ("e", "b", "j"):
            assert np.array_equal(fa[name], fb[name]), name
        for s in range(2):
            ga = both.read_species(2 * k + s)
            gb = one.read_species(s)
            for name in ("x", "u", "cell"):
                assert np.array_equal(ga[name], gb[name]), name
        one.close()
    both.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_deterministic_rerun(fx, precision):
    """Two identical runs (with sorts, whose in-triangle order depends on atomics) are bit-identical."""
    fetdpic, _ = fx
    w = inputs.pair_plasma(16, 8, kT=0.1, seed=13, pusher="vay")
    outs = []
    for _ in range(2):
        s = fetdpic.Simulation(w, precision=precision, spai_level=2, sort_interval=4).load()
        s.step(13, "vay").sync()
        outs.append((s.read_fields(), s.read_species(0), s.read_species(1)))
        s.close()
    for a, b in zip(outs[0], outs[1]):
        for k in a:
            assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("precision,variant", [("fp64", 0), ("fp32", 0), ("fp32", 18), ("fp32", 10)])
def test_graph_replay_equals_plain_launches(fx, precision, variant):
    """Steps replayed from captured CUDA graphs (all pushers' graphs, both particle-buffer parities,
    sorting and non-sorting steps, the sort on its side stream beside the Ampere update; for the
    hybrid variant both of its kernels) give bit-identical results to plain launches with stage
    events, where every stage runs in order on one stream."""
    fetdpic, _ = fx
    w = inputs.pair_plasma(12, 5, kT=0.2, seed=17, pusher="boris")
    outs = []
    for graphs in (False, True):
        s = fetdpic.Simulation(w, precision=precision, spai_level=1, sort_interval=5, use_graphs=graphs,
                               time_stages=not graphs, kernel_variant=variant).load()
        s.step(5, "boris").step(4, "vay").step(7, "hc").sync()
        outs.append((s.read_fields(), s.read_species(0), s.read_species(1)))
        s.close()
    for a, b in zip(outs[0], outs[1]):
        for k in a:
            assert np.array_equal(a[k], b[k]), k


def test_fp32_kernel_variants_bit_identical(fx):
    """Every FP32 particle-kernel variant (register prefetch at 2, 3 or 4 resident blocks per SM;
    shared-memory staging by bulk asynchronous copies; two particles per thread; per-block
    deposit windows in shared memory) computes the same per-particle arithmetic and integer
    deposits, so all give bit-identical particles and fields over steps with walks, wall
    reflections, sorts and all three pushers, on enough particles for many chunks per warp."""
    fetdpic, _ = fx
    w = inputs.pair_plasma(48, 24, kT=0.3, seed=23, pusher="vay")
    outs = {}
    for v in (3, 2, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22):
        s = fetdpic.Simulation(w, precision="fp32", spai_level=1, sort_interval=4, kernel_variant=v,
                               check_interval=5).load()
        s.step(5, "vay").step(4, "hc").step(6, "boris").sync()
        c = fetdpic.fetdpic_check(s.h, 0)
        assert c["dce"] < 2e-5, (v, c)
        outs[v] = (s.read_fields(), s.read_species(0), s.read_species(1))
        s.close()
    for v in (2, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22):
        for a, b in zip(outs[3], outs[v]):
            for k in a:
                assert np.array_equal(a[k], b[k]), (v, k)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autotune_leaves_state_unchanged(fx, precision, tmp_path):
    """The autotuner's trials start from and restore the current state: a tuned run equals an
    untuned run configured with the same choice, bit for bit; the cache reproduces the choice."""
    fetdpic, _ = fx
    w = inputs.pair_plasma(16, 6, kT=0.2, seed=19, pusher="vay")
    a = fetdpic.Simulation(w, precision=precision, spai_level=1).load()
    a.step(3, "vay")
    cache = str(tmp_path / "tune.json")
    v, s = a.autotune("vay", trial_steps=16, cache=cache)
    assert v in range(2, 23) and s in (8, 12, 16, 32)
    a.step(20, "vay").sync()
    b = fetdpic.Simulation(w, precision=precision, spai_level=1).load()
    b.step(3, "vay")
    assert b.autotune("vay", cache=cache) == (v, s)        # served from the cache
    b.step(20, "vay").sync()
    for sid in range(2):
        ga, gb = a.read_species(sid), b.read_species(sid)
        for k in ga:
            assert np.array_equal(ga[k], gb[k]), k
    fa, fb = a.read_fields(), b.read_fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    a.close()
    b.close()


def test_fp32_single_step_tolerance(fx):
    """FP32 path vs the FP64 oracle after one step from the same state.  Tolerances from FP32
    round-off (eps = 6e-8) amplified by the gather/push chain: momenta 2e-5 relative, positions
    1e-5 of the cell size, current 1e-4 of its scale; triangles equal except within that
    distance of an edge."""
    fetdpic, oracle = fx
    w, rng = random_state(3, fast=0)
    om = oracle.OracleMesh(w.mesh.nodes, w.mesh.triangles)
    e, b = random_fields(om, rng)
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
        dx = np.hypot(g["x"][:, 0] - s["x"], g["x"][:, 1] - s["y"])
        assert (dx <= 1e-5 * h).all(), dx.max()
        same = g["cell"] == s["cell"]
        if not same.all():
            lam = om.lambdas(s["cell"][~same], s["x"][~same], s["y"][~same])
            assert (lam.min(1) < 1e-5).all()
        assert same.mean() > 0.999
    f = sim.read_fields()
    assert np.abs(f["j"] - ora.i).max() <= 1e-4 * np.abs(ora.i_abs).max()
    sim.close()


def test_fp32_gyrofrequency_error(fx):
    """Precision form of the cyclotron case (gamma = 2, dt = 0.05/omega_c, 2000 steps): the FP32
    gyro-phase of every electron matches the FP64 oracle to < 1e-4 relative frequency error."""
    fetdpic, oracle = fx
    w = inputs.cyclotron(gamma=2.0, n=64, nx=32, seed=1, pusher="boris")
    sim, ora = make_pair(fetdpic, oracle, w, precision="fp32", record=0, sort_interval=16)
    n = 2000
    fetdpic.fetdpic_step(sim.h, n, "boris")
    fetdpic.fetdpic_sync(sim.h)
    s0 = ora.species[0]
    ang0 = np.arctan2(s0["uy"], s0["ux"]).copy()
    unw_o = np.zeros(64)
    prev = ang0.copy()
    for _ in range(n):
        ora.step("boris")
        a = np.arctan2(s0["uy"], s0["ux"])
        unw_o += np.angle(np.exp(1j * (a - prev)))
        prev = a.copy()
    g = sim.read_species(0)
    ag = np.arctan2(g["u"][:, 1], g["u"][:, 0])
    # the final phases agree to the accumulated-angle precision: frequency error = dphase / total
    dphi = np.abs(np.angle(np.exp(1j * (ag - prev))))
    assert (dphi / np.abs(unw_o) < 1e-4).all(), (dphi / np.abs(unw_o)).max()
    np.testing.assert_allclose(np.hypot(g["u"][:, 0], g["u"][:, 1]), np.hypot(s0["ux"], s0["uy"]), rtol=1e-5)
    sim.close()


def test_edge_cases(fx):
    """Empty species, points exactly on an edge and on a vertex, zero steps, walk limit, bad input."""
    fetdpic, oracle = fx
    m = inputs.jittered_delaunay(6, 6, 1.0, 1.0, 0.3, seed=5)
    om = oracle.OracleMesh(m.nodes, m.triangles)
    e_int = np.nonzero(om.edge_bnd == 0)[0][3]
    a, b = m.nodes[om.edge[e_int]]
    inner = [k for k in range(len(m.nodes)) if 0 < m.nodes[k, 0] < 1 and 0 < m.nodes[k, 1] < 1][0]
    x = np.array([(a + b) / 2, m.nodes[inner], [0.5, 0.5]])
    u = np.array([[1e7, 2e7], [-3e7, 1e6], [0.0, 0.0]])
    sp_ = [inputs.Species(-QE, ME, x, u, np.full(3, -1, np.int32)),
           inputs.Species(QE, ME, np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(0, np.int32))]
    w = inputs.Workload("edge", m, sp_, 1e-10, b0=0.3)
    sim, ora = make_pair(fetdpic, oracle, w, record=4)
    fetdpic.fetdpic_step(sim.h, 0, "boris")
    fetdpic.fetdpic_sync(sim.h)
    fetdpic.fetdpic_step(sim.h, 3, "boris")
    fetdpic.fetdpic_sync(sim.h)
    for _ in range(3):
        ora.step("boris", record=4)
    g = sim.read_species(0)
    s = ora.species[0]
    assert np.array_equal(g["cell"], s["cell"]) and np.array_equal(g["x"][:, 0], s["x"])
    assert sim.read_species(1)["x"].shape == (0, 2)
    with pytest.raises(fetdpic.FetdpicError) as ei:
        fetdpic.fetdpic_step(sim.h, 1, 7)
    assert ei.value.code == fetdpic.EINVAL
    sim.close()
    # walk limit: fast particles with max_crossings = 1
    wf, _ = random_state(4, n_e=500, n_p=10, dt=3e-9)
    for prec in ("fp64", "fp32"):
        sim = fetdpic.Simulation(wf, precision=prec, max_crossings=1, sort_interval=-1).load()
        fetdpic.fetdpic_step(sim.h, 1, "boris")
        with pytest.raises(fetdpic.FetdpicError) as ei:
            fetdpic.fetdpic_sync(sim.h)
        assert ei.value.code == fetdpic.EWALK, prec
        sim.close()
    # a triangle outside the mesh given to write_particles: found on the device, the particle dropped,
    # EINVAL at the next sync
    for prec in ("fp64", "fp32"):
        sim = fetdpic.Simulation(w, precision=prec).load()
        g = sim.read_species(0)
        cells = g["cell"].copy()
        cells[1] = len(m.triangles) + 5
        fetdpic.fetdpic_write_particles(sim.h, 0, g["x"], g["u"], cells)
        with pytest.raises(fetdpic.FetdpicError) as ei:
            fetdpic.fetdpic_sync(sim.h)
        assert ei.value.code == fetdpic.EINVAL and "outside the mesh" in str(ei.value)
        sim.close()
    # an overflowing field makes the momenta non-finite: reported as ENONFINITE at the next sync
    # (with NaN positions the walk finds no exit edge, so every triangle index stays valid)
    for prec in ("fp64", "fp32"):
        sim = fetdpic.Simulation(w, precision=prec).load()
        ne = sim.read_fields()["e"].shape[0]
        fetdpic.fetdpic_write_fields(sim.h, 0, e=np.full(ne, 1e300))
        fetdpic.fetdpic_step(sim.h, 2, "vay")
        with pytest.raises(fetdpic.FetdpicError) as ei:
            fetdpic.fetdpic_sync(sim.h)
        assert ei.value.code == fetdpic.ENONFINITE, (prec, ei.value)
        sim.close()
    # a point outside the mesh is rejected at load
    bad = fetdpic.Simulation(inputs.Workload("o", m, [], 1e-10), precision="fp64")
    with pytest.raises(fetdpic.FetdpicError) as ei:
        fetdpic.fetdpic_load_particles(bad.h, 0, -QE, ME, np.array([[2.0, 0.5]]), np.zeros((1, 2)))
    assert ei.value.code == fetdpic.EOUTSIDE
    bad.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_pair_plasma_sampled(fx, precision):
    """The benchmark workload (200k triangles, 8M particles, Vay) in the launch configuration the
    benchmark times: one step on the GPU; a seeded sample of 4096 particles per species is stepped
    by the oracle from the same pre-step state and fields (FP64: bit-identical triangles, positions
    and momenta; FP32: momenta within 2e-5, positions within 1e-5 of the mean edge)."""
    fetdpic, oracle = fx
    w = inputs.pair_plasma(317, 20, kT=0.1, wc_over_wp=0.5, seed=2, pusher="vay")
    sim = fetdpic.Simulation(w, precision=precision, spai_level=2, sort_interval=16).load()
    sim.step(3, "vay").sync()                       # leave the initial state
    pre = [sim.read_species(k) for k in range(2)]
    f0 = sim.read_fields()
    sim.step(1, "vay").sync()
    post = [sim.read_species(k) for k in range(2)]
    ora = oracle.OracleSim(w.mesh.nodes, w.mesh.triangles, w.dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                           b0=w.b0, fields=False)
    ora.e = f0["e"].copy()
    ora.b = f0["b"].copy()
    rng = np.random.default_rng(99)
    idxs = []
    for k, s in enumerate(w.species):
        idx = np.sort(rng.choice(len(s.x), 4096, replace=False))
        idxs.append(idx)
        ora.load(s.q, s.m, pre[k]["x"][idx], pre[k]["u"][idx], cell=pre[k]["cell"][idx])
    ora.step("vay", only_particles=True)            # one Faraday update, both species
    om = ora.mesh
    h = float(np.linalg.norm(w.mesh.nodes[om.edge[:, 1]] - w.mesh.nodes[om.edge[:, 0]], axis=1).mean())
    for k, idx in enumerate(idxs):
        o = ora.species[k]
        if precision == "fp64":
            assert np.array_equal(o["cell"], post[k]["cell"][idx])
            assert np.array_equal(o["x"], post[k]["x"][idx, 0]) and np.array_equal(o["uy"], post[k]["u"][idx, 1])
        else:
            du = np.hypot(o["ux"] - post[k]["u"][idx, 0], o["uy"] - post[k]["u"][idx, 1])
            assert (du <= 2e-5 * np.hypot(o["ux"], o["uy"]) + 1e-3).all()
            assert (o["cell"] == post[k]["cell"][idx]).mean() > 0.999
            # positions within 1e-5 of the mean edge length (FP32 barycentric storage)
            dx = np.hypot(o["x"] - post[k]["x"][idx, 0], o["y"] - post[k]["x"][idx, 1])
            assert (dx <= 1e-5 * h).all(), dx.max() / h
    sim.close()
