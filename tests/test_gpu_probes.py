"""Field probes on the GPU against the oracle's field at the same points, and the Bernstein-mode
band frequencies of the FP32 path against the FP64 path (Sec. III.C)."""
import math

import numpy as np
import pytest

from paper_1707_04333_gb300 import bernstein, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fx():
    import torch
    assert torch.cuda.is_available()
    from paper_1707_04333_gb300 import build_lib, fetdpic
    build_lib.build()
    from oracle import oracle
    oracle.build()
    return fetdpic, oracle


def _workload(seed=51):
    return inputs.pair_plasma(14, 6, kT=0.3, wc_over_wp=0.5, seed=seed, pusher="vay")


def _points(w, n, seed):
    rng = np.random.default_rng(seed)
    return inputs.sample_in_triangles(w.mesh, rng.integers(0, len(w.mesh.triangles), n), rng)


def _oracle(oracle, w):
    ora = oracle.OracleSim(w.mesh.nodes, w.mesh.triangles, w.dt, eps0=inputs.EPS0, mu0=inputs.MU0,
                           c=inputs.C_LIGHT, spai_level=2, b0=w.b0)
    for s in w.species:
        ora.load(s.q, s.m, s.x, s.u, s.hint)
    return ora


def test_probes_match_oracle_field_and_ring_wraps(fx):
    """FP64: each recorded row equals the oracle's Whitney-interpolated e^{n+1} at the probe points
    (fields agree to 1e-10 of their scale); a ring of 5 rows keeps the last 5 of 12 steps."""
    fetdpic, oracle = fx
    w = _workload()
    pts = _points(w, 60, 1)
    sim = fetdpic.Simulation(w, precision="fp64", spai_level=2, sort_interval=4).load()
    sim.set_probes(pts, capacity=5)
    ora = _oracle(oracle, w)
    want = []
    for _ in range(12):
        sim.step(1, "vay")
        ora.step("vay")
        want.append(ora.mesh.field_at(ora.e, pts[:, 0], pts[:, 1]))
    rows, total = sim.read_probes()
    assert total == 12 and rows.shape == (5, 60, 2)
    scale = np.abs(np.array(want)).max()
    assert scale > 0
    for r, wv in zip(rows, want[-5:]):
        np.testing.assert_allclose(r, wv, rtol=0, atol=1e-10 * scale)
    two, _ = sim.read_probes(max_rows=2)
    assert np.array_equal(two, rows[-2:])
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_probes_in_graph_replay_equal_plain_launches(fx, precision):
    fetdpic, _ = fx
    w = _workload(52)
    pts = _points(w, 33, 2)
    out = []
    for graphs in (False, True):
        s = fetdpic.Simulation(w, precision=precision, spai_level=1, sort_interval=3, use_graphs=graphs).load()
        s.set_probes(pts, capacity=16)
        s.step(7, "boris").step(4, "hc").sync()
        out.append(s.read_probes())
        s.close()
    assert out[0][1] == out[1][1] == 11
    assert np.array_equal(out[0][0], out[1][0])


def test_probes_fp32_close_to_oracle(fx):
    """FP32 path: probe rows within FP32 round-off of the FP64 oracle over 8 steps (1e-3 of the field
    scale: FP32 currents are within 1e-4 of theirs, accumulated over the steps)."""
    fetdpic, oracle = fx
    w = _workload(53)
    pts = _points(w, 40, 3)
    sim = fetdpic.Simulation(w, precision="fp32", spai_level=2, sort_interval=-1).load()
    sim.set_probes(pts, capacity=8)
    ora = _oracle(oracle, w)
    want = []
    for _ in range(8):
        sim.step(1, "vay")
        ora.step("vay")
        want.append(ora.mesh.field_at(ora.e, pts[:, 0], pts[:, 1]))
    rows, _ = sim.read_probes()
    scale = np.abs(np.array(want)).max()
    np.testing.assert_allclose(rows, np.array(want), rtol=0, atol=1e-3 * scale)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autotune_leaves_the_probe_record_alone(fx, precision):
    """Autotuning between steps records no rows from its trial steps: the record equals that of the
    same steps without tuning (the tuned kernel variant and sort interval give identical results)."""
    fetdpic, _ = fx
    w = _workload(55)
    pts = _points(w, 20, 5)
    out = []
    for tune in (True, False):
        s = fetdpic.Simulation(w, precision=precision, spai_level=1).load()
        s.set_probes(pts, capacity=32)
        s.step(3, "vay")
        if tune:
            s.autotune("vay", trial_steps=8)
        s.step(5, "vay").sync()
        out.append(s.read_probes())
        s.close()
    assert out[0][1] == out[1][1] == 8
    assert np.array_equal(out[0][0], out[1][0])


def test_probe_outside_mesh_rejected(fx):
    fetdpic, _ = fx
    w = _workload(54)
    sim = fetdpic.Simulation(w, precision="fp64", spai_level=1).load()
    with pytest.raises(fetdpic.FetdpicError) as ei:
        sim.set_probes(np.array([[0.5 * w.mesh.lx, 0.5 * w.mesh.ly], [-1.0, 0.0]]))
    assert ei.value.code == fetdpic.EOUTSIDE
    sim.close()


def _kinetic(species_list):
    """sum over particles of m c^2 (gamma - 1), gamma = sqrt(1 + |u|^2 / c^2) (superparticle mass m)."""
    c = inputs.C_LIGHT
    return sum(float((m * c * c * (np.sqrt(1.0 + (u * u).sum(axis=1) / (c * c)) - 1.0)).sum())
               for m, u in species_list)


def bernstein_run(fetdpic, w, precision, n_probes, steps):
    """(k, omega, P) of E_x on a line across the middle, and (kinetic, field) energy changes over the
    run relative to the initial kinetic energy (field energy of the uniform B0 subtracted)."""
    L = w.mesh.lx
    x = (np.arange(n_probes) + 0.5) * L / n_probes
    pts = np.stack([x, np.full(n_probes, 0.5 * w.mesh.ly)], axis=1)
    sim = fetdpic.Simulation(w, precision=precision, spai_level=2, sort_interval=16, use_graphs=True,
                             check_interval=steps).load()
    sim.set_probes(pts, capacity=steps)
    sim.step(steps, "vay").sync()
    rows, total = sim.read_probes()
    k0 = _kinetic([(s.m, s.u) for s in w.species])
    k1 = _kinetic([(s.m, sim.read_species(i)["u"]) for i, s in enumerate(w.species)])
    w0 = w.b0 ** 2 / (2 * inputs.MU0) * w.mesh.lx * w.mesh.ly      # e = 0, b = B0 A_f at the start
    w1 = fetdpic.fetdpic_check(sim.h, 0)["energy"]
    sim.close()
    assert total == steps
    return bernstein.spectrum(rows[:, :, 0], L / n_probes, w.dt), ((k1 - k0) / k0, (w1 - w0) / k0)


BERNSTEIN_CASES = {
    # PEC square, 8,192 triangles, 327,680 particles, kT = 0.1 mc^2, omega_c/omega_p = 0.5
    "square": (lambda: inputs.pair_plasma(64, 20, kT=0.1, wc_over_wp=0.5, seed=2, pusher="vay"),
               128, 16384, (1, 2, 3, 4)),
    # the benchmark workload itself: 200,978 triangles, 8,039,120 particles (16,384 steps of each path)
    "pair-200k": (lambda: inputs.pair_plasma(317, 20, kT=0.1, wc_over_wp=0.5, seed=2, pusher="vay"),
                  256, 16384, (1, 2, 3, 4)),
    # the paper's geometry (Sec. III.C): a 1024 x 4 strip periodic top and bottom (PEC in place of
    # PML at the ends), 8,192 triangles, 327,680 particles, kT = 0.05 mc^2, omega_p = 3 omega_c
    "periodic-strip": (lambda: inputs.pair_plasma(1024, 20, kT=0.05, wc_over_wp=1 / 3, seed=6, pusher="vay",
                                                  ny=4, periodic_y=True),
                       256, 32768, (1, 2, 3, 4, 5)),
}


@pytest.mark.parametrize("case", sorted(BERNSTEIN_CASES))
def test_bernstein_band_frequencies_fp32_vs_fp64(fx, case):
    """Pair plasma, E_x on a line of probes every step in each precision, the (k, omega) power of
    each, and the power-weighted frequency of each cyclotron-harmonic band [(n - 1/2) omega_c,
    (n + 1/2) omega_c).  The FP32 path's band frequencies agree with the FP64 path's within one
    frequency bin of the record (2 pi / (N dt)); the two runs start from the same state and
    diverge only through rounding.  Energy: the kinetic and field energy changes over the run
    (units of the initial kinetic energy K0; the same self-heating in both) agree within 1e-3 K0
    between the precisions."""
    fetdpic, _ = fx
    make, n_probes, steps, bands = BERNSTEIN_CASES[case]
    w = make()
    wc = inputs.Q_E * w.b0 / inputs.M_E
    (k, om, P64), en64 = bernstein_run(fetdpic, w, "fp64", n_probes, steps)
    (_, _, P32), en32 = bernstein_run(fetdpic, w, "fp32", n_probes, steps)
    c64 = bernstein.band_centroids(k, om, P64, wc, harmonics=bands)
    c32 = bernstein.band_centroids(k, om, P32, wc, harmonics=bands)
    res = 2 * math.pi / (steps * w.dt)
    err = np.abs(c32 - c64) / wc
    print(case, "band centroids / wc fp64", c64 / wc, "fp32", c32 / wc, "error / wc", err, "bin / wc", res / wc)
    print(case, "energy change / K0 (kinetic, field, total) fp64", en64, sum(en64), "fp32", en32, sum(en32))
    assert np.isfinite(c64).all() and np.isfinite(c32).all()
    assert (err < res / wc).all(), err
    assert abs(sum(en32) - sum(en64)) < 1e-3, (en32, en64)
    assert abs(en32[0] - en64[0]) < 1e-3 and abs(en32[1] - en64[1]) < 1e-3
