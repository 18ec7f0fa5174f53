"""Pins of the oracle's applied fields that vary in space and time, and the synchrocyclotron case
built on them (Sec. III.A): a magnet over the whole square, an RF field in a vertical gap."""
import math

import numpy as np

from paper_1707_04333_gb300 import inputs

C = inputs.C_LIGHT
QE, ME = inputs.Q_E, inputs.M_E


def _sim(oracle_mod, w, **kw):
    sim = oracle_mod.OracleSim(w.mesh.nodes, w.mesh.triangles, w.dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                               spai_level=1, b0=w.b0, ext=w.ext, **kw)
    for s in w.species:
        sim.load(s.q, s.m, s.x, s.u)
    return sim


def _kinetic(u):
    return ME * C * C * (math.sqrt(1.0 + (u[0] ** 2 + u[1] ** 2) / C ** 2) - 1.0)


def test_unit_weights_reproduce_uniform_external_fields(oracle_mod):
    """Weights 1 and amplitude 1 give bit-identical particles to the uniform external fields."""
    w = inputs.high_gamma_beam(n_tri_side=20, n_particles=500, seed=3, pusher="hc", side=10.0)
    a = _sim(oracle_mod, w, fields=False)
    b = _sim(oracle_mod, w, fields=False)
    b.ext_profile = np.ones((len(w.mesh.triangles), 2))
    for _ in range(5):
        a.step("hc", only_particles=True)
        b.step("hc", only_particles=True)
    for k in ("x", "y", "ux", "uy", "cell"):
        assert np.array_equal(a.species[0][k], b.species[0][k]), k


def test_static_gap_energy_gain(oracle_mod):
    """An electron crossing the gap (|x - 0.5| < 0.01, mesh lines at its edges) of a static
    E_x = -2e5 V/m with no magnetic field gains |q| E w = 4 keV: the work of the field, up to one
    step's displacement at each gap edge (the field acts by the triangle holding the particle at
    the start of a step)."""
    w = inputs.synchrocyclotron(n=100)
    prof = w.ext_profile.copy()
    prof[:, 1] = 0.0                                      # no magnet
    dt = 2e-12
    v0 = 1e7
    g0 = 1.0 / math.sqrt(1 - (v0 / C) ** 2)
    el = inputs.Species(-QE, ME, np.array([[0.47, 0.5]]), np.array([[g0 * v0, 0.0]]), np.full(1, -1, np.int32))
    w2 = inputs.Workload("gap", w.mesh, [el], dt, ext=(-2e5, 0.0, 0.0), ext_profile=prof)
    sim = _sim(oracle_mod, w2, fields=False)
    sim.ext_profile = prof
    vmax = v0
    while sim.species[0]["x"][0] < 0.53:
        sim.step("boris", only_particles=True)
        s = sim.species[0]
        vmax = max(vmax, math.hypot(s["ux"][0], s["uy"][0]))
    s = sim.species[0]
    gain = _kinetic((s["ux"][0], s["uy"][0])) - _kinetic((g0 * v0, 0.0))
    work = QE * 2e5 * 0.02
    assert abs(gain - work) <= QE * 2e5 * vmax * dt * 2, (gain, work)
    assert abs(s["y"][0] - 0.5) < 1e-12 and abs(s["uy"][0]) == 0.0


def _run_synchro(oracle_mod, synchronized, steps):
    w = inputs.synchrocyclotron(n=100)
    sim = _sim(oracle_mod, w, fields=False)
    sim.ext_profile = w.ext_profile
    drive = inputs.RFDrive(w.ext[2], w.dt, synchronized)
    speed, kin, x = [], [], []
    for _ in range(steps):
        sim.ext_amp = drive.amplitude()
        sim.step("boris_tan", only_particles=True)
        s = sim.species[0]
        u = (s["ux"][0], s["uy"][0])
        drive.advance(u)
        g = math.sqrt(1 + (u[0] ** 2 + u[1] ** 2) / C ** 2)
        speed.append(math.hypot(*u) / g)
        kin.append(_kinetic(u))
        x.append(s["x"][0])
    return np.array(speed), np.array(kin), np.array(x), w


def test_synchronised_drive_accelerates_every_crossing(oracle_mod):
    """Synchronised RF (f = qB / (2 pi gamma m0)): the kinetic energy rises at every gap crossing
    over 12 turns, by at most the work |q| E w = 4 keV of a crossing at the crest (plus the field
    the start-of-step triangle applies over at most one step beyond each gap edge) and by at least
    60 % of it (the transit-time factor of the sine over the crossing)."""
    speed, kin, x, w = _run_synchro(oracle_mod, True, 24000)
    in_gap = np.abs(x - 0.5) < 0.01
    edges = np.flatnonzero(np.diff(in_gap.astype(int)) == -1)     # steps where a crossing ends
    assert len(edges) >= 22
    k_at = np.concatenate([[kin[0]], kin[edges]])
    gains = np.diff(k_at)
    work = QE * 2e5 * 0.02
    step = speed.max() * w.dt
    assert (gains > 0.6 * work).all(), gains / work
    assert (gains < work * (1 + 2 * step / 0.02)).all(), gains / work
    assert kin[-1] > 20 * work


def test_unsynchronised_drive_falls_out_of_phase(oracle_mod):
    """Constant RF frequency (the rest-mass cyclotron frequency, 79.6 MHz for the printed field):
    the relativistic mass increase slips the phase; the electron first gains and then loses
    speed, as in the paper's comparison of velocity magnitudes."""
    speed, kin, x, w = _run_synchro(oracle_mod, False, 24000)
    k = int(np.argmax(speed))
    assert 2000 < k < 22000
    assert speed[-1] < 0.8 * speed[k]
    wc = QE * w.ext[2] / ME
    assert abs(wc / (2 * math.pi) / 1e6 - 79.6) < 0.05
