"""Pins of the oracle's relativistic pushers (Sec. II.C) against closed forms."""
import json
import math
import os

import numpy as np
import pytest

from paper_1707_04333_gb300 import inputs

C = inputs.C_LIGHT
QE, ME = inputs.Q_E, inputs.M_E
PUSHERS = ["boris", "boris_tan", "vay", "hc"]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def _u_of_gamma(g, ang):
    s = C * math.sqrt(g * g - 1.0)
    return np.array([s * math.cos(ang), s * math.sin(ang), 0.0])


def _theta(pusher, beta, g):
    if pusher == "boris_tan":
        return 2 * beta / g
    if pusher == "hc":
        sig = g * g - beta * beta
        gh = math.sqrt(0.5 * (sig + math.sqrt(sig * sig + 4 * beta * beta)))
        # independent check of gamma_H = gamma(u_bar): |u_bar|^2 = (g^2-1) cos^2(theta/2)
        th = 2 * math.atan(abs(beta) / gh)
        assert abs(1 + (g * g - 1) * math.cos(th / 2) ** 2 - gh * gh) < 1e-12 * g * g
        return 2 * math.atan(beta / gh)
    return 2 * math.atan(beta / g)


@pytest.mark.parametrize("pusher", PUSHERS)
@pytest.mark.parametrize("g", [1.1, 2.0, 10.0, 1000.0])
def test_pure_magnetic_rotation_angle(oracle_mod, pusher, g):
    """E = 0: every pusher rotates u about z and keeps |u|.  The angle is
    2 atan(|beta|/gamma) for Boris and Vay, 2|beta|/gamma for Boris with the tan
    correction, and 2 atan(|beta|/gamma_H) for Higuera-Cary, whose gamma_H is the
    Lorentz factor of the mean momentum (u^- + u^+)/2 (Sec. II.C(c)): with
    |u_bar| = |u| cos(theta/2) and tan(theta/2) = |beta|/gamma_H this gives
    gamma_H^4 - (gamma^2 - |beta|^2) gamma_H^2 - |beta|^2 = 0."""
    q, m, B, dt = -QE, ME, 1.0, 1e-12
    alpha = q * dt / (2 * m)
    u0 = _u_of_gamma(g, 0.3)
    u, gn = oracle_mod.push_only(pusher, alpha, C, [0, 0, 0], [0, 0, B], u0)
    assert u[2] == 0.0
    np.testing.assert_allclose(np.linalg.norm(u), np.linalg.norm(u0), rtol=1e-15)
    np.testing.assert_allclose(gn, g, rtol=1e-14)
    ang = math.atan2(u0[0] * u[1] - u0[1] * u[0], u0 @ u)
    beta = alpha * B
    want = _theta(pusher, beta, g)
    # u x t with t along +z for beta > 0 turns u clockwise: angle = -want
    np.testing.assert_allclose(ang, -want, rtol=1e-12)


@pytest.mark.parametrize("pusher", PUSHERS)
def test_electric_only_kick(oracle_mod, pusher):
    """B = 0: all pushers reduce to u^{n+1/2} = u^{n-1/2} + 2 alpha E."""
    q, m, dt = QE, ME, 1e-12
    alpha = q * dt / (2 * m)
    E = np.array([2e8, -5e7, 0.0])
    u0 = _u_of_gamma(3.0, 1.0)
    u, _ = oracle_mod.push_only(pusher, alpha, C, E, [0, 0, 0], u0)
    np.testing.assert_allclose(u, u0 + 2 * alpha * E, rtol=1e-15, atol=1e-15 * np.abs(u0).max())


def test_cross_pusher_equality_pure_b(oracle_mod):
    """With E = 0 Boris and Vay give the same rotation (to round-off); Higuera-Cary differs
    at O(|beta|^3) through gamma_H (see the rotation-angle pin)."""
    alpha = -QE * 1e-12 / (2 * ME)
    for g in (1.01, 5.0, 300.0):
        u0 = _u_of_gamma(g, 2.0)
        outs = [oracle_mod.push_only(p, alpha, C, [0, 0, 0], [0, 0, 0.7], u0)[0] for p in ("boris", "vay")]
        for o in outs[1:]:
            np.testing.assert_allclose(o, outs[0], rtol=0, atol=4e-15 * np.linalg.norm(u0))


def test_vay_force_free_drift(oracle_mod):
    """E + v x B = 0 (v = E x B / B^2): Vay keeps u unchanged (its design property);
    Higuera-Cary too; Boris does not."""
    B = np.array([0, 0, 1.0])
    vd = 0.9 * C
    E = np.array([0.0, vd * B[2], 0.0])       # v = (vd, 0, 0): v x B = (0, -vd B, 0)
    g = 1 / math.sqrt(1 - 0.81)
    u0 = np.array([g * vd, 0.0, 0.0])
    alpha = -QE * 1e-11 / (2 * ME)
    dev = {}
    for p in ("vay", "hc", "boris"):
        u = u0.copy()
        for _ in range(200):
            u, _ = oracle_mod.push_only(p, alpha, C, E, B, u)
        dev[p] = np.linalg.norm(u - u0) / np.linalg.norm(u0)
    assert dev["vay"] < 1e-13
    assert dev["hc"] < 1e-13
    assert dev["boris"] > 1e-6


def _orbit_run(oracle_mod, pusher, g, dt_factor, nsteps, b0=1.0, only_particles=True):
    """Single electron at the centre of a 1 m PEC square with uniform B_z = b0."""
    m = inputs.jittered_delaunay(16, 16, 1.0, 1.0, 0.3, seed=11)
    wc = QE * b0 / ME
    dt = dt_factor / wc
    sim = oracle_mod.OracleSim(m.nodes, m.triangles, dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                               spai_level=1, b0=b0)
    u0 = _u_of_gamma(g, 0.7)[:2]
    x0 = np.array([[0.5, 0.5]])
    sim.load(-QE, ME, x0, u0[None, :])
    xs = [x0[0].copy()]
    for _ in range(nsteps):
        sim.step(pusher, only_particles=only_particles)
        s = sim.species[0]
        xs.append(np.array([s["x"][0], s["y"][0]]))
    return sim, np.array(xs), u0, dt


@pytest.mark.parametrize("pusher", PUSHERS)
@pytest.mark.parametrize("g", [1.1, 2.0, 10.0])
def test_discrete_orbit_closed_form(oracle_mod, pusher, g):
    """Config-1 orbit (dt = 0.05/omega_c, 10^4 steps) against the exact discrete map
    z_N = z_0 + (dt/gamma) w rho (rho^N - 1)/(rho - 1), rho = exp(-i theta) (electron, B_z > 0)."""
    n = 10_000
    sim, xs, u0, dt = _orbit_run(oracle_mod, pusher, g, 0.05, n)
    beta = abs(-QE * dt / (2 * ME)) * 1.0
    theta = _theta(pusher, beta, g)
    rho = complex(math.cos(theta), math.sin(theta))   # electron: counter-clockwise
    w0 = complex(u0[0], u0[1])
    k = np.arange(n + 1)
    z = complex(0.5, 0.5) + (dt / g) * w0 * rho * (rho ** k - 1) / (rho - 1)
    radius = abs(w0) * dt / g / (2 * math.sin(theta / 2))
    err = np.abs((xs[:, 0] + 1j * xs[:, 1]) - z).max()
    assert err < 1e-10 * radius * n ** 0.5 + 1e-13, (err, radius)


@pytest.mark.parametrize("pusher", PUSHERS)
def test_continuum_gyro_radius_and_frequency(oracle_mod, pusher):
    """Relativistic gyro-radius gamma m v/(|q|B) and gyrofrequency |q|B/(gamma m) to 1e-6,
    at a step small enough that the O((omega dt)^2) discretisation error is below it."""
    g = 2.0
    wg = QE * 1.0 / (g * ME)
    dtf = 0.002 * g            # omega dt = 0.002
    n = 4000
    sim, xs, u0, dt = _orbit_run(oracle_mod, pusher, g, dtf, n)
    z = xs[:, 0] + 1j * xs[:, 1]
    # circle fit by the mean of the points over whole turns -> centre; radius from distances
    per = 2 * math.pi / (wg * dt)
    nt = int(n // per) * per
    cnt = int(nt)
    centre = z[:cnt].mean()
    r = np.abs(z[:cnt] - centre)
    v = math.sqrt(g * g - 1) / g * C
    r_th = g * ME * v / (QE * 1.0)
    np.testing.assert_allclose(r.mean(), r_th, rtol=1e-6)
    ang = np.unwrap(np.angle(z - centre))
    freq = (ang[cnt - 1] - ang[0]) / ((cnt - 1) * dt)
    np.testing.assert_allclose(abs(freq), wg, rtol=1e-6)


def test_synchrocyclotron_constants_from_paper(oracle_mod):
    """The paper's synchrocyclotron numbers (Sec. III.A): B = m0 v0/(q r) = 2.84281e-3 T for r = 0.02 m,
    RF 79.6 MHz = qB/(2 pi m0).  A Boris-tan oracle orbit with v0 = 1e7 m/s in that B closes at
    r = gamma m v/(qB) and turns at qB/(2 pi gamma m)."""
    gd = json.load(open(GOLDEN))["synchrocyclotron"]
    B_paper = ME * gd["v0"] / (QE * gd["r"])
    np.testing.assert_allclose(B_paper, gd["B"], rtol=2e-6)
    np.testing.assert_allclose(QE * gd["B"] / (2 * math.pi * ME) / 1e6, gd["f_MHz"], atol=0.05)
    g = 1 / math.sqrt(1 - (gd["v0"] / C) ** 2)
    m = inputs.jittered_delaunay(16, 16, 1.0, 1.0, 0.3, seed=5)
    dt = 1e-11
    sim = oracle_mod.OracleSim(m.nodes, m.triangles, dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                               spai_level=1, b0=gd["B"])
    # injected at (0.52, 0.5) moving along +y: centre at (0.5, 0.5) for an electron (counter-clockwise)
    sim.load(-QE, ME, np.array([[0.52, 0.5]]), np.array([[0.0, g * gd["v0"]]]))
    pts = []
    nsteps = int(round(2 * math.pi * g * ME / (QE * gd["B"]) / dt))
    for _ in range(nsteps):
        sim.step("boris_tan", only_particles=True)
        pts.append((sim.species[0]["x"][0], sim.species[0]["y"][0]))
    pts = np.array(pts)
    r = np.hypot(pts[:, 0] - 0.5, pts[:, 1] - 0.5)
    np.testing.assert_allclose(r.mean(), gd["r"], rtol=1e-3)     # gamma - 1 = 5.6e-4
    f = QE * gd["B"] / (2 * math.pi * g * ME)
    np.testing.assert_allclose(f / 1e6, gd["f_MHz"], rtol=1.5e-3)
