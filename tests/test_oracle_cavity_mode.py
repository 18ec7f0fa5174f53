"""Pin of the oracle's field-update scale: the lowest TE mode of an empty PEC square cavity.

In a square cavity of side L with perfectly conducting walls, B_z = B0 cos(pi x / L) cos(w t),
E_y = c B0 sin(pi x / L) sin(w t) solves Maxwell's equations with tangential E = 0 on all four
walls, at the angular frequency w = c pi / L.  The leapfrog of Sec. II.A (Eqs. (semi.dis.curl.1)
and (semi.dis.curl.2)) reproduces it up to the mesh's O((kh)^2) dispersion and the leapfrog's
O((w dt)^2) phase error, so the frequency of the oracle's discrete b oscillation fixes the product
of every scale factor in the update: the diagonal [*mu^-1] = 1/(mu0 A_f), the Galerkin [*eps]
behind M, and the dt of each half step.  A factor 2 in any of them moves w by sqrt(2) (or, for
[*eps], 1/sqrt(2)); the tests below check that such a mistake, planted in a copy of the step
loop, fails the same bound.  (CPU only.)
"""
import ctypes as C

import numpy as np
import pytest

from paper_1707_04333_gb300 import inputs

CL = inputs.C_LIGHT


def _face_flux_cos(om, L):
    """b_f = integral over triangle f of cos(pi x / L): 7-point Gauss rule of degree 5."""
    a, b = 0.059715871789770, 0.470142064105115
    c, d = 0.797426985353087, 0.101286507323456
    w = np.array([0.225] + [0.132394152788506] * 3 + [0.125939180544827] * 3)
    bary = np.array([[1 / 3, 1 / 3, 1 / 3], [a, b, b], [b, a, b], [b, b, a], [c, d, d], [d, c, d], [d, d, c]])
    x = bary @ om.nx.T                       # [7, nf]
    area = 0.5 * om.d2A
    return (w[:, None] * np.cos(np.pi * x / L)).sum(0) * area


def _mode_amplitude(om, b, L):
    xc = om.nx.mean(1)
    return float(np.sum(b * np.cos(np.pi * xc / L)))


def _frequency(series, dt):
    """Angular frequency from the zero crossings of a sampled oscillation: crossing times by
    linear interpolation, then a least-squares line through them (half a period apart)."""
    s = np.asarray(series)
    k = np.nonzero(np.signbit(s[:-1]) != np.signbit(s[1:]))[0]
    t = (k + s[k] / (s[k] - s[k + 1])) * dt
    assert len(t) >= 4, len(t)
    half = np.polyfit(np.arange(len(t)), t, 1)[0]
    return np.pi / half


def _cavity(oracle_mod, n=16, exact=True, seed=71):
    m = inputs.jittered_delaunay(n, n, 1.0, 1.0, 0.3, seed=seed)
    om = oracle_mod.OracleMesh(m.nodes, m.triangles)
    el = np.linalg.norm(m.nodes[om.edge[:, 1]] - m.nodes[om.edge[:, 0]], axis=1)
    dt = 0.3 * el.min() / CL
    sim = oracle_mod.OracleSim(m.nodes, m.triangles, dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=CL,
                               spai_level=2, exact_inverse=exact)
    sim.b = _face_flux_cos(sim.mesh, 1.0)
    return sim


def _periods_steps(sim, periods):
    return int(periods * (2.0 / CL) / sim.dt) + 2      # period of the exact mode: 2 L / c


def _planted_step(oracle_mod, sim, f_dt=1.0, a_dt=1.0, mu_scale=1.0):
    """The oracle's field-only step (Faraday, C^T H b, Ampere) written out from its C functions,
    with factors planted in the Faraday dt, the Ampere dt or mu0 of [*mu^-1]."""
    lib = oracle_mod.lib()
    m = sim.mesh
    p = oracle_mod._p
    b_new = np.zeros(m.nf)
    lib.ora_faraday(m.cs, C.c_double(f_dt * sim.dt), p(sim.e), p(sim.b), p(b_new))
    r = np.zeros(m.ne)
    i0 = np.zeros(m.ne)
    lib.ora_curl_h(m.cs, C.c_double(mu_scale * sim.mu0), p(b_new), p(i0), p(r))
    lib.ora_ampere(len(m.free), p(m.free), p(sim._rp), p(sim._ci), p(sim._v), C.c_double(a_dt * sim.dt),
                   p(r), p(sim.e), p(sim.d), m.ne)
    sim.b = b_new


def test_lowest_te_mode_frequency_exact_inverse(oracle_mod):
    """Exact [*eps]^-1 on a 16 x 16 jittered mesh (kh = pi/16): w within 0.5 % of c pi / L
    (measured: 2e-4 low)."""
    sim = _cavity(oracle_mod, exact=True)
    amp = []
    for _ in range(_periods_steps(sim, 4)):
        sim.step()
        amp.append(_mode_amplitude(sim.mesh, sim.b, 1.0))
    w = _frequency(amp, sim.dt)
    assert abs(w / (CL * np.pi) - 1.0) < 0.005, w / (CL * np.pi)
    # the field-only step written out above is the oracle's step (bit for bit), so the planted
    # variants below test the same arithmetic
    a = _cavity(oracle_mod, exact=True)
    b = _cavity(oracle_mod, exact=True)
    for _ in range(50):
        a.step()
        _planted_step(oracle_mod, b)
    assert np.array_equal(a.b, b.b) and np.array_equal(a.e, b.e)


def test_lowest_te_mode_frequency_spai(oracle_mod):
    """The level-2 SPAI (the benchmark's M) on a 24 x 24 mesh: w within 0.5 % of c pi / L
    (measured: 4e-4 high)."""
    sim = _cavity(oracle_mod, n=24, exact=False, seed=72)
    amp = []
    for _ in range(_periods_steps(sim, 3)):
        sim.step()
        amp.append(_mode_amplitude(sim.mesh, sim.b, 1.0))
    w = _frequency(amp, sim.dt)
    assert abs(w / (CL * np.pi) - 1.0) < 0.005, w / (CL * np.pi)


@pytest.mark.parametrize("plant", [dict(f_dt=2.0), dict(a_dt=2.0), dict(mu_scale=0.5), dict(mu_scale=2.0)])
def test_planted_scale_error_fails_the_bound(oracle_mod, plant):
    """A factor 2 in the Faraday dt, the Ampere dt or [*mu^-1] moves w by 29-41 %, far outside the 0.5 %
    bound
    (run at Courant 0.15 so the planted update stays stable)."""
    sim = _cavity(oracle_mod, exact=True)
    sim.dt *= 0.5
    amp = []
    for _ in range(_periods_steps(sim, 4)):
        _planted_step(oracle_mod, sim, **plant)
        amp.append(_mode_amplitude(sim.mesh, sim.b, 1.0))
    w = _frequency(amp, sim.dt)
    assert abs(w / (CL * np.pi) - 1.0) > 0.25, (plant, w / (CL * np.pi))
