"""GPU runs of the paper-shaped workloads against closed forms and the oracle:
the relativistic cyclotron (10^4 steps, discrete orbit in closed form), its
precision form (FP32 error budget), the high-gamma beam in crossed fields
(FP64 push branch of the FP32 path), and a batch of uneven pair plasmas in one
launch."""
import math

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


def _theta(pusher, beta, g):
    if pusher == "boris_tan":
        return 2 * beta / g
    if pusher == "hc":
        sig = g * g - beta * beta
        gh = math.sqrt(0.5 * (sig + math.sqrt(sig * sig + 4 * beta * beta)))
        return 2 * math.atan(beta / gh)
    return 2 * math.atan(beta / g)


@pytest.mark.parametrize("pusher", ["boris", "vay", "hc"])
@pytest.mark.parametrize("g", [1.1, 2.0, 10.0])
def test_cyclotron_discrete_orbit_fp64(fx, pusher, g):
    """Cyclotron case (64 electrons, B_z = 1 T, dt = 0.05/omega_c, 10^4 steps, field update on,
    CUDA graphs): every electron follows the exact discrete rotation map
    z_N = z_0 + (dt/gamma) w rho (rho^N - 1)/(rho - 1) to 1e-10 of its orbit radius (the
    self-field of 64 electrons is far below that)."""
    fetdpic, _ = fx
    w = inputs.cyclotron(gamma=g, n=64, nx=32, seed=1, pusher=pusher)
    sim = fetdpic.Simulation(w, precision="fp64", spai_level=2, sort_interval=-1, use_graphs=True).load()
    n = 10_000
    sim.step(n, pusher).sync()
    got = sim.read_species(0)
    s = w.species[0]
    beta = QE * w.dt * w.b0 / (2 * ME)
    th = _theta(pusher, beta, g)
    rho = complex(math.cos(th), math.sin(th))           # electron in B_z > 0: counter-clockwise
    w0 = s.u[:, 0] + 1j * s.u[:, 1]
    z0 = s.x[:, 0] + 1j * s.x[:, 1]
    zN = z0 + (w.dt / g) * w0 * rho * (rho ** n - 1) / (rho - 1)
    radius = np.abs(w0) * w.dt / g / (2 * math.sin(th / 2))
    err = np.abs(got["x"][:, 0] + 1j * got["x"][:, 1] - zN)
    assert (err < 1e-10 * radius * math.sqrt(n) + 1e-12).all(), (err / radius).max()
    np.testing.assert_allclose(np.abs(got["u"][:, 0] + 1j * got["u"][:, 1]), np.abs(w0), rtol=1e-12)
    sim.close()


def test_cyclotron_walk_stress_matches_oracle(fx):
    """Walk-stress variant (r_g = 0.25 m: every electron crosses many triangles): 2000 coupled FP64
    steps on the GPU stay with the oracle (same triangles, positions to 1e-9)."""
    fetdpic, oracle = fx
    w = inputs.cyclotron(gamma=2.0, n=64, nx=32, seed=3, pusher="vay", walk_stress=True)
    sim = fetdpic.Simulation(w, precision="fp64", spai_level=1, sort_interval=8).load()
    ora = oracle.OracleSim(w.mesh.nodes, w.mesh.triangles, w.dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                           spai_level=1, b0=w.b0)
    ora.load(w.species[0].q, w.species[0].m, w.species[0].x, w.species[0].u)
    sim.step(2000, "vay").sync()
    for _ in range(2000):
        ora.step("vay")
    got = sim.read_species(0)
    o = ora.species[0]
    assert np.array_equal(got["cell"], o["cell"])
    np.testing.assert_allclose(got["x"][:, 0], o["x"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(got["x"][:, 1], o["y"], rtol=0, atol=1e-9)


def test_cyclotron_precision_form_fp32(fx):
    """Precision form of the cyclotron case: FP32 path vs the FP64 oracle over 10^4 steps;
    gyro-frequency error < 1e-4 (the FP32 error budget), |u| drift < 1e-4 (FP32 rounding of a rotation
    that conserves |u| exactly in exact arithmetic), continuity residual at FP32 round-off every
    100 steps.  The FP32 residual is the rounding of the stored barycentrics (sum 1 to one FP32 ulp)
    relative to one step's barycentric displacement, here ~2.5e-3 (sub-cell orbits): ~ eps32 / 2.5e-3
    = 2.4e-5, so the bound is 1e-4."""
    fetdpic, oracle = fx
    w = inputs.cyclotron(gamma=2.0, n=64, nx=32, seed=1, pusher="boris")
    sim = fetdpic.Simulation(w, precision="fp32", spai_level=2, sort_interval=16, check_interval=100).load()
    n = 10_000
    s = w.species[0]
    beta = QE * w.dt * w.b0 / (2 * ME)
    th = _theta("boris", beta, 2.0)
    for k in range(n // 100):
        sim.step(100, "boris").sync()
        c = fetdpic.fetdpic_check(sim.h, 0)
        assert c["dce"] < 1e-4
    got = sim.read_species(0)
    # accumulated rotation angle vs the exact n * theta: frequency error = angle error / total
    a0 = np.angle(s.u[:, 0] + 1j * s.u[:, 1])
    aN = np.angle(got["u"][:, 0] + 1j * got["u"][:, 1])
    want = (a0 + n * th) % (2 * np.pi)
    dphi = np.abs(np.angle(np.exp(1j * (aN - want))))
    assert (dphi / (n * th) < 1e-4).all(), (dphi / (n * th)).max()
    np.testing.assert_allclose(np.abs(got["u"][:, 0] + 1j * got["u"][:, 1]), np.abs(s.u[:, 0] + 1j * s.u[:, 1]),
                               rtol=1e-4)
    sim.close()


@pytest.mark.parametrize("pusher", ["hc", "vay", "boris"])
def test_high_gamma_beam_fp32_vs_oracle(fx, pusher):
    """High-gamma beam (gamma log-uniform in [10, 1000], external E_x = 0.5 c B_z, B_z = 1 T): the
    FP32 path pushes these particles in FP64 and stays within FP32 round-off of the oracle over
    5 coupled steps (momenta 1e-5 relative, positions 1e-6 of the domain)."""
    fetdpic, oracle = fx
    w = inputs.high_gamma_beam(n_tri_side=60, n_particles=20_000, seed=4, pusher=pusher, side=10.0)
    sim = fetdpic.Simulation(w, precision="fp32", spai_level=1, sort_interval=-1).load()
    ora = oracle.OracleSim(w.mesh.nodes, w.mesh.triangles, w.dt, eps0=inputs.EPS0, mu0=inputs.MU0, c=C,
                           spai_level=1, b0=w.b0, ext=w.ext)
    ora.load(w.species[0].q, w.species[0].m, w.species[0].x, w.species[0].u, w.species[0].hint)
    sim.step(5, pusher).sync()
    for _ in range(5):
        ora.step(pusher)
    got = sim.read_species(0)
    o = ora.species[0]
    umag = np.hypot(o["ux"], o["uy"])
    du = np.hypot(got["u"][:, 0] - o["ux"], got["u"][:, 1] - o["uy"])
    assert (du <= 1e-5 * umag).all(), (du / umag).max()
    dx = np.hypot(got["x"][:, 0] - o["x"], got["x"][:, 1] - o["y"])
    assert (dx <= 1e-6 * 10.0).all(), dx.max()
    assert (got["cell"] == o["cell"]).mean() > 0.999
    sim.close()


def test_batched_uneven_instances(fx):
    """Eight uneven pair-plasma instances (different meshes, particle counts, fields, temperatures,
    time steps) advance in one launch per stage: each equals its own single-instance run bit for
    bit (FP32 and FP64), and each instance's continuity residual stays at round-off."""
    fetdpic, _ = fx
    ws = inputs.batched_pair_plasmas(n_inst=8, seed=5, f_range=(500, 6000), p_range=(2_000, 60_000))
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-5)):
        both = fetdpic.Simulation(ws, precision=prec, spai_level=1, sort_interval=4, check_interval=3).load()
        both.step(9, "vay").sync()
        for k in range(len(ws)):
            c = fetdpic.fetdpic_check(both.h, k)
            assert c["dce"] < tol, (k, c)
        for k, w in enumerate(ws):
            one = fetdpic.Simulation(w, precision=prec, spai_level=1, sort_interval=4, check_interval=3).load()
            one.step(9, "vay").sync()
            fa, fb = both.read_fields(k), one.read_fields(0)
            for name in ("e", "b", "j"):
                assert np.array_equal(fa[name], fb[name]), (prec, k, name)
            for s in range(2):
                ga, gb = both.read_species(2 * k + s), one.read_species(s)
                for name in ("x", "u", "cell"):
                    assert np.array_equal(ga[name], gb[name]), (prec, k, s, name)
            one.close()
        both.close()
