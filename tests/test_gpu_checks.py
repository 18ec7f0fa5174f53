"""GPU conservation checks: discrete continuity (Eq. full.dis.cont) and Gauss law
(Eq. semi.dis.div.2, dual-flux form) computed by the library every step, and the
field energy compared with the oracle's."""
import numpy as np
import pytest

from paper_1707_04333_gb300 import inputs

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


def _workload(seed=41):
    w = inputs.pair_plasma(14, 6, kT=0.3, wc_over_wp=0.5, seed=seed, pusher="vay")
    # shift the positrons so the net charge density is not zero
    rng = np.random.default_rng(seed)
    p = w.species[1]
    x = np.clip(p.x + rng.normal(0, 0.05 * w.mesh.lx, p.x.shape), 1e-9 * w.mesh.lx, w.mesh.lx * (1 - 1e-9))
    w.species[1] = inputs.Species(p.q, p.m, x, p.u, np.full(len(x), -1, np.int32))
    return w


@pytest.mark.parametrize("precision,tol_dce,tol_dgl", [("fp64", 1e-12, 1e-12), ("fp32", 2e-5, 1e-4)])
def test_continuity_and_gauss_every_step(fx, precision, tol_dce, tol_dgl):
    """DCE and DGL residuals (normalised per node by the magnitude of the terms) at round-off of the
    path's arithmetic on every step, through crossings, wall reflections and sorts."""
    fetdpic, _ = fx
    w = _workload()
    sim = fetdpic.Simulation(w, precision=precision, spai_level=2, sort_interval=4, check_interval=1).load()
    worst = [0.0, 0.0]
    for _ in range(25):
        sim.step(1, "vay").sync()
        c = fetdpic.fetdpic_check(sim.h, 0)
        worst = [max(worst[0], c["dce"]), max(worst[1], c["dgl"])]
        assert c["dce"] < tol_dce, c
        assert c["dgl"] < tol_dgl, c
        assert c["energy"] > 0
    sim.close()


def test_energy_matches_oracle(fx):
    """FP64: the library's field energy e.[*eps].e/2 + b.[*mu^-1].b/2 follows the oracle's."""
    fetdpic, oracle = fx
    w = _workload(43)
    sim = fetdpic.Simulation(w, precision="fp64", spai_level=2, sort_interval=-1, check_interval=5).load()
    ora = oracle.OracleSim(w.mesh.nodes, w.mesh.triangles, w.dt, eps0=inputs.EPS0, mu0=inputs.MU0,
                           c=inputs.C_LIGHT, spai_level=2, b0=w.b0)
    for s in w.species:
        ora.load(s.q, s.m, s.x, s.u, s.hint)
    for k in range(15):
        sim.step(1, "vay")
        ora.step("vay")
        if (k + 1) % 5 == 0:
            c = fetdpic.fetdpic_check(sim.h, 0)
            np.testing.assert_allclose(c["energy"], ora.field_energy(), rtol=1e-10)
    sim.close()


def test_checks_per_instance_and_disabled(fx):
    fetdpic, _ = fx
    w1, w2 = _workload(44), _workload(45)
    sim = fetdpic.Simulation([w1, w2], precision="fp64", spai_level=1, check_interval=2).load()
    sim.step(6, "hc").sync()
    for k in range(2):
        c = fetdpic.fetdpic_check(sim.h, k)
        assert c["dce"] < 1e-12 and c["dgl"] < 1e-12 and c["energy"] > 0
    sim.close()
    off = fetdpic.Simulation(w1, precision="fp64", spai_level=1).load()
    off.step(1, "hc").sync()
    with pytest.raises(fetdpic.FetdpicError) as ei:
        fetdpic.fetdpic_check(off.h, 0)
    assert ei.value.code == fetdpic.ESTATE
    off.close()
