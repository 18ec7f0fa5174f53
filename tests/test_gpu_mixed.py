"""Instances of different kinds in one launch per stage: a periodic strip, a PEC square with applied
fields weighted per triangle and its own amplitude, and a non-neutral load with its initial
electrostatic field.  Each must equal its own single-instance run bit for bit: the batch shares
kernels, never state."""
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
    return fetdpic


def _instances():
    strip = inputs.pair_plasma(16, 6, kT=0.3, wc_over_wp=0.5, seed=71, pusher="vay", ny=6, periodic_y=True)
    square = inputs.pair_plasma(10, 5, kT=0.2, wc_over_wp=0.5, seed=72, pusher="vay")
    nf = len(square.mesh.triangles)
    rng = np.random.default_rng(72)
    square.ext = (3e3, -1e3, 0.2)
    square.ext_profile = np.stack([rng.uniform(0, 1, nf), rng.uniform(0.5, 1.5, nf)], axis=1)
    charged = inputs.pair_plasma(12, 4, kT=0.2, wc_over_wp=0.5, seed=73, pusher="vay")
    p = charged.species[1]
    x = p.x.copy()
    x[:, 0] = np.clip(x[:, 0] + rng.normal(0, 0.1 * charged.mesh.lx, len(x)), 1e-9 * charged.mesh.lx,
                      charged.mesh.lx * (1 - 1e-9))
    charged.species[1] = inputs.Species(p.q, p.m, x, p.u, np.full(len(x), -1, np.int32))
    return [strip, square, charged]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mixed_batch_equals_separate_runs(fx, precision):
    fetdpic = fx
    ws = _instances()
    amp = 0.37                                   # amplitude of the square's applied E

    def advance(sim, k_square, k_charged):
        if k_charged is not None:
            sim.solve_electrostatic(k_charged)
        if k_square is not None:
            sim.set_external_amplitude(amp, k_square)
        sim.step(4, "vay")
        if k_square is not None:
            sim.set_external_amplitude(-amp, k_square)
        sim.step(5, "hc").sync()

    both = fetdpic.Simulation(ws, precision=precision, spai_level=1, sort_interval=3, check_interval=4).load()
    advance(both, 1, 2)
    for k, w in enumerate(ws):
        one = fetdpic.Simulation(w, precision=precision, spai_level=1, sort_interval=3, check_interval=4).load()
        advance(one, 0 if k == 1 else None, 0 if k == 2 else None)
        fa, fb = both.read_fields(k), one.read_fields(0)
        for name in ("e", "b", "j"):
            assert np.array_equal(fa[name], fb[name]), (precision, k, name)
        for s in range(2):
            ga, gb = both.read_species(2 * k + s), one.read_species(s)
            for name in ("x", "u", "cell"):
                assert np.array_equal(ga[name], gb[name]), (precision, k, s, name)
        ca, cb = fetdpic.fetdpic_check(both.h, k), fetdpic.fetdpic_check(one.h, 0)
        assert ca["dce"] == cb["dce"] and ca["dgl"] == cb["dgl"], (k, ca, cb)
        # the energy is a block-wise sum whose partials depend on the instance's offset in the batch
        assert abs(ca["energy"] - cb["energy"]) <= 1e-12 * abs(cb["energy"]), (k, ca, cb)
        one.close()
    c = fetdpic.fetdpic_check(both.h, 2)
    assert c["dgl"] < (1e-12 if precision == "fp64" else 1e-4)       # absolute Gauss law after the solve
    both.close()
