"""The allocation-free particle read (fetdpic_read_particles_static).

Callers that cannot allocate device memory when they read particles back
(allocation-free real-time loops, or plug-ins whose host framework owns all
device memory) use this entry point; it must give exactly what fetdpic_read
gives.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1707_04333_gb300 import inputs

pytestmark = pytest.mark.gpu


def _static_read(fetdpic, h, species, n):
    L = fetdpic.lib()
    fn = L.fetdpic_read_particles_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    x = np.full((n, 2), np.nan)
    u = np.full((n, 2), np.nan)
    c = np.full(n, -7, np.int32)
    rc = fn(h, species, fetdpic._ptr(x), fetdpic._ptr(u), fetdpic._ptr(c))
    return rc, x, u, c


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_read_matches_fetdpic_read(precision):
    import torch
    assert torch.cuda.is_available()
    from paper_1707_04333_gb300 import build_lib, fetdpic
    build_lib.build()
    w = inputs.pair_plasma(20, 6, kT=0.2, seed=21, pusher="hc")
    sim = fetdpic.Simulation(w, precision=precision, spai_level=1, sort_interval=3).load()
    # not stepped yet: the context has no particle storage, the call must refuse
    rc, *_ = _static_read(fetdpic, sim.h, 0, len(w.species[0].x))
    assert rc == fetdpic.ESTATE
    for rep in range(2):                           # two calls in a row, state changes between them
        sim.step(5, "hc").sync()
        for sid, (_, _, n) in enumerate(sim.species):
            ref = sim.read_species(sid)
            rc, x, u, c = _static_read(fetdpic, sim.h, sid, n)
            assert rc == 0, fetdpic.lib().fetdpic_last_error(sim.h)
            # same kernel and same data: identical, well within the FP64 parity tolerance
            assert np.array_equal(x, ref["x"]) and np.array_equal(u, ref["u"]) and np.array_equal(c, ref["cell"])
    sim.close()


def _uniform_species(m, n, seed):
    rng = np.random.default_rng(seed)
    tri = rng.integers(0, len(m.triangles), n).astype(np.int32)
    x = inputs.sample_in_triangles(m, tri, rng)
    u = rng.normal(0, 1e7, (n, 2))
    return inputs.Species(-inputs.Q_E, inputs.M_E, x, u, tri)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_read_size_limits(precision):
    """The largest species the array holds (262,144 particles: its last byte written) reads the
    same as fetdpic_read; one particle more is rejected with the limit in the message; an empty
    species reads nothing and succeeds."""
    from paper_1707_04333_gb300 import fetdpic
    m = inputs.jittered_delaunay(40, 40, 1.0, 1.0, 0.3, seed=3)
    lim = 262_144
    sp = [_uniform_species(m, lim, 0), _uniform_species(m, lim + 1, 1),
          inputs.Species(inputs.Q_E, inputs.M_E, np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(0, np.int32))]
    sim = fetdpic.Simulation(inputs.Workload("big", m, sp, 1e-12), precision=precision, spai_level=1).load()
    sim.step(1, "boris").sync()
    ref = sim.read_species(0)
    for _ in range(2):
        rc, x, u, c = _static_read(fetdpic, sim.h, 0, lim)
        assert rc == 0, fetdpic.lib().fetdpic_last_error(sim.h)
        assert np.array_equal(x, ref["x"]) and np.array_equal(u, ref["u"]) and np.array_equal(c, ref["cell"])
    rc, *_ = _static_read(fetdpic, sim.h, 1, lim + 1)
    assert rc == fetdpic.EINVAL
    assert b"262144" in fetdpic.lib().fetdpic_last_error(sim.h)
    rc, x, u, c = _static_read(fetdpic, sim.h, 2, 0)
    assert rc == 0 and x.shape == (0, 2)
    sim.close()
