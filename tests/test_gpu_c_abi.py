"""The library driven from plain C (tests/c_abi_roundtrip.c) against the oracle run on the same mesh,
particles and steps."""
import os
import subprocess

import numpy as np
import pytest

from paper_1707_04333_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_matches_oracle(tmp_path):
    from paper_1707_04333_gb300 import build_lib
    build_lib.build()
    from oracle import oracle
    oracle.build()
    libdir = os.path.dirname(build_lib.LIB)
    exe = str(tmp_path / "c_abi_roundtrip")
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_abi_roundtrip.c"), "-L", libdir, "-lfetdpic",
                        f"-Wl,-rpath,{libdir}", "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    got = np.array([[float(v) for v in line.split()] for line in r.stdout.strip().splitlines()])
    # the same problem on the oracle: 4 x 4 cells, two triangles each, B_z = 0.05 T, dt = 1e-10 s
    n = 4
    g = np.arange(n + 1) / n
    nodes = np.array([[x, y] for y in g for x in g])
    tri = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            b, c = a + 1, a + n + 1
            tri += [[a, b, c + 1], [a, c + 1, c]]
    ora = oracle.OracleSim(nodes, np.array(tri), 1e-10, eps0=inputs.EPS0, mu0=inputs.MU0, c=inputs.C_LIGHT,
                           spai_level=1, b0=0.05)
    ora.load(-inputs.Q_E, inputs.M_E, np.array([[0.31, 0.42], [0.66, 0.71]]),
             np.array([[2.0e7, -1.0e7], [-3.0e7, 5.0e6]]))
    for _ in range(3):
        ora.step("boris")
    s = ora.species[0]
    want = np.stack([s["x"], s["y"], s["ux"], s["uy"], s["cell"]], axis=1)
    assert np.array_equal(got[:, 4], want[:, 4])                        # triangles
    np.testing.assert_allclose(got[:, :2], want[:, :2], rtol=0, atol=1e-12)
    np.testing.assert_allclose(got[:, 2:4], want[:, 2:4], rtol=1e-12)
