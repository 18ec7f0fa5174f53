"""Lane-by-lane host model of the FP32 particle kernel's current reduction (CPU only).

The kernel (two particles per lane) reduces the fixed-point current of the particles that stay in
their triangle over runs of equal triangle across a warp: a lane's first particle that belongs to a
different run than its second is handed to the previous lane or deposits on its own; the run heads
deposit the run sums with the edge words of their own second particle's triangle.  This model
replays those shuffles on random warps (sorted runs, drifted particles, walkers and padding) and
checks that every triangle receives exactly the current of its particles, and that no head deposits
a run of another triangle.
"""
import numpy as np


def _up(x):
    return [x[0]] + x[:-1]


def _down(x):
    return x[1:] + [x[-1]]


def _reduce(akey, bkey, av, bv):
    dep, wrong = {}, 0
    L = 32

    def add(k, v):
        dep[k] = dep.get(k, 0) + v

    same = [akey[l] == bkey[l] for l in range(L)]
    key = list(bkey)
    okey = [-1 if same[l] else akey[l] for l in range(L)]
    kp = _up(key)
    given = [l > 0 and okey[l] >= 0 and okey[l] == kp[l] for l in range(L)]
    for l in range(L):
        if okey[l] >= 0 and not given[l]:
            add(okey[l], av[l])
    gd, on = _down(given), _down(list(av))
    v0 = [bv[l] + (av[l] if same[l] else 0) + (on[l] if (gd[l] and l < 31) else 0) for l in range(L)]
    k = list(key)
    kpp = _up(k)
    for l in range(L):
        if (l == 0 or kpp[l] != k[l]) and k[l] >= 0:
            e, s = l, 0
            while e < L and k[e] == k[l]:
                s += v0[e]
                e += 1
            wrong += bkey[l] != k[l]
            add(bkey[l], s)
    return {a: b for a, b in dep.items() if b}, wrong


def _truth(akey, bkey, av, bv):
    t = {}
    for l in range(32):
        for kk, vv in ((akey[l], av[l]), (bkey[l], bv[l])):
            if kk >= 0:
                t[kk] = t.get(kk, 0) + vv
    return {a: b for a, b in t.items() if b}


def test_every_triangle_gets_exactly_its_current():
    rng = np.random.default_rng(0)
    for _ in range(4000):
        keys = np.array(sorted(rng.integers(0, 4, 64)))
        stray = rng.random(64) < rng.uniform(0, 0.6)          # drifted since the last sort
        keys[stray] = rng.integers(10, 14, stray.sum())
        keys[rng.random(64) < 0.1] = -1                        # walkers and padding
        a, b = keys[0::2].tolist(), keys[1::2].tolist()
        av = [int(rng.integers(1, 1000)) if x >= 0 else 0 for x in a]
        bv = [int(rng.integers(1, 1000)) if x >= 0 else 0 for x in b]
        got, wrong = _reduce(a, b, av, bv)
        assert wrong == 0
        assert got == _truth(a, b, av, bv)


def test_runs_split_by_walkers_and_strays():
    """A run interrupted by walkers (key -1) and by lone particles of other triangles, with first
    particles handed across lanes: still exact."""
    b = [3] * 6 + [-1, 3, 13, 3, -1, -1, 3] + [4] * 19
    a = [3] * 6 + [3, -1, 3, 13, 3, 4, -1] + [4] * 19
    av = [i + 1 if x >= 0 else 0 for i, x in enumerate(a)]
    bv = [i + 101 if x >= 0 else 0 for i, x in enumerate(b)]
    got, wrong = _reduce(a, b, av, bv)
    assert wrong == 0 and got == _truth(a, b, av, bv)
