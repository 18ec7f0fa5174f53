"""Seeded synthetic workload generators.

This module is shared by the CUDA path, the oracle and the benchmark.  It holds
no arithmetic of the FETD-PIC method itself: it only produces inputs (mesh
nodes and triangles, particle positions with a hint triangle, momenta, species
charges and masses, uniform field amplitudes).  Each consumer derives edges,
Whitney-form geometry, Hodge matrices and field degrees of freedom on its own.

Workload shapes follow the paper's cases (Sec. III): a Delaunay triangulation
of seeded jittered points, a cyclotron test with a handful of electrons, and a
magnetized electron-positron pair plasma loaded pairwise with opposite 2-D
Maxwell-Juettner momenta.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# CODATA constants, MKS (the paper works in MKS units, Sec. I)
C_LIGHT = 299792458.0
Q_E = 1.602176634e-19
M_E = 9.1093837015e-31
EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6


@dataclasses.dataclass
class Mesh:
    nodes: np.ndarray      # [N,2] float64
    triangles: np.ndarray  # [F,3] int32, counter-clockwise
    lx: float
    ly: float
    # periodic walls: (pairs [k,2] int32, (tx, ty)); node pairs[k,1] is node pairs[k,0] moved by (tx, ty)
    periodic: object = None


@dataclasses.dataclass
class Species:
    q: float               # superparticle charge (C per unit depth)
    m: float               # superparticle rest mass
    x: np.ndarray          # [n,2] float64 positions
    u: np.ndarray          # [n,2] float64 u = gamma*v (m/s), loaded as u^{-1/2}
    hint: np.ndarray       # [n] int32 triangle the point was drawn in (a hint, may be off by round-off)


@dataclasses.dataclass
class Workload:
    name: str
    mesh: Mesh
    species: list
    dt: float
    b0: float = 0.0        # uniform initial B_z (projected onto face DoFs by each consumer)
    e0: tuple = (0.0, 0.0)  # uniform initial E (projected onto free-edge DoFs)
    ext: tuple = (0.0, 0.0, 0.0)  # external uniform (E_x, E_y, B_z) added at the particle
    pusher: str = "boris"
    # per-triangle weights [F,2] of the external E and B_z (None = 1 everywhere)
    ext_profile: object = None

    @property
    def n_particles(self) -> int:
        return int(sum(len(s.x) for s in self.species))


def jittered_delaunay(nx: int, ny: int, lx: float = 1.0, ly: float = 1.0,
                      jitter: float = 0.3, seed: int = 1, periodic_y: bool = False) -> Mesh:
    """Delaunay mesh of an (nx+1) x (ny+1) grid of jittered points on [0,lx]x[0,ly].

    Interior points move by up to +-jitter*h in each direction; boundary points
    slide only along their side and corners stay fixed, so the hull is the
    rectangle.  About 2*nx*ny triangles.  periodic_y: the top row repeats the
    bottom row's x positions and Mesh.periodic pairs each bottom node with the
    top node above it, period (0, ly).
    """
    import scipy.spatial

    rng = np.random.default_rng(seed)
    hx, hy = lx / nx, ly / ny
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    x = ii * hx
    y = jj * hy
    jx = rng.uniform(-jitter, jitter, x.shape) * hx
    jy = rng.uniform(-jitter, jitter, y.shape) * hy
    on_x_side = (ii == 0) | (ii == nx)
    on_y_side = (jj == 0) | (jj == ny)
    jx[on_x_side] = 0.0
    jy[on_y_side] = 0.0
    if periodic_y:
        jx[:, ny] = jx[:, 0]
    x = x + jx
    y = y + jy
    pts = np.stack([x.ravel(), y.ravel()], 1)
    tri = scipy.spatial.Delaunay(pts).simplices.astype(np.int32)
    p0, p1, p2 = pts[tri[:, 0]], pts[tri[:, 1]], pts[tri[:, 2]]
    o = (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1])
    cw = o < 0
    tri[cw] = tri[cw][:, [0, 2, 1]]
    keep = o != 0
    tri = np.ascontiguousarray(tri[keep])
    periodic = None
    if periodic_y:
        col = np.arange(nx + 1) * (ny + 1)                  # node id of grid point (i, j) = i (ny+1) + j
        periodic = (np.stack([col, col + ny], 1).astype(np.int32), (0.0, float(ly)))
    return Mesh(np.ascontiguousarray(pts), tri, lx, ly, periodic)


def sample_in_triangles(mesh: Mesh, tri_ids: np.ndarray, rng) -> np.ndarray:
    """Uniform points in the given triangles (square-root barycentric sampling)."""
    r1 = np.sqrt(rng.random(len(tri_ids)))
    r2 = rng.random(len(tri_ids))
    w0 = 1.0 - r1
    w1 = r1 * (1.0 - r2)
    w2 = r1 * r2
    t = mesh.triangles[tri_ids]
    p = mesh.nodes
    return (w0[:, None] * p[t[:, 0]] + w1[:, None] * p[t[:, 1]] + w2[:, None] * p[t[:, 2]])


def maxwell_juttner_2d(n: int, eta: float, rng) -> np.ndarray:
    """In-plane momenta u = gamma*v (m/s) from a 2-D isotropic Maxwell-Juttner law.

    With f ~ exp(-eta*gamma) d^2p the density of gamma on [1, inf) is
    ~ gamma*exp(-eta*gamma), i.e. gamma-1 is a mixture of Exp(eta)
    (weight eta/(eta+1)) and Gamma(2, 1/eta) (weight 1/(eta+1)).
    eta = m0 c^2 / (k_B T).
    """
    pick = rng.random(n) < eta / (eta + 1.0)
    g1 = np.where(pick, rng.exponential(1.0 / eta, n), rng.gamma(2.0, 1.0 / eta, n))
    gamma = 1.0 + g1
    pmag = np.sqrt(gamma * gamma - 1.0) * C_LIGHT
    th = rng.uniform(0.0, 2.0 * math.pi, n)
    return np.stack([pmag * np.cos(th), pmag * np.sin(th)], 1)


def cyclotron(gamma: float = 2.0, n: int = 64, nx: int = 32, seed: int = 1,
              b0: float = 1.0, radius: float = 0.05, pusher: str = "boris",
              walk_stress: bool = False) -> Workload:
    """Relativistic cyclotron test: electrons near the centre of a 1 m PEC square.

    dt = 0.05/omega_c with omega_c = |q| B / m0.  With walk_stress the field is
    lowered so the gyro-radius is 0.25 m and the particles cross many cells.
    """
    mesh = jittered_delaunay(nx, nx, 1.0, 1.0, 0.3, seed)
    rng = np.random.default_rng(seed + 1000)
    speed_u = C_LIGHT * math.sqrt(gamma * gamma - 1.0)
    if walk_stress:
        b0 = speed_u * M_E / (Q_E * 0.25)
    r = radius * np.sqrt(rng.random(n))
    th = rng.uniform(0, 2 * math.pi, n)
    x = np.stack([0.5 + r * np.cos(th), 0.5 + r * np.sin(th)], 1)
    ph = rng.uniform(0, 2 * math.pi, n)
    u = np.stack([speed_u * np.cos(ph), speed_u * np.sin(ph)], 1)
    omega_c = Q_E * b0 / M_E
    dt = 0.05 / omega_c
    hint = np.full(n, -1, np.int32)
    sp = Species(-Q_E, M_E, x, u, hint)
    return Workload(f"cyclotron-g{gamma}", mesh, [sp], dt, b0=b0, pusher=pusher)


def pair_plasma(n_tri_side: int = 317, ppc: int = 20, kT: float = 0.1,
                wc_over_wp: float = 0.5, courant: float = 0.2, seed: int = 2,
                pusher: str = "vay", ny: int | None = None, periodic_y: bool = False) -> Workload:
    """Magnetized electron-positron pair plasma (the paper's Bernstein-mode case shape).

    Mesh: jittered Delaunay of (n+1)^2 points, about 2 n^2 triangles, PEC walls
    (ny rows instead of n gives an n x ny strip; periodic_y joins its top and
    bottom walls, the paper's Bernstein geometry with PEC in place of PML).
    Side length set so the mean edge length is about one Debye length
    lambda_D ~ v_th/omega_p.  ppc particles per species per triangle, each
    electron collocated with a positron of opposite momentum (2-D
    Maxwell-Juttner, eta = 1/kT).  Superparticle weight gives the density
    n = omega_p^2 eps0 m / e^2 per unit depth.  dt = min(courant*h_min/c,
    0.05/omega_c).
    """
    b0 = 5.0
    wc = Q_E * b0 / M_E
    wp = wc / wc_over_wp
    vth = C_LIGHT * math.sqrt(kT)
    lam_d = vth / wp
    h = lam_d
    side = h * n_tri_side
    nyr = n_tri_side if ny is None else ny
    side_y = h * nyr
    mesh = jittered_delaunay(n_tri_side, nyr, side, side_y, 0.3, seed, periodic_y=periodic_y)
    rng = np.random.default_rng(seed + 1000)
    nf = len(mesh.triangles)
    tri_ids = np.repeat(np.arange(nf, dtype=np.int32), ppc)
    x = sample_in_triangles(mesh, tri_ids, rng)
    u = maxwell_juttner_2d(len(x), 1.0 / kT, rng)
    dens = wp * wp * EPS0 * M_E / (Q_E * Q_E)      # per m^3; per unit depth -> per m^2 * 1 m
    area = side * side_y
    weight = dens * area / len(x)
    e_sp = Species(-Q_E * weight, M_E * weight, x, u, tri_ids.copy())
    p_sp = Species(+Q_E * weight, M_E * weight, x.copy(), -u, tri_ids.copy())
    p = mesh.nodes
    t = mesh.triangles
    el = np.concatenate([np.linalg.norm(p[t[:, a]] - p[t[:, b]], axis=1)
                         for a, b in ((0, 1), (1, 2), (2, 0))])
    dt = min(courant * el.min() / C_LIGHT, 0.05 / wc)
    return Workload(f"pair-plasma-{nf}tri-{2*len(x)}p", mesh, [e_sp, p_sp], dt, b0=b0, pusher=pusher)


def high_gamma_beam(n_tri_side: int = 707, n_particles: int = 50_000_000, seed: int = 4,
                    pusher: str = "hc", side: float = 10.0) -> Workload:
    """Magnetized beam with gamma log-uniform in [10, 1000] drifting in crossed E_x, B_z.

    B_z = 1 T on the face DoFs, external uniform E_x = 0.5 c B_z so the E x B
    drift is 0.5 c along -y.  Positions uniform over the mesh.
    """
    mesh = jittered_delaunay(n_tri_side, n_tri_side, side, side, 0.3, seed)
    rng = np.random.default_rng(seed + 1000)
    nf = len(mesh.triangles)
    tri_ids = rng.integers(0, nf, n_particles).astype(np.int32)
    x = sample_in_triangles(mesh, tri_ids, rng)
    g = np.exp(rng.uniform(math.log(10.0), math.log(1000.0), n_particles))
    ux = C_LIGHT * np.sqrt(g * g - 1.0)
    u = np.stack([ux, np.zeros_like(ux)], 1)
    b0 = 1.0
    p = mesh.nodes
    t = mesh.triangles
    el = np.concatenate([np.linalg.norm(p[t[:, a]] - p[t[:, b]], axis=1)
                         for a, b in ((0, 1), (1, 2), (2, 0))])
    dt = 0.2 * el.min() / C_LIGHT
    sp = Species(-Q_E, M_E, x, u, tri_ids)
    return Workload(f"beam-{nf}tri-{n_particles}p", mesh, [sp], dt, b0=b0,
                    ext=(0.5 * C_LIGHT * b0, 0.0, 0.0), pusher=pusher)


def batched_pair_plasmas(n_inst: int = 64, seed: int = 5, f_range=(5_000, 200_000),
                         p_range=(10_000, 1_000_000), scale: float = 1.0) -> list:
    """Independent pair-plasma instances of uneven sizes (field-strength and temperature sweep).

    Triangle and particle counts log-uniform in the given ranges (times
    `scale`); omega_c/omega_p swept linearly in [0.25, 1], kT/mc^2 log-swept in
    [0.01, 0.3].
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_inst):
        f = int(math.exp(rng.uniform(math.log(f_range[0]), math.log(f_range[1]))) * scale)
        pcount = int(math.exp(rng.uniform(math.log(p_range[0]), math.log(p_range[1]))) * scale)
        side_n = max(4, int(round(math.sqrt(f / 2.0))))
        nf = 2 * side_n * side_n
        ppc = max(1, int(round(pcount / (2.0 * nf))))
        frac = k / max(1, n_inst - 1)
        wc_wp = 0.25 + 0.75 * frac
        kT = math.exp(math.log(0.01) + (math.log(0.3) - math.log(0.01)) * ((k * 37) % n_inst) / max(1, n_inst - 1))
        out.append(pair_plasma(side_n, ppc, kT, wc_wp, seed=seed * 1000 + k))
    return out


def synchrocyclotron(n: int = 100, v0: float = 1e7, radius: float = 0.02, e0: float = 2e5,
                     gap: float = 0.02, steps_per_turn: int = 2000, courant: float = 0.2) -> Workload:
    """The paper's synchrocyclotron case (Sec. III.A): a 1 m x 1 m square, B_z from the magnet
    everywhere (its poles cover the gap too) and an RF field E_x in a vertical gap strip
    |x - 0.5| < gap/2.

    B_z = m0 v0 / (|q| r) for an initial orbit radius r (2.84281e-3 T for v0 = 1e7 m/s, r = 0.02 m,
    as printed), E_x amplitude e0, one electron injected at (0.5 + r, 0.5) moving along +y
    (counter-clockwise about (0.5, 0.5)).  Structured mesh of n x n cells (jitter 0) so the gap
    edges are mesh lines; dt = min((2 pi / omega_c) / steps_per_turn, courant h_min / c), the second
    bound keeping the explicit field update stable.  The external E carries weight 1
    in the gap and 0 elsewhere, the external B weight 1 everywhere (Workload.ext_profile); the RF
    time dependence is an amplitude set every step (RFDrive)."""
    mesh = jittered_delaunay(n, n, 1.0, 1.0, 0.0, seed=0)
    t = mesh.triangles
    xc = mesh.nodes[t, 0].mean(axis=1)
    in_gap = np.abs(xc - 0.5) < 0.5 * gap
    profile = np.stack([in_gap, np.ones_like(in_gap)], axis=1).astype(np.float64)
    b0 = M_E * v0 / (Q_E * radius)
    wc = Q_E * b0 / M_E
    p = mesh.nodes
    el = np.concatenate([np.linalg.norm(p[t[:, a]] - p[t[:, b]], axis=1) for a, b in ((0, 1), (1, 2), (2, 0))])
    dt = min(2.0 * math.pi / wc / steps_per_turn, courant * el.min() / C_LIGHT)
    g = 1.0 / math.sqrt(1.0 - (v0 / C_LIGHT) ** 2)
    x = np.array([[0.5 + radius, 0.5]])
    u = np.array([[0.0, g * v0]])
    electron = Species(-Q_E, M_E, x, u, np.full(1, -1, np.int32))
    return Workload(f"synchrocyclotron-{len(t)}tri", mesh, [electron], dt, b0=0.0, ext=(e0, 0.0, b0),
                    pusher="boris", ext_profile=profile)


class RFDrive:
    """Phase of the synchrocyclotron's RF gap field, E_x = e0 sin(phi).  The electron (counter-
    clockwise in B_z > 0) crosses the gap moving -x at the top of its orbit a quarter turn after
    injection and +x at the bottom, so sin(phi) with phi(0) = 0 accelerates it at both crossings
    while the drive keeps pace.  Each step phi advances by omega dt: omega = omega_c / gamma
    (synchronized: the paper's f = qB / (2 pi gamma m0), gamma of the electron after the step) or
    the constant omega_c (f = 79.6 MHz for the printed field)."""

    def __init__(self, b0: float, dt: float, synchronized: bool):
        self.wc = Q_E * b0 / M_E
        self.dt = dt
        self.synchronized = synchronized
        self.phi = 0.0

    def amplitude(self) -> float:
        return math.sin(self.phi)

    def advance(self, u) -> None:
        u = np.asarray(u, np.float64).reshape(-1)
        gamma = math.sqrt(1.0 + (u[0] * u[0] + u[1] * u[1]) / (C_LIGHT * C_LIGHT))
        self.phi += (self.wc / gamma if self.synchronized else self.wc) * self.dt
