"""Python driver of the FP64 CPU oracle (fetdpic_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it; the library never imports it.  Array marshalling and
sparse assembly (scipy COO->CSR, transpose) live here; every step of the
method is in the C file, one function per equation of the paper.

What the oracle computes, in the paper's order (Sec. II):
  Faraday   b^{n+1/2} = b^{n-1/2} - dt C e^n                   Eq. (semi.dis.curl.1)
  gather    E^n, B^n = (B^{n+1/2}+B^{n-1/2})/2 at r^n            Sec. II.B, II.C(a)
  push      Boris / Boris-tan / Vay / Higuera-Cary               Sec. II.C
  move      r^{n+1} = r^n + dt u^{n+1/2}/gamma^{n+1/2}           Eq. (eq.motion.dis)
  deposit   i += (Q/dt)(l_a^s l_b^f - l_a^f l_b^s) per crossed
            triangle                                              Eq. (I.assign)
  Ampere    e^{n+1} = e^n + dt M (C^T [*mu^-1] b^{n+1/2} - i)    Eq. (semi.dis.curl.2)
with M the sparse approximate inverse of [*eps] (Sec. II.A).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fetdpic_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libfetdpic_oracle.so")

PUSHERS = {"boris": 0, "boris_tan": 1, "vay": 2, "hc": 3}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
                               "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.ora_spai_count.restype = C.c_longlong
        _lib.ora_push_only.restype = C.c_double
    return _lib


class _MeshC(C.Structure):
    _fields_ = [("nn", C.c_int), ("nf", C.c_int), ("ne", C.c_int),
                ("xy", C.c_void_p), ("tri", C.c_void_p), ("edge", C.c_void_p),
                ("tri_edge", C.c_void_p), ("tri_sign", C.c_void_p), ("tri_nb", C.c_void_p),
                ("edge_bnd", C.c_void_p), ("d2A", C.c_void_p), ("inv2A", C.c_void_p),
                ("gx", C.c_void_p), ("gy", C.c_void_p), ("nx_", C.c_void_p), ("ny_", C.c_void_p),
                ("rep", C.c_void_p), ("tri_shift", C.c_void_p), ("tx", C.c_double), ("ty", C.c_double)]


class _StepC(C.Structure):
    _fields_ = [("dt", C.c_double), ("c", C.c_double), ("q", C.c_double), ("m", C.c_double),
                ("ext_ex", C.c_double), ("ext_ey", C.c_double), ("ext_bz", C.c_double),
                ("pusher", C.c_int), ("max_cross", C.c_int), ("ext_w", C.c_void_p), ("ext_amp", C.c_double)]


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class OracleMesh:
    """Topology (incidence C, S~), orientation and Whitney geometry of a triangle mesh."""

    def __init__(self, nodes, triangles, periodic=None):
        """periodic = (pairs, (tx, ty)): pairs[k] = (node a, node b) with node b the image of node a
        one period (tx, ty) away; the two nodes become one, and so do the edges they bound."""
        self.xy = np.ascontiguousarray(nodes, np.float64)
        tri_in = np.ascontiguousarray(triangles, np.int32)
        nn, nf = len(self.xy), len(tri_in)
        self.rep = None
        self.tri_shift = None
        self.period = (0.0, 0.0)
        if periodic is not None:
            pairs, (tx, ty) = periodic
            pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
            rep = np.arange(nn, dtype=np.int32)
            span = float(np.abs(self.xy).max()) + abs(tx) + abs(ty)
            for a, b in pairs:
                if a == b or rep[b] != b or rep[a] != a:
                    raise ValueError("periodic pairs must join distinct nodes, each image once")
                d = self.xy[b] - self.xy[a] - (tx, ty)
                if np.abs(d).max() > 1e-9 * span:
                    raise ValueError(f"node {b} is not node {a} translated by the period")
                rep[b] = a
            self.rep = rep
            self.tri_shift = np.zeros((nf, 3), np.int32)
            self.period = (float(tx), float(ty))
        self.tri = np.zeros((nf, 3), np.int32)
        self.edge = np.zeros((3 * nf, 2), np.int32)
        self.tri_edge = np.zeros((nf, 3), np.int32)
        self.tri_sign = np.zeros((nf, 3), np.int32)
        self.tri_nb = np.zeros((nf, 3), np.int32)
        self.edge_bnd = np.zeros(3 * nf, np.int32)
        self.d2A = np.zeros(nf)
        self.inv2A = np.zeros(nf)
        self.gx = np.zeros((nf, 3))
        self.gy = np.zeros((nf, 3))
        self.nx = np.zeros((nf, 3))
        self.ny = np.zeros((nf, 3))
        s = _MeshC(nn, nf, 0, _p(self.xy), _p(self.tri), _p(self.edge), _p(self.tri_edge),
                   _p(self.tri_sign), _p(self.tri_nb), _p(self.edge_bnd), _p(self.d2A),
                   _p(self.inv2A), _p(self.gx), _p(self.gy), _p(self.nx), _p(self.ny),
                   None if self.rep is None else _p(self.rep),
                   None if self.tri_shift is None else _p(self.tri_shift),
                   self.period[0], self.period[1])
        ne = lib().ora_mesh_build(C.byref(s), _p(tri_in))
        if ne < 0:
            raise ValueError(f"oracle: invalid mesh (status {ne})")
        self.edge = self.edge[:ne].copy()
        self.edge_bnd = self.edge_bnd[:ne].copy()
        self.nn, self.nf, self.ne = nn, nf, ne
        self._s = s
        self._s.edge = _p(self.edge).value
        self._s.edge_bnd = _p(self.edge_bnd).value
        self._s.ne = ne
        self.free = np.nonzero(self.edge_bnd == 0)[0].astype(np.int32)

    @property
    def cs(self):
        return C.byref(self._s)

    def edge_vectors(self) -> np.ndarray:
        """r_j - r_i of every edge (i -> j), read off a triangle that holds it (with periodic walls
        the two nodes of an edge may be stored one period apart)."""
        v = np.zeros((self.ne, 2))
        for m in range(3):
            a, b = (m + 1) % 3, (m + 2) % 3
            d = np.stack([self.nx[:, b] - self.nx[:, a], self.ny[:, b] - self.ny[:, a]], axis=1)
            v[self.tri_edge[:, m]] = d * self.tri_sign[:, m, None]
        return v

    def curl(self) -> sp.csr_matrix:
        """C (faces x edges), entries in {-1,0,1}."""
        r = np.repeat(np.arange(self.nf), 3)
        return sp.csr_matrix((self.tri_sign.ravel().astype(np.float64), (r, self.tri_edge.ravel())),
                             shape=(self.nf, self.ne))

    def div_dual(self) -> sp.csr_matrix:
        """S~ (nodes x edges): +1 where the edge leaves the node, -1 where it enters."""
        e = np.arange(self.ne)
        rows = np.concatenate([self.edge[:, 0], self.edge[:, 1]])
        cols = np.concatenate([e, e])
        vals = np.concatenate([np.ones(self.ne), -np.ones(self.ne)])
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.nn, self.ne))

    def lambdas(self, cell, x, y):
        cell = np.ascontiguousarray(cell, np.int32)
        x = np.ascontiguousarray(x, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        lam = np.zeros((len(cell), 3))
        lib().ora_lambdas(self.cs, len(cell), _p(cell), _p(x), _p(y), _p(lam))
        return lam

    def locate(self, x, y, hint=None):
        x = np.ascontiguousarray(x, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        cell = np.zeros(len(x), np.int32)
        h = None if hint is None else np.ascontiguousarray(hint, np.int32)
        bad = lib().ora_locate(self.cs, len(x), _p(x), _p(y), None if h is None else _p(h), _p(cell))
        return cell, bad

    def field_at(self, e, x, y, cell=None):
        """E (n x 2) of the edge unknowns e at points (x, y), by the Whitney 1-form interpolation
        of the particle gather (Sec. II.B); cell = the triangles holding the points (located
        here when None)."""
        x = np.ascontiguousarray(x, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        if cell is None:
            cell, bad = self.locate(x, y)
            if bad:
                raise ValueError(f"{bad} points outside the mesh")
        cell = np.ascontiguousarray(cell, np.int32)
        e = np.ascontiguousarray(e, np.float64)
        out = np.zeros((len(x), 2))
        lib().ora_field_at(self.cs, _p(e), len(x), _p(cell), _p(x), _p(y), _p(out))
        return out

    def hodge_eps(self, eps0: float) -> sp.csr_matrix:
        """[*eps] over all edges (Galerkin edge mass matrix)."""
        el = np.zeros((self.nf, 3, 3))
        lib().ora_hodge_eps_elements(self.cs, C.c_double(eps0), _p(el))
        r = np.repeat(self.tri_edge, 3, axis=1).ravel()
        c = np.tile(self.tri_edge, (1, 3)).ravel()
        return sp.coo_matrix((el.ravel(), (r, c)), shape=(self.ne, self.ne)).tocsr()

    def hodge_mu_inv(self, mu0: float) -> np.ndarray:
        """Diagonal of [*mu^-1]: 1/(mu0 A_f)."""
        return 1.0 / (mu0 * (0.5 * self.d2A))


def spai(A: sp.csr_matrix, k: int) -> sp.csr_matrix:
    """Level-k sparse approximate inverse of a symmetric matrix, symmetrised."""
    A = sp.csr_matrix(A)
    A.sort_indices()
    n = A.shape[0]
    rp = np.ascontiguousarray(A.indptr, np.int32)
    ci = np.ascontiguousarray(A.indices, np.int32)
    v = np.ascontiguousarray(A.data, np.float64)
    nnz = lib().ora_spai_count(n, _p(rp), _p(ci), k)
    colptr = np.zeros(n + 1, np.int64)
    rows = np.zeros(nnz, np.int32)
    vals = np.zeros(nnz)
    st = lib().ora_spai(n, _p(rp), _p(ci), _p(v), k, _p(colptr), _p(rows), _p(vals))
    if st != 0:
        raise ValueError("oracle SPAI: rank-deficient column")
    Mcsc = sp.csc_matrix((vals, rows, colptr), shape=(n, n))
    return sp.csr_matrix(0.5 * (Mcsc + Mcsc.T))


class OracleSim:
    """One FETD-PIC instance advanced by the oracle, FP64 throughout.

    State: e^n (edges), b^{n-1/2} (faces), d^n = dual flux (edges), particles
    per species (x, y, u_x, u_y, u_z, cell).  Loaded u is u^{-1/2}; b^{-1/2}
    and e^0 come from the uniform initial fields.
    """

    def __init__(self, nodes, triangles, dt, *, eps0, mu0, c, spai_level=2, exact_inverse=False,
                 b0=0.0, e0=(0.0, 0.0), ext=(0.0, 0.0, 0.0), max_cross=64, fields=True, periodic=None):
        """fields=False skips [*eps] and the SPAI (particle-only steps on large meshes);
        periodic: as for OracleMesh."""
        self.mesh = m = OracleMesh(nodes, triangles, periodic)
        self.dt, self.eps0, self.mu0, self.c = dt, eps0, mu0, c
        self.ext = tuple(float(v) for v in ext)
        self.max_cross = max_cross
        self.has_fields = fields
        if fields:
            self.star_eps = m.hodge_eps(eps0)
            Af = self.star_eps[m.free][:, m.free].tocsr()
            if exact_inverse:
                Minv = sp.csr_matrix(np.linalg.inv(Af.toarray()))
            else:
                Minv = spai(Af, spai_level)
        else:
            self.star_eps = sp.csr_matrix((m.ne, m.ne))
            Minv = sp.csr_matrix((len(m.free), len(m.free)))
        Minv.sort_indices()
        self.Minv = Minv
        self._rp = np.ascontiguousarray(Minv.indptr, np.int64)
        self._ci = np.ascontiguousarray(Minv.indices, np.int32)
        self._v = np.ascontiguousarray(Minv.data, np.float64)
        # uniform initial fields: b_f = B0 A_f (flux), e_k = E0 . (r_j - r_i) on free edges
        self.b = b0 * (0.5 * m.d2A)
        t = m.edge_vectors()
        self.e = (e0[0] * t[:, 0] + e0[1] * t[:, 1]) * (m.edge_bnd == 0)
        self.d = self.star_eps @ self.e
        self.i = np.zeros(m.ne)
        self.i_abs = np.zeros(m.ne)
        self.b_half = self.b.copy()    # b^{n+1/2} of the last step
        self.species = []
        self.step_count = 0
        # applied fields varying in space and time: per-triangle weights (E, B) of ext and an
        # amplitude multiplying the external E (None = weights 1)
        self.ext_profile = None
        self.ext_amp = 1.0

    def load(self, q, m_, x, u, hint=None, cell=None):
        """Add a species; `cell` (if given) is taken as the host triangle of each point as is."""
        x = np.asarray(x, np.float64)
        u = np.asarray(u, np.float64)
        if cell is None:
            cell, bad = self.mesh.locate(x[:, 0], x[:, 1], hint)
            if bad:
                raise ValueError(f"oracle: {bad} particles outside the mesh")
        else:
            cell = np.ascontiguousarray(cell, np.int32).copy()
        self.species.append(dict(q=float(q), m=float(m_), x=x[:, 0].copy(), y=x[:, 1].copy(),
                                 ux=u[:, 0].copy(), uy=u[:, 1].copy(), uz=np.zeros(len(x)),
                                 cell=cell))
        return cell

    def charge(self) -> np.ndarray:
        q = np.zeros(self.mesh.nn)
        for s in self.species:
            n = len(s["x"])
            lib().ora_charge(self.mesh.cs, C.c_double(s["q"]), n, _p(s["x"]), _p(s["y"]),
                             _p(s["cell"]), _p(q))
        return q

    def step(self, pusher="boris", record=0, only_particles=False):
        """One leapfrog step; returns the per-species walk records if record > 0."""
        m = self.mesh
        pid = PUSHERS[pusher] if isinstance(pusher, str) else int(pusher)
        b_new = np.zeros(m.nf)
        lib().ora_faraday(m.cs, C.c_double(self.dt), _p(self.e), _p(self.b), _p(b_new))
        self.i = np.zeros(m.ne)
        self.i_abs = np.zeros(m.ne)
        recs = []
        status = 0
        for s in self.species:
            n = len(s["x"])
            prof = None if self.ext_profile is None else np.ascontiguousarray(self.ext_profile, np.float64)
            P = _StepC(self.dt, self.c, s["q"], s["m"], self.ext[0], self.ext[1], self.ext[2], pid,
                       self.max_cross, None if prof is None else _p(prof), float(self.ext_amp))
            cnt = np.zeros(n, np.int32) if record else None
            rec = np.full((n, max(record, 1)), -(1 << 30), np.int32) if record else None
            st = lib().ora_particles(m.cs, C.byref(P), _p(self.e), _p(self.b), _p(b_new), n,
                                     _p(s["x"]), _p(s["y"]), _p(s["ux"]), _p(s["uy"]), _p(s["uz"]),
                                     _p(s["cell"]), _p(self.i), _p(self.i_abs), record,
                                     None if cnt is None else _p(cnt),
                                     None if rec is None else _p(rec))
            status = status or st
            recs.append((cnt, rec))
        if not only_particles:
            if not self.has_fields:
                raise ValueError("oracle built with fields=False: particle-only steps")
            r = np.zeros(m.ne)
            lib().ora_curl_h(m.cs, C.c_double(self.mu0), _p(b_new), _p(self.i), _p(r))
            lib().ora_ampere(len(m.free), _p(m.free), _p(self._rp), _p(self._ci), _p(self._v),
                             C.c_double(self.dt), _p(r), _p(self.e), _p(self.d), m.ne)
        self.b_half = b_new
        self.b = b_new
        self.step_count += 1
        self.status = status
        return recs

    def electrostatic_solve(self):
        """Initial electrostatic field of the loaded charge (Gauss law, Eq. (semi.dis.div.2), with
        e = -G phi): [*eps] restricted to free edges, G the node-to-edge gradient incidence
        (G = -S~^T), phi = 0 on nodes of PEC edges; solves G^T [*eps] G phi = q on the other nodes
        and adds e = -G phi to the edge unknowns; d = [*eps] e.  Returns phi."""
        m = self.mesh
        G = -m.div_dual().T.tocsr()                       # edges x nodes: +1 at the head, -1 at the tail
        pec_nodes = np.unique(m.edge[m.edge_bnd == 1])
        has_edge = np.zeros(m.nn, bool)
        has_edge[m.edge.ravel()] = True
        free_n = np.setdiff1d(np.nonzero(has_edge)[0], pec_nodes)
        free_e = m.edge_bnd == 0
        Gf = G[free_e][:, free_n]
        Ef = self.star_eps[free_e][:, free_e]
        K = (Gf.T @ Ef @ Gf).tocsc()
        q = self.charge()
        phi = np.zeros(m.nn)
        phi[free_n] = spla.spsolve(K, q[free_n])
        de = -(G @ phi)
        de[~free_e] = 0.0
        self.e = self.e + de
        self.d = self.star_eps @ self.e
        return phi

    def field_energy(self) -> float:
        """eps-energy e.[*eps].e/2 + mu-energy b.[*mu^-1].b/2 (FP64)."""
        h = self.mesh.hodge_mu_inv(self.mu0)
        return 0.5 * float(self.e @ (self.star_eps @ self.e)) + 0.5 * float(self.b @ (h * self.b))


def push_only(pusher, alpha, c, E, B, u):
    """Single velocity update (no mesh), for the closed-form pusher pins."""
    E = np.ascontiguousarray(E, np.float64)
    B = np.ascontiguousarray(B, np.float64)
    u = np.ascontiguousarray(u, np.float64).copy()
    g = lib().ora_push_only(PUSHERS[pusher], C.c_double(alpha), C.c_double(c), _p(E), _p(B), _p(u))
    return u, g
