"""ctypes binding of the fetdpic C ABI (include/fetdpic.h).

Argument marshalling only: every step of the method runs in libfetdpic.so
(sm_103a kernels).  There is no CPU fallback: importing this module raises if
the library has not been built (python -m paper_1707_04333_gb300.build_lib).

Function names match the C ABI.  `Simulation` wraps a context for the common
case of one workload from `inputs`.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import build_lib

OK, EINVAL, ENOMEM, ECUDA, EMESH, EWALK, EOUTSIDE, ENONFINITE, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
PUSHERS = {"boris": 0, "boris_tan": 1, "vay": 2, "hc": 3}
FP64, FP32 = 0, 1

_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Params(C.Structure):
    _fields_ = [("eps0", C.c_double), ("mu0", C.c_double), ("c", C.c_double),
                ("precision", C.c_int), ("spai_level", C.c_int), ("sort_interval", C.c_int),
                ("max_crossings", C.c_int), ("check_interval", C.c_int), ("record_walk", C.c_int),
                ("block_size", C.c_int), ("use_graphs", C.c_int), ("time_stages", C.c_int), ("kernel_variant", C.c_int),
                ("cuda_stream", C.c_void_p),
                ("dev_alloc", _ALLOC), ("dev_free", _FREE), ("alloc_user", C.c_void_p),
                ("wait_spin_limit", C.c_longlong), ("fuse_field_update", C.c_int)]


class Instance(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("nodes_xy", C.c_void_p), ("n_tri", C.c_int),
                ("triangles", C.c_void_p), ("n_edges", C.c_int), ("edges", C.c_void_p),
                ("edge_tags", C.c_void_p), ("dt", C.c_double), ("b0", C.c_double),
                ("e0x", C.c_double), ("e0y", C.c_double), ("ext_ex", C.c_double),
                ("ext_ey", C.c_double), ("ext_bz", C.c_double), ("n_periodic", C.c_int),
                ("periodic_nodes", C.c_void_p), ("period_x", C.c_double), ("period_y", C.c_double)]


class FetdpicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fetdpic error {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return build_lib.LIB


def lib():
    """Load libfetdpic.so (built in-tree).  Raises when it is missing."""
    global _lib
    if _lib is None:
        path = build_lib.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libfetdpic.so is not built ({path}); run the build first")
        L = C.CDLL(path)
        vp, i32, i64, dp = C.c_void_p, C.c_int, C.c_longlong, C.c_double
        sig = {
            "fetdpic_create": (i32, [C.POINTER(vp), C.POINTER(Params), i32, vp]),
            "fetdpic_load_particles": (i32, [vp, i32, dp, dp, i64, vp, vp, vp]),
            "fetdpic_write_particles": (i32, [vp, i32, vp, vp, vp]),
            "fetdpic_write_fields": (i32, [vp, i32, vp, vp]),
            "fetdpic_step": (i32, [vp, i64, i32]),
            "fetdpic_sync": (i32, [vp]),
            "fetdpic_read": (i32, [vp, i32, vp, vp, vp, i32, vp, vp, vp]),
            "fetdpic_read_walk": (i32, [vp, i32, vp, vp]),
            "fetdpic_read_charge": (i32, [vp, i32, vp, vp]),
            "fetdpic_read_particles_static": (i32, [vp, i32, vp, vp, vp]),
            "fetdpic_read_particles_async": (i32, [vp, i32, vp, vp, vp]),
            "fetdpic_check": (i32, [vp, i32, vp, vp, vp]),
            "fetdpic_info": (i32, [vp, i32, vp]),
            "fetdpic_read_edges": (i32, [vp, i32, vp]),
            "fetdpic_set_probes": (i32, [vp, i64, vp, vp, i64]),
            "fetdpic_solve_electrostatic": (i32, [vp, i32, vp, vp]),
            "fetdpic_set_external_profile": (i32, [vp, i32, vp]),
            "fetdpic_set_external_amplitude": (i32, [vp, i32, dp]),
            "fetdpic_read_probes": (i32, [vp, vp, i64, vp, vp]),
            "fetdpic_read_spai": (i32, [vp, i32, vp, vp, vp, vp]),
            "fetdpic_stage_times": (i32, [vp, vp, vp]),
            "fetdpic_autotune": (i32, [vp, i32, i32, vp, vp]),
            "fetdpic_set_tuning": (i32, [vp, i32, i32]),
            "fetdpic_set_wait_limit": (i32, [vp, i64]),
            "fetdpic_particle_bytes": (i32, [vp, vp, vp]),
            "fetdpic_fma_rate": (i32, [i32, vp]),
            "fetdpic_last_error": (C.c_char_p, [vp]),
            "fetdpic_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def declared_symbols() -> list:
    """Every function the public header declares."""
    hdr = os.path.join(build_lib.INCLUDE, "fetdpic.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"\b(fetdpic_[a-z_0-9]+)\s*\(", txt)))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(ctx, rc):
    if rc < 0:
        msg = lib().fetdpic_last_error(ctx)
        raise FetdpicError(rc, msg.decode() if msg else "")
    return rc


# ---------------------------------------------------------------- raw ABI

def fetdpic_create(params: Params, instances: list):
    arr = (Instance * len(instances))(*instances)
    h = C.c_void_p()
    rc = lib().fetdpic_create(C.byref(h), C.byref(params), len(instances), C.cast(arr, C.c_void_p))
    if rc < 0:
        raise FetdpicError(rc, "fetdpic_create failed")
    return h


def fetdpic_load_particles(h, inst, q, m, x, u, hint=None):
    x = np.ascontiguousarray(x, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    hint = None if hint is None else np.ascontiguousarray(hint, np.int32)
    return _check(h, lib().fetdpic_load_particles(h, inst, q, m, len(x), _ptr(x), _ptr(u), _ptr(hint)))


def fetdpic_write_particles(h, species, x, u, cell=None):
    x = np.ascontiguousarray(x, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    cell = None if cell is None else np.ascontiguousarray(cell, np.int32)
    return _check(h, lib().fetdpic_write_particles(h, species, _ptr(x), _ptr(u), _ptr(cell)))


def fetdpic_write_fields(h, inst, e=None, b=None):
    e = None if e is None else np.ascontiguousarray(e, np.float64)
    b = None if b is None else np.ascontiguousarray(b, np.float64)
    return _check(h, lib().fetdpic_write_fields(h, inst, _ptr(e), _ptr(b)))


def fetdpic_step(h, nsteps, pusher):
    p = PUSHERS[pusher] if isinstance(pusher, str) else int(pusher)
    return _check(h, lib().fetdpic_step(h, int(nsteps), p))


def fetdpic_sync(h):
    return _check(h, lib().fetdpic_sync(h))


def fetdpic_info(h, inst=0):
    out = np.zeros(6, np.int64)
    _check(h, lib().fetdpic_info(h, inst, _ptr(out)))
    return dict(n_nodes=int(out[0]), n_edges=int(out[1]), n_tri=int(out[2]), n_free=int(out[3]),
                spai_nnz=int(out[4]), n_particles=int(out[5]))


def fetdpic_read(h, inst=0, species=None, fields=True, n=None):
    info = fetdpic_info(h, inst)
    out = {}
    e = b = j = None
    if fields:
        e = np.zeros(info["n_edges"])
        b = np.zeros(info["n_tri"])
        j = np.zeros(info["n_edges"])
    x = u = cell = None
    if species is not None:
        x = np.zeros((n, 2))
        u = np.zeros((n, 2))
        cell = np.zeros(n, np.int32)
    _check(h, lib().fetdpic_read(h, inst, _ptr(e), _ptr(b), _ptr(j), -1 if species is None else species,
                                 _ptr(x), _ptr(u), _ptr(cell)))
    if fields:
        out.update(e=e, b=b, j=j)
    if species is not None:
        out.update(x=x, u=u, cell=cell)
    return out


def fetdpic_read_particles_async(h, species, x=None, u=None, cell=None):
    """Enqueue the load-order read of one species into the given host arrays (x [n][2], u [n][2]
    float64, cell [n] int32, C-contiguous; page-locked for full speed).  The arrays are filled when
    fetdpic_sync returns and must be kept alive and untouched until then."""
    for a, dt in ((x, np.float64), (u, np.float64), (cell, np.int32)):
        if a is not None and (a.dtype != dt or not a.flags["C_CONTIGUOUS"]):
            raise ValueError("fetdpic_read_particles_async: arrays must be C-contiguous float64 / int32")
    _check(h, lib().fetdpic_read_particles_async(h, species, _ptr(x), _ptr(u), _ptr(cell)))


def fetdpic_read_walk(h, species, n, cap):
    cnt = np.zeros(n, np.int32)
    rec = np.zeros((n, cap), np.int32)
    _check(h, lib().fetdpic_read_walk(h, species, _ptr(cnt), _ptr(rec)))
    return cnt, rec


def fetdpic_read_charge(h, inst=0):
    """(nodal charge [n_nodes] of the current particle state, fixed-point quantum)."""
    info = fetdpic_info(h, inst)
    q = np.zeros(info["n_nodes"])
    qu = C.c_double()
    _check(h, lib().fetdpic_read_charge(h, inst, _ptr(q), C.byref(qu)))
    return q, qu.value


def fetdpic_check(h, inst=0):
    v = (C.c_double * 3)()
    _check(h, lib().fetdpic_check(h, inst, C.byref(v, 0), C.byref(v, 8), C.byref(v, 16)))
    return dict(dce=v[0], dgl=v[1], energy=v[2])


def fetdpic_read_edges(h, inst=0):
    info = fetdpic_info(h, inst)
    ed = np.zeros((info["n_edges"], 2), np.int32)
    _check(h, lib().fetdpic_read_edges(h, inst, _ptr(ed)))
    return ed


def fetdpic_set_probes(h, xy, inst=None, capacity=4096):
    """Field probes at points xy (n x 2, metres) of instances inst (default 0), recording the last
    `capacity` steps on the device."""
    xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
    n = len(xy)
    inst = np.zeros(n, np.int32) if inst is None else np.ascontiguousarray(inst, np.int32)
    _check(h, lib().fetdpic_set_probes(h, n, _ptr(inst), _ptr(xy), capacity))


def fetdpic_read_probes(h, n, max_rows):
    """(exy [rows][n][2] oldest first, total steps recorded)."""
    out = np.zeros((max_rows, n, 2))
    rows, total = C.c_longlong(), C.c_longlong()
    _check(h, lib().fetdpic_read_probes(h, _ptr(out), max_rows, C.byref(rows), C.byref(total)))
    return out[:rows.value], total.value


def fetdpic_read_spai(h, inst=0):
    info = fetdpic_info(h, inst)
    rp = np.zeros(info["n_free"] + 1, np.int64)
    re_ = np.zeros(info["n_free"], np.int32)
    ci = np.zeros(info["spai_nnz"], np.int32)
    v = np.zeros(info["spai_nnz"])
    _check(h, lib().fetdpic_read_spai(h, inst, _ptr(rp), _ptr(re_), _ptr(ci), _ptr(v)))
    return rp, re_, ci, v


def fetdpic_stage_times(h):
    out = np.zeros(6)
    n = C.c_longlong()
    _check(h, lib().fetdpic_stage_times(h, _ptr(out), C.byref(n)))
    return out, n.value


def fetdpic_autotune(h, pusher, trial_steps=32):
    p = PUSHERS[pusher] if isinstance(pusher, str) else int(pusher)
    v = C.c_int()
    s = C.c_int()
    _check(h, lib().fetdpic_autotune(h, p, trial_steps, C.byref(v), C.byref(s)))
    return v.value, s.value


def fetdpic_set_tuning(h, variant, sort_interval):
    return _check(h, lib().fetdpic_set_tuning(h, variant, sort_interval))


def fetdpic_set_wait_limit(h, limit):
    return _check(h, lib().fetdpic_set_wait_limit(h, int(limit)))


def fetdpic_particle_bytes(h):
    b = C.c_double()
    n = C.c_longlong()
    _check(h, lib().fetdpic_particle_bytes(h, C.byref(b), C.byref(n)))
    return b.value, n.value


def fetdpic_fma_rate(fp64: bool) -> float:
    """Measured FMA rate of the current device in TFLOP/s (FP64 or FP32)."""
    t = C.c_double()
    _check(None, lib().fetdpic_fma_rate(1 if fp64 else 0, C.byref(t)))
    return t.value


def fetdpic_destroy(h):
    if h:
        lib().fetdpic_destroy(h)


# ------------------------------------------------------------ convenience

def _torch_allocator():
    """Device allocation through PyTorch's caching allocator (plumbing only)."""
    import torch
    dev = torch.cuda.current_device()

    @_ALLOC
    def alloc(nbytes, user):
        return torch.cuda.caching_allocator_alloc(int(nbytes), dev)

    @_FREE
    def free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    return alloc, free


class Simulation:
    """A context built from one or more `inputs.Workload`s (batched when several)."""

    def __init__(self, workloads, precision="fp64", spai_level=2, sort_interval=16, max_crossings=64,
                 record_walk=0, block_size=0, check_interval=0, use_torch=True, stream=None,
                 edges=None, edge_tags=None, time_stages=False, kernel_variant=0, use_graphs=False,
                 wait_spin_limit=0, fuse_field_update=False):
        if not isinstance(workloads, (list, tuple)):
            workloads = [workloads]
        self.workloads = list(workloads)
        self._keep = []
        p = Params()
        p.precision = FP32 if precision == "fp32" else FP64
        p.spai_level = spai_level
        p.sort_interval = sort_interval
        p.max_crossings = max_crossings
        p.record_walk = record_walk
        p.block_size = block_size
        p.check_interval = check_interval
        p.time_stages = 1 if time_stages else 0
        p.kernel_variant = kernel_variant
        p.use_graphs = 1 if use_graphs else 0
        p.wait_spin_limit = wait_spin_limit
        p.fuse_field_update = 1 if fuse_field_update else 0
        self.stream = None
        if use_torch:
            import torch
            if stream is None:
                stream = torch.cuda.current_stream()
            if stream.cuda_stream == 0:
                # the legacy default stream has handle 0, which the C ABI reads as "make a private
                # stream"; give the context an explicit stream that torch events can bracket
                stream = torch.cuda.Stream()
            self.stream = stream
            p.cuda_stream = C.c_void_p(stream.cuda_stream)
            a, f = _torch_allocator()
            p.dev_alloc, p.dev_free = a, f
            self._keep += [a, f]
        insts = []
        for k, w in enumerate(self.workloads):
            nodes = np.ascontiguousarray(w.mesh.nodes, np.float64)
            tris = np.ascontiguousarray(w.mesh.triangles, np.int32)
            self._keep += [nodes, tris]
            I = Instance()
            I.n_nodes, I.nodes_xy = len(nodes), _ptr(nodes)
            I.n_tri, I.triangles = len(tris), _ptr(tris)
            if edges is not None:
                ed = np.ascontiguousarray(edges[k], np.int32)
                self._keep.append(ed)
                I.n_edges, I.edges = len(ed), _ptr(ed)
            if edge_tags is not None:
                tg = np.ascontiguousarray(edge_tags[k], np.int32)
                self._keep.append(tg)
                I.edge_tags = _ptr(tg)
            I.dt, I.b0 = w.dt, w.b0
            I.e0x, I.e0y = w.e0
            I.ext_ex, I.ext_ey, I.ext_bz = w.ext
            per = getattr(w.mesh, "periodic", None)
            if per is not None:
                pairs = np.ascontiguousarray(per[0], np.int32).reshape(-1, 2)
                self._keep.append(pairs)
                I.n_periodic, I.periodic_nodes = len(pairs), _ptr(pairs)
                I.period_x, I.period_y = float(per[1][0]), float(per[1][1])
            insts.append(I)
        self.params = p
        self.h = fetdpic_create(p, insts)
        for k, w in enumerate(self.workloads):
            if getattr(w, "ext_profile", None) is not None:
                self.set_external_profile(w.ext_profile, k)
        self.species = []          # (instance, species id, n)
        self.record_walk = record_walk

    def load(self, inst_index=None, hints=True):
        for k, w in enumerate(self.workloads):
            if inst_index is not None and k != inst_index:
                continue
            for s in w.species:
                sid = fetdpic_load_particles(self.h, k, s.q, s.m, s.x, s.u, s.hint if hints else None)
                self.species.append((k, sid, len(s.x)))
        return self

    def step(self, n=1, pusher=None):
        pusher = pusher or self.workloads[0].pusher
        fetdpic_step(self.h, n, pusher)
        return self

    def sync(self):
        fetdpic_sync(self.h)
        return self

    def autotune(self, pusher=None, trial_steps=32, cache=None):
        """Pick the particle-kernel variant and sort interval by timing trials (state restored),
        or reuse a choice cached in the JSON file `cache` under (GPU, workload shape, precision,
        pusher).  Returns (variant, sort_interval)."""
        import json
        import torch
        pusher = pusher or self.workloads[0].pusher
        key = "|".join([torch.cuda.get_device_name(), self.workloads_signature(), str(self.params.precision),
                        pusher])
        table = {}
        if cache and os.path.exists(cache):
            try:
                table = json.load(open(cache))
            except (OSError, ValueError):
                table = {}
        if key in table:
            v, s = table[key]
            fetdpic_set_tuning(self.h, v, s)
            return v, s
        v, s = fetdpic_autotune(self.h, pusher, trial_steps)
        if cache:
            table[key] = [v, s]
            tmp = cache + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return v, s

    def workloads_signature(self):
        tri = sum(len(w.mesh.triangles) for w in self.workloads)
        par = sum(w.n_particles for w in self.workloads)
        return f"{len(self.workloads)}inst-{tri}tri-{par}p"

    def read_species(self, sid):
        k, _, n = self.species[sid]
        return fetdpic_read(self.h, k, species=sid, fields=False, n=n)

    def read_fields(self, inst=0):
        return fetdpic_read(self.h, inst, species=None, fields=True)

    def set_external_profile(self, w, inst=0):
        """Per-triangle weights (E, B) [n_tri][2] of the instance's applied fields (None = 1)."""
        if w is None:
            _check(self.h, lib().fetdpic_set_external_profile(self.h, inst, None))
            return self
        w = np.ascontiguousarray(w, np.float64).reshape(-1, 2)
        _check(self.h, lib().fetdpic_set_external_profile(self.h, inst, _ptr(w)))
        return self

    def set_external_amplitude(self, a, inst=0):
        _check(self.h, lib().fetdpic_set_external_amplitude(self.h, inst, float(a)))
        return self

    def solve_electrostatic(self, inst=0):
        """Initial field of the loaded charge (before the first step): (CG iterations, residual)."""
        it, res = C.c_int(), C.c_double()
        _check(self.h, lib().fetdpic_solve_electrostatic(self.h, inst, C.byref(it), C.byref(res)))
        return it.value, res.value

    def set_probes(self, xy, inst=None, capacity=4096):
        fetdpic_set_probes(self.h, xy, inst, capacity)
        self._probe_n, self._probe_cap = len(np.asarray(xy).reshape(-1, 2)), capacity
        return self

    def read_probes(self, max_rows=None):
        """E at the probes for the recorded steps, oldest first: (rows x n x 2, total steps)."""
        return fetdpic_read_probes(self.h, self._probe_n, max_rows or self._probe_cap)

    def close(self):
        if self.h:
            fetdpic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
