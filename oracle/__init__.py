"""Python access to the CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use
this package.  It wraps ``pdfx_oracle.c`` (plain FP64 C, one thread) through ctypes and
shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdfx_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

NF = 32
NS = 13


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    deps = [_SRC, os.path.join(_HERE, "pdfx_oracle.h")]
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(d) for d in deps)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-Wall", "-shared", "-fPIC",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("C1", "C2", "C3", "C4", "CT", "CL", "Ceta", "Cv", "gamma5", "Cw1", "Cw2", "nu")] + [
        ("c0_mode", C.c_int), ("C0", C.c_double),
        ("tm_mode", C.c_int), ("Cs", C.c_double), ("Ct", C.c_double), ("Cphi", C.c_double),
        ("src_x", C.c_double), ("src_y", C.c_double), ("src_r", C.c_double),
        ("bins", C.c_int * 3), ("min_per_bin", C.c_int), ("minnpel", C.c_int),
        ("interp_mode", C.c_int), ("source_on", C.c_int),
        ("seed", C.c_uint64), ("instance", C.c_uint32), ("period_x", C.c_double),
        ("cond_mode", C.c_int), ("fox_bins", C.c_int), ("model", C.c_int), ("alpha", C.c_double),
        ("cfl", C.c_double),
    ]


class Diag(C.Structure):
    _fields_ = [(n, C.c_longlong) for n in
                ("hops_total", "walk_fallback", "walk_brute", "lost", "wall_hits", "wall_hits_a",
                 "freeslip_hits", "omega_reflect", "c0_clamp", "gamma_exhausted", "moves",
                 "source_hits")] + [("hop_hist", C.c_longlong * 8)]


_DEFAULTS = dict(C1=1.85, C2=0.63, C3=5.0, C4=0.25, CT=6.0, CL=0.134, Ceta=72.0, Cv=1.4,
                 gamma5=0.1, Cw1=0.5, Cw2=0.73, nu=1e-4, c0_mode=0, C0=0.0, tm_mode=0,
                 Cs=0.02, Ct=0.7, Cphi=2.0, src_x=0.5, src_y=0.5, src_r=0.02, bins=(4, 4, 4),
                 min_per_bin=2, minnpel=0, interp_mode=0, source_on=1, seed=1, instance=0,
                 period_x=0.0, cond_mode=0, fox_bins=5, model=0, alpha=0.5, cfl=0.7)


def make_params(d: dict) -> Params:
    full = dict(_DEFAULTS)
    full.update({k: v for k, v in d.items() if k in _DEFAULTS})
    p = Params()
    for k, v in full.items():
        if k == "bins":
            p.bins = (C.c_int * 3)(*[int(b) for b in v])
        else:
            setattr(p, k, v)
    return p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int32)
            u32p = C.POINTER(C.c_uint32)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_uniform.restype = C.c_double
            L.orc_uniform.argtypes = [C.c_uint32]
            L.orc_box_muller.argtypes = [C.c_uint32, C.c_uint32, dp, dp]
            L.orc_gamma_draw.restype = C.c_double
            L.orc_gamma_draw.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                         C.c_uint32, C.c_double, C.c_double, C.POINTER(C.c_int)]
            L.orc_step_gaussians.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, dp, dp]
            L.orc_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(Params), C.c_int, dp,
                                     C.c_int, ip, C.POINTER(C.c_int8)]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_set_params.argtypes = [C.c_void_p, C.POINTER(Params)]
            L.orc_set_fields.argtypes = [C.c_void_p, dp]
            L.orc_lambda.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, dp]
            L.orc_walk.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_int)]
            L.orc_brute_locate.argtypes = [C.c_void_p, C.c_double, C.c_double]
            L.orc_interp.argtypes = [C.c_void_p, C.c_int, dp, dp]
            L.orc_neighbors.argtypes = [C.c_void_p, ip]
            L.orc_init_particles.argtypes = [C.c_void_p, C.c_int]
            L.orc_init_elements.argtypes = [C.c_void_p, C.c_int, C.c_int, ip]
            L.orc_set_particles_ids.argtypes = ([C.c_void_p, C.c_int] + [dp] * 7 +
                                                [ip, C.POINTER(C.c_uint32), C.c_uint32])
            L.orc_get_pids.argtypes = [C.c_void_p, C.POINTER(C.c_uint32)]
            L.orc_set_particles.argtypes = [C.c_void_p, C.c_int] + [dp] * 7 + [ip, C.c_uint32]
            L.orc_get_particles.argtypes = [C.c_void_p] + [dp] * 7 + [ip, C.POINTER(C.c_uint8)]
            L.orc_num_particles.argtypes = [C.c_void_p]
            L.orc_step_index.argtypes = [C.c_void_p]
            L.orc_step_index.restype = C.c_uint32
            for f in ("orc_advance", "orc_step"):
                getattr(L, f).argtypes = [C.c_void_p, C.c_double]
            for f in ("orc_redistribute", "orc_statistics", "orc_bins_capacity"):
                getattr(L, f).argtypes = [C.c_void_p]
            L.orc_finish_step.argtypes = [C.c_void_p]
            L.orc_get_element_stats.argtypes = [C.c_void_p, dp, ip]
            L.orc_get_nodal_stats.argtypes = [C.c_void_p, dp]
            L.orc_get_bins.argtypes = [C.c_void_p, dp, ip]
            L.orc_scalar_stats.argtypes = [C.c_void_p, C.c_int, ip, C.c_int, ip, dp, dp, dp, dp]
            L.orc_cfl_dt.argtypes = [C.c_void_p, dp]
            L.orc_node_gradient.argtypes = [C.c_void_p, dp, dp]
            L.orc_derive_fields.argtypes = [C.c_void_p]
            L.orc_get_fields.argtypes = [C.c_void_p, dp]
            L.orc_correct_velocity.argtypes = [C.c_void_p, dp, C.c_double]
            L.orc_last_dt.argtypes = [C.c_void_p]
            L.orc_last_dt.restype = C.c_double
            L.orc_wp_rhs.argtypes = [C.c_void_p, dp, dp]
            L.orc_wp_solve.argtypes = [C.c_void_p, dp, dp, dp, C.c_double, C.c_int, ip]
            L.orc_update_wp.argtypes = [C.c_void_p, C.c_double, C.c_int, ip]
            L.orc_fem_apply.argtypes = [C.c_void_p, C.c_int, dp, dp]
            L.orc_wp_apply.argtypes = [C.c_void_p, dp, dp, dp]
            L.orc_pressure_rhs.argtypes = [C.c_void_p, dp, dp, C.c_double, C.c_double, dp, dp]
            L.orc_pressure_solve.argtypes = [C.c_void_p, dp, dp, dp, C.c_double, C.c_int, ip]
            L.orc_coupled_step.argtypes = [C.c_void_p, C.c_double, C.c_double, dp, dp, C.c_double,
                                           C.c_int, ip, ip]
            L.orc_get_diag.argtypes = [C.c_void_p, C.POINTER(Diag)]
            L.orc_reset_diag.argtypes = [C.c_void_p]
            L.orc_redistribution_counts.argtypes = [ip, C.c_int, C.c_int, ip]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


# ---- primitives --------------------------------------------------------------------------

def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def box_muller(w1, w2):
    a, b = C.c_double(), C.c_double()
    lib().orc_box_muller(w1, w2, C.byref(a), C.byref(b))
    return a.value, b.value


def gamma_draw(seed, instance, pid, step, purpose, shape, scale):
    ex = C.c_int()
    v = lib().orc_gamma_draw(seed, instance, pid, step, purpose, shape, scale, C.byref(ex))
    return v, ex.value


def step_gaussians(seed, instance, pid, step):
    xi = np.zeros(6)
    eta = C.c_double()
    lib().orc_step_gaussians(seed, instance, pid, step, _dp(xi), C.byref(eta))
    return xi, eta.value


def redistribution_counts(counts, minnpel):
    c = np.ascontiguousarray(counts, dtype=np.int32)
    out = np.zeros_like(c)
    moves = lib().orc_redistribution_counts(_ip(c), c.size, int(minnpel), _ip(out))
    return out, moves


# ---- context -----------------------------------------------------------------------------

class Oracle:
    """One oracle instance: grid, fields, particles indexed by particle id."""

    def __init__(self, grid, params: dict, fields=None):
        L = lib()
        p = dict(params)
        p.setdefault("period_x", grid.period_x)
        self.params = make_params(p)
        self.nn, self.ne = grid.nn, grid.ne
        self._node_xy = np.ascontiguousarray(grid.node_xy, dtype=np.float64)
        self._tri = np.ascontiguousarray(grid.tri, dtype=np.int32)
        self._tag = np.ascontiguousarray(grid.edge_tag, dtype=np.int8)
        h = C.c_void_p()
        rc = L.orc_create(C.byref(h), C.byref(self.params), self.nn, _dp(self._node_xy), self.ne,
                          _ip(self._tri), self._tag.ctypes.data_as(C.POINTER(C.c_int8)))
        if rc != 0:
            raise ValueError("orc_create failed: %d" % rc)
        self.h = h
        self.G = L.orc_bins_capacity(h)
        if fields is not None:
            self.set_fields(fields)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_destroy(h)
            self.h = None

    def set_params(self, params: dict):
        p = dict(params)
        p.setdefault("period_x", self.params.period_x)
        self.params = make_params(p)
        rc = lib().orc_set_params(self.h, C.byref(self.params))
        if rc:
            raise ValueError("orc_set_params failed: %d" % rc)

    def set_fields(self, fields):
        f = np.ascontiguousarray(fields, dtype=np.float64)
        assert f.shape == (self.nn, NF)
        self._fields = f
        lib().orc_set_fields(self.h, _dp(f))

    def lam(self, e, x, y):
        out = np.zeros(3)
        lib().orc_lambda(self.h, int(e), float(x), float(y), _dp(out))
        return out

    def walk(self, e0, x, y):
        hops = C.c_int()
        e = lib().orc_walk(self.h, int(e0), float(x), float(y), C.byref(hops))
        return e, hops.value

    def brute(self, x, y):
        return lib().orc_brute_locate(self.h, float(x), float(y))

    def interp(self, e, lam):
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        q = np.zeros(NF)
        lib().orc_interp(self.h, int(e), _dp(lam), _dp(q))
        return q

    def neighbors(self):
        out = np.zeros((self.ne, 3), dtype=np.int32)
        lib().orc_neighbors(self.h, _ip(out))
        return out

    def init_particles(self, ppe):
        rc = lib().orc_init_particles(self.h, int(ppe))
        if rc:
            raise ValueError("orc_init_particles failed: %d" % rc)

    def init_elements(self, ppe, elems):
        """The particles of a ppe-per-element initialisation in the listed elements only
        (same ids and draws as the full initialisation)."""
        el = np.ascontiguousarray(np.sort(np.asarray(elems)), dtype=np.int32)
        rc = lib().orc_init_elements(self.h, int(ppe), int(el.shape[0]), _ip(el))
        if rc:
            raise ValueError("orc_init_elements failed: %d" % rc)

    def set_particles(self, st: dict, step: int, pid=None):
        """State arrays (ids 0..n-1, or the strictly ascending ids pid)."""
        n = int(st["x"].shape[0])
        arrs = [np.ascontiguousarray(st[k], dtype=np.float64) for k in ("x", "y", "u", "v", "w", "om", "psi")]
        el = np.ascontiguousarray(st["elem"], dtype=np.int32)
        if pid is None:
            rc = lib().orc_set_particles(self.h, n, *[_dp(a) for a in arrs], _ip(el), int(step))
        else:
            ids = np.ascontiguousarray(pid, dtype=np.uint32)
            rc = lib().orc_set_particles_ids(self.h, n, *[_dp(a) for a in arrs], _ip(el),
                                             ids.ctypes.data_as(C.POINTER(C.c_uint32)), int(step))
        if rc:
            raise ValueError("orc_set_particles failed: %d" % rc)

    def pids(self):
        out = np.zeros(self.np_, dtype=np.uint32)
        lib().orc_get_pids(self.h, out.ctypes.data_as(C.POINTER(C.c_uint32)))
        return out

    @property
    def np_(self):
        return lib().orc_num_particles(self.h)

    @property
    def step_index(self):
        return lib().orc_step_index(self.h)

    def get_particles(self) -> dict:
        n = self.np_
        out = {k: np.zeros(n) for k in ("x", "y", "u", "v", "w", "om", "psi")}
        out["elem"] = np.zeros(n, dtype=np.int32)
        out["cp"] = np.zeros(n, dtype=np.uint8)
        lib().orc_get_particles(self.h, *[_dp(out[k]) for k in ("x", "y", "u", "v", "w", "om", "psi")],
                                _ip(out["elem"]), out["cp"].ctypes.data_as(C.POINTER(C.c_uint8)))
        return out

    def step(self, dt):
        rc = lib().orc_step(self.h, float(dt))
        if rc:
            raise RuntimeError("orc_step failed: %d" % rc)

    def cfl_dt(self) -> float:
        """The time step of Eq. 26 from the current nodal means."""
        v = C.c_double()
        if lib().orc_cfl_dt(self.h, C.byref(v)):
            raise RuntimeError("orc_cfl_dt: every nodal mean vector is zero")
        return v.value

    @property
    def last_dt(self) -> float:
        return float(lib().orc_last_dt(self.h))

    def node_gradient(self, q):
        """Node-transferred gradient (Eqs. 39-40) of a nodal quantity: [nn][2]."""
        qq = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros((qq.size, 2))
        lib().orc_node_gradient(self.h, _dp(qq), _dp(out))
        return out

    def fields(self):
        out = np.zeros((self.nn, 32))
        lib().orc_get_fields(self.h, _dp(out))
        return out

    def correct_velocity(self, dp, dt: float):
        """Eq. 31 applied to the particles with the nodal pressure change dp[nn]."""
        d = np.ascontiguousarray(dp, dtype=np.float64)
        if lib().orc_correct_velocity(self.h, _dp(d), float(dt)):
            raise RuntimeError("orc_correct_velocity: no particles")

    def derive_fields(self):
        """Overwrite the nodal fields the particles' statistics provide (slots 0-2, 5-13,
        23-29) from the current nodal statistics."""
        lib().orc_derive_fields(self.h)

    def wp_rhs(self):
        """Eqs. 12-18 at every node from the current fields: (rhs[nn][3][3], L[nn])."""
        rhs = np.zeros((self.nn, 9))
        L = np.zeros(self.nn)
        if lib().orc_wp_rhs(self.h, _dp(rhs), _dp(L)):
            raise RuntimeError("orc_wp_rhs: a node has eps <= 0")
        return rhs.reshape(self.nn, 3, 3), L

    def wp_solve(self, rhs, L, wp0=None, tol: float = 1e-13, max_iter: int = 100000):
        """Eq. 12 by Galerkin FEM and Jacobi-PCG (Eq. 59 and the symmetry conditions at the
        boundaries): returns (wp[nn][3][3], iterations)."""
        r = np.ascontiguousarray(np.asarray(rhs, dtype=np.float64).reshape(self.nn, 9))
        LL = np.ascontiguousarray(L, dtype=np.float64)
        wp = (np.zeros((self.nn, 9)) if wp0 is None
              else np.array(np.asarray(wp0, dtype=np.float64).reshape(self.nn, 9)))
        it = C.c_int()
        rc = lib().orc_wp_solve(self.h, _dp(r), _dp(LL), _dp(wp), float(tol), int(max_iter),
                                C.byref(it))
        if rc:
            raise RuntimeError("orc_wp_solve failed: %d" % rc)
        return wp.reshape(self.nn, 3, 3), it.value

    def update_wp(self, tol: float = 1e-13, max_iter: int = 100000) -> int:
        """Eq. 12's update of the fields' wp_ij (slots 14-22); returns the iterations."""
        it = C.c_int()
        rc = lib().orc_update_wp(self.h, float(tol), int(max_iter), C.byref(it))
        if rc:
            raise RuntimeError("orc_update_wp failed: %d" % rc)
        return it.value

    def fem_apply(self, which: int, x):
        """The Galerkin mass (which = 0) or laplacian stiffness (1) applied to x[nn]."""
        xx = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.nn)
        lib().orc_fem_apply(self.h, int(which), _dp(xx), _dp(y))
        return y

    def wp_apply(self, L, x):
        """Eq. 12's Galerkin operator (M + K_L) applied to x[nn] with the length scale L[nn]."""
        LL = np.ascontiguousarray(L, dtype=np.float64)
        xx = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.nn)
        lib().orc_wp_apply(self.h, _dp(LL), _dp(xx), _dp(y))
        return y

    def pressure_rhs(self, ustar, P, dt: float, Cp: float = 1e-3):
        """Eq. 33's nodal right-hand side and Eq. 61's increment flux: (src[nn], flux[nn])."""
        u = np.ascontiguousarray(np.asarray(ustar, dtype=np.float64).reshape(self.nn, 3))
        p = np.ascontiguousarray(P, dtype=np.float64)
        src, flux = np.zeros(self.nn), np.zeros(self.nn)
        if lib().orc_pressure_rhs(self.h, _dp(u), _dp(p), float(dt), float(Cp), _dp(src), _dp(flux)):
            raise RuntimeError("orc_pressure_rhs: dt must be positive")
        return src, flux

    def pressure_solve(self, src, flux, dP0=None, tol: float = 1e-13, max_iter: int = 100000):
        """Eq. 33 by Galerkin FEM and Jacobi-PCG: (zero-mean dP[nn], iterations)."""
        s = np.ascontiguousarray(src, dtype=np.float64)
        f = np.ascontiguousarray(flux, dtype=np.float64)
        d = np.zeros(self.nn) if dP0 is None else np.array(dP0, dtype=np.float64)
        it = C.c_int()
        rc = lib().orc_pressure_solve(self.h, _dp(s), _dp(f), _dp(d), float(tol), int(max_iter),
                                      C.byref(it))
        if rc:
            raise RuntimeError("orc_pressure_solve failed: %d" % rc)
        return d, it.value

    def coupled_step(self, dt, P, dP=None, Cp: float = 1e-3, tol: float = 1e-13,
                     max_iter: int = 100000):
        """One step of the coupled loop (Table 1 order).  P[nn] is updated in place; returns
        (dP, wp iterations, pressure iterations)."""
        assert P.dtype == np.float64 and P.flags.c_contiguous and P.size == self.nn
        d = np.zeros(self.nn) if dP is None else np.array(dP, dtype=np.float64)
        wi, pi = C.c_int(), C.c_int()
        rc = lib().orc_coupled_step(self.h, float(dt), float(Cp), _dp(P), _dp(d), float(tol),
                                    int(max_iter), C.byref(wi), C.byref(pi))
        if rc:
            raise RuntimeError("orc_coupled_step failed: %d" % rc)
        return d, wi.value, pi.value

    def advance(self, dt):
        return lib().orc_advance(self.h, float(dt))

    def redistribute(self):
        return lib().orc_redistribute(self.h)

    def statistics(self):
        return lib().orc_statistics(self.h)

    def finish_step(self):
        lib().orc_finish_step(self.h)

    def element_stats(self):
        out = np.zeros((self.ne, NS))
        cnt = np.zeros(self.ne, dtype=np.int32)
        lib().orc_get_element_stats(self.h, _dp(out), _ip(cnt))
        return out, cnt

    def nodal_stats(self):
        out = np.zeros((self.nn, NS))
        lib().orc_get_nodal_stats(self.h, _dp(out))
        return out

    def scalar_stats(self, elems, nb: int = 200) -> dict:
        """Scalar statistics of probe elements (Sect. 4.1.2, Eqs. 67-69): per element the
        bin counts, Eq. 68's phi~, the conditional diffusion and dissipation per unit 1/t_m
        over nb equal bins of [0, 1], and <phi>, <phi'^2>, <phi'^3>, <phi'^4>, min, max."""
        el = np.ascontiguousarray(elems, dtype=np.int32)
        n = int(el.size)
        out = dict(count=np.zeros((n, nb), np.int32), phit=np.zeros((n, nb)),
                   cdiff=np.zeros((n, nb)), cdiss=np.zeros((n, nb)), mom=np.zeros((n, 6)))
        rc = lib().orc_scalar_stats(self.h, n, _ip(el), int(nb), _ip(out["count"]),
                                    _dp(out["phit"]), _dp(out["cdiff"]), _dp(out["cdiss"]),
                                    _dp(out["mom"]))
        if rc:
            raise RuntimeError("orc_scalar_stats failed (%d)" % rc)
        return out

    def bins(self):
        v = np.zeros((self.ne, self.G))
        g = np.zeros((self.ne, 3), dtype=np.int32)
        lib().orc_get_bins(self.h, _dp(v), _ip(g))
        return v, g

    def diag(self) -> dict:
        d = Diag()
        lib().orc_get_diag(self.h, C.byref(d))
        out = {n: getattr(d, n) for n, _ in Diag._fields_ if n != "hop_hist"}
        out["hop_hist"] = list(d.hop_hist)
        return out

    def reset_diag(self):
        lib().orc_reset_diag(self.h)
