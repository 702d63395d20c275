"""ctypes binding of the pdfx C ABI (include/pdfx.h).

Argument marshalling only: every step of the particle path runs in the CUDA library.
Device memory of a context comes from PyTorch's caching allocator (through the
``pdfx_allocator`` callbacks) and work is enqueued on PyTorch's current CUDA stream unless
a stream is given.  Loading fails loudly if the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

NF = 32
NS = 13

_lock = threading.Lock()
_lib = None


class PdfxError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = lib().pdfx_strerror(code).decode() if _lib is not None else str(code)
        super().__init__("%s failed: %s (%d)" % (what, msg, code))
        self.code = code


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("C1", "C2", "C3", "C4", "CT", "CL", "Ceta", "Cv", "gamma5", "Cw1", "Cw2", "nu")] + [
        ("c0_mode", C.c_int), ("C0", C.c_double),
        ("tm_mode", C.c_int), ("Cs", C.c_double), ("Ct", C.c_double), ("Cphi", C.c_double),
        ("src_x", C.c_double), ("src_y", C.c_double), ("src_r", C.c_double),
        ("bins", C.c_int * 3), ("min_per_bin", C.c_int), ("minnpel", C.c_int),
        ("interp_mode", C.c_int), ("source_on", C.c_int),
        ("seed", C.c_uint64), ("instance", C.c_uint32), ("period_x", C.c_double),
        ("precision", C.c_int), ("sort_every", C.c_int), ("acc64", C.c_int),
        ("cond_mode", C.c_int), ("fox_bins", C.c_int), ("model", C.c_int), ("alpha", C.c_double),
        ("cfl", C.c_double),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("user", C.c_void_p)]


class Soa(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("x", "y", "u", "v", "w", "om", "psi", "elem", "cp")]


DIAG_NAMES = ("steps", "hops_total", "walk_fallback", "walk_brute", "lost", "wall_hits",
              "freeslip_hits", "omega_reflect", "c0_clamp", "gamma_exhausted", "moves",
              "source_hits", "capacity_overflow", "nonfinite")


class Diag(C.Structure):
    _fields_ = [(n, C.c_int64) for n in DIAG_NAMES] + [("hop_hist", C.c_int64 * 8),
                                                        ("error", C.c_int32),
                                                        ("lost_records", C.c_int32),
                                                        ("lost_xy", C.c_double * 16),
                                                        ("bad_element", C.c_int64)]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libpdfx.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError("pdfx CUDA library not built: %s (run __graft_entry__.build())" % path)
            L = C.CDLL(path)
            vp, i32, i64, u32, dp = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_double
            sig = {
                "pdfx_default_params": (None, [C.POINTER(Params)]),
                "pdfx_create": (C.c_int, [C.POINTER(Params), C.POINTER(Allocator), C.POINTER(vp)]),
                "pdfx_destroy": (None, [vp]),
                "pdfx_set_params": (C.c_int, [vp, C.POINTER(Params)]),
                "pdfx_set_grid": (C.c_int, [vp, i32, vp, i32, vp, vp]),
                "pdfx_set_fields": (C.c_int, [vp, vp, C.c_int, vp]),
                "pdfx_init_particles": (C.c_int, [vp, i32, vp]),
                "pdfx_set_particles": (C.c_int, [vp, i64, C.POINTER(Soa), u32, C.c_int, vp]),
                "pdfx_get_particles": (C.c_int, [vp, C.POINTER(Soa), C.c_int, vp]),
                "pdfx_num_particles": (i64, [vp]),
                "pdfx_step_index": (u32, [vp]),
                "pdfx_step": (C.c_int, [vp, dp, vp]),
                "pdfx_last_dt": (C.c_int, [vp, C.POINTER(dp)]),
                "pdfx_derive_fields": (C.c_int, [vp, vp]),
                "pdfx_correct_velocity": (C.c_int, [vp, vp, dp, vp]),
                "pdfx_get_fields": (C.c_int, [vp, vp, vp]),
                "pdfx_batch_step": (C.c_int, [vp, i32, dp, vp]),
                "pdfx_set_instances": (C.c_int, [vp, i32, C.POINTER(Params), vp]),
                "pdfx_step_many": (C.c_int, [vp, dp, i32, C.c_int, vp]),
                "pdfx_autotune": (C.c_int, [vp, dp, vp, vp, vp]),
                "pdfx_instance_ranges": (C.c_int, [vp, vp, vp]),
                "pdfx_init_particles_batch": (C.c_int, [vp, vp, vp]),
                "pdfx_get_nodal_stats": (C.c_int, [vp, vp, C.c_int, vp]),
                "pdfx_get_element_stats": (C.c_int, [vp, vp, vp, C.c_int, vp]),
                "pdfx_get_bins": (C.c_int, [vp, vp, vp, C.c_int, vp]),
                "pdfx_bins_capacity": (C.c_int, [vp]),
                "pdfx_scalar_stats": (C.c_int, [vp, i32, vp, i32, vp, vp, vp, vp, vp, C.c_int, vp]),
                "pdfx_get_diag": (C.c_int, [vp, C.POINTER(Diag), vp]),
                "pdfx_reset_diag": (C.c_int, [vp, vp]),
                "pdfx_check": (C.c_int, [vp, vp]),
                "pdfx_set_profiling": (C.c_int, [vp, C.c_int]),
                "pdfx_stage_times": (C.c_int, [vp, C.POINTER(dp), C.POINTER(i64), C.c_int, vp]),
                "pdfx_kernel_launches": (i64, [vp]),
                "pdfx_element_stats_noalloc": (C.c_int, [vp, i64] + [vp] * 11 + [vp]),
                "pdfx_measure_fp64_rate": (C.c_int, [C.POINTER(C.c_double), vp]),
                "pdfx_get_launch_shapes": (C.c_int, [vp, vp, vp, vp]),
                "pdfx_set_launch_shapes": (C.c_int, [vp, i32, i32, i32]),
                "pdfx_wp_rhs": (C.c_int, [vp, vp, vp, vp]),
                "pdfx_wp_solve": (C.c_int, [vp, vp, vp, vp, dp, i32, C.POINTER(i32), vp]),
                "pdfx_update_wp": (C.c_int, [vp, dp, i32, C.POINTER(i32), vp]),
                "pdfx_pressure_rhs": (C.c_int, [vp, vp, vp, dp, dp, vp, vp, vp]),
                "pdfx_pressure_solve": (C.c_int, [vp, vp, vp, vp, dp, i32, C.POINTER(i32), vp]),
                "pdfx_set_pressure": (C.c_int, [vp, vp, vp]),
                "pdfx_get_pressure": (C.c_int, [vp, vp, vp, vp]),
                "pdfx_coupled_step": (C.c_int, [vp, dp, dp, dp, i32, vp, vp]),
                "pdfx_strerror": (C.c_char_p, [C.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def make_params(d: dict | None = None) -> Params:
    p = Params()
    lib().pdfx_default_params(C.byref(p))
    for k, v in (d or {}).items():
        if k == "bins":
            p.bins = (C.c_int * 3)(*[int(b) for b in v])
        elif any(k == f[0] for f in Params._fields_):
            setattr(p, k, v)
    return p


def _ptr(a) -> int | None:
    """Raw address of a contiguous numpy array or torch tensor (None passes through)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def batch_step(contexts, dt: float, stream=None):
    """One step of each of several independent contexts on one stream (pdfx_batch_step)."""
    hs = (C.c_void_p * len(contexts))(*[c.h for c in contexts])
    rc = lib().pdfx_batch_step(hs, len(contexts), float(dt), _stream(stream))
    if rc != 0:
        raise PdfxError(rc, "pdfx_batch_step")


class Context:
    """One pdfx instance on the current CUDA device."""

    def __init__(self, params: dict | None = None, use_torch_allocator: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("pdfx needs a CUDA device")
        L = lib()
        self.params = make_params(params)
        self._device = torch.cuda.current_device()
        self._alloc_ref = None
        alloc_p = None
        if use_torch_allocator:
            dev = self._device

            def _a(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev)
                except Exception:
                    return None

            def _r(ptr, nbytes, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_ref = Allocator(ALLOC_FN(_a), RELEASE_FN(_r), None)
            alloc_p = C.byref(self._alloc_ref)
        h = C.c_void_p()
        rc = L.pdfx_create(C.byref(self.params), alloc_p, C.byref(h))
        if rc:
            raise PdfxError(rc, "pdfx_create")
        self.h = h
        self.G = L.pdfx_bins_capacity(h)
        self.nn = self.ne = 0

    def close(self):
        if getattr(self, "h", None):
            lib().pdfx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc:
            raise PdfxError(rc, what)

    def set_params(self, params: dict):
        p = make_params(params)
        self._check(lib().pdfx_set_params(self.h, C.byref(p)), "pdfx_set_params")
        self.params = p

    def set_instances(self, params_list, elem_first):
        """Batch of independent instances (call before set_grid with the union grid)."""
        n = len(params_list)
        arr = (Params * n)(*[make_params(p) for p in params_list])
        ef = np.ascontiguousarray(elem_first, dtype=np.int32)
        self._check(lib().pdfx_set_instances(self.h, n, arr, ef.ctypes.data), "pdfx_set_instances")

    def instance_ranges(self):
        """(elem_first[K + 1], part_first[K + 1]) of the instances."""
        k = int(lib().pdfx_instance_ranges(self.h, None, None))
        ef = np.zeros(k + 1, dtype=np.int32)
        pf = np.zeros(k + 1, dtype=np.int64)
        lib().pdfx_instance_ranges(self.h, ef.ctypes.data, pf.ctypes.data)
        return ef, pf

    def init_particles_batch(self, ppe, stream=None):
        arr = np.ascontiguousarray(ppe, dtype=np.int32)
        self._check(lib().pdfx_init_particles_batch(self.h, arr.ctypes.data, _stream(stream)),
                    "pdfx_init_particles_batch")

    def set_grid(self, grid):
        xy = np.ascontiguousarray(grid.node_xy, dtype=np.float64)
        tri = np.ascontiguousarray(grid.tri, dtype=np.int32)
        tag = np.ascontiguousarray(grid.edge_tag, dtype=np.int8)
        self._check(lib().pdfx_set_grid(self.h, xy.shape[0], xy.ctypes.data, tri.shape[0],
                                        tri.ctypes.data, tag.ctypes.data), "pdfx_set_grid")
        self.nn, self.ne = xy.shape[0], tri.shape[0]

    def set_fields(self, fields, stream=None):
        on_dev = not isinstance(fields, np.ndarray)
        if not on_dev:
            fields = np.ascontiguousarray(fields, dtype=np.float64)
        self._keep_fields = fields
        self._check(lib().pdfx_set_fields(self.h, _ptr(fields), int(on_dev), _stream(stream)),
                    "pdfx_set_fields")
        if not on_dev:
            self.sync(stream)

    def sync(self, stream=None):
        import torch
        if stream is None:
            torch.cuda.current_stream().synchronize()
        else:
            stream.synchronize()

    def init_particles(self, ppe: int, stream=None):
        self._check(lib().pdfx_init_particles(self.h, int(ppe), _stream(stream)), "pdfx_init_particles")

    @property
    def np_(self) -> int:
        return int(lib().pdfx_num_particles(self.h))

    @property
    def step_index(self) -> int:
        return int(lib().pdfx_step_index(self.h))

    def set_particles(self, st: dict, step: int, stream=None):
        """State by particle id: FP64 arrays x, y, u, v, w, om, psi and int32 elem (host or device)."""
        keys = ("x", "y", "u", "v", "w", "om", "psi")
        on_dev = not isinstance(st["x"], np.ndarray)
        if not on_dev:
            arrs = {k: np.ascontiguousarray(st[k], dtype=np.float64) for k in keys}
            arrs["elem"] = np.ascontiguousarray(st["elem"], dtype=np.int32)
        else:
            arrs = {k: st[k].contiguous() for k in keys + ("elem",)}
        n = int(arrs["x"].shape[0])
        soa = Soa(*[_ptr(arrs[k]) for k in keys], _ptr(arrs["elem"]), None)
        self._check(lib().pdfx_set_particles(self.h, n, C.byref(soa), int(step), int(on_dev),
                                             _stream(stream)), "pdfx_set_particles")
        if on_dev:
            self._keep_state = arrs

    def get_particles(self, stream=None) -> dict:
        n = self.np_
        out = {k: np.zeros(n) for k in ("x", "y", "u", "v", "w", "om", "psi")}
        out["elem"] = np.zeros(n, dtype=np.int32)
        out["cp"] = np.zeros(n, dtype=np.uint8)
        soa = Soa(*[_ptr(out[k]) for k in ("x", "y", "u", "v", "w", "om", "psi", "elem", "cp")])
        self._check(lib().pdfx_get_particles(self.h, C.byref(soa), 0, _stream(stream)),
                    "pdfx_get_particles")
        return out

    def step(self, dt: float, stream=None):
        """One step of dt (dt <= 0: the step of Eq. 26 from the current nodal means)."""
        self._check(lib().pdfx_step(self.h, float(dt), _stream(stream)), "pdfx_step")

    def derive_fields(self, stream=None):
        """Overwrite the fields the particles' statistics provide (pdfx_derive_fields)."""
        self._check(lib().pdfx_derive_fields(self.h, _stream(stream)), "pdfx_derive_fields")

    def correct_velocity(self, dp, dt: float, stream=None):
        """Eq. 31 applied to the particles with the nodal pressure change dp[nn]."""
        d = np.ascontiguousarray(dp, dtype=np.float64)
        self._check(lib().pdfx_correct_velocity(self.h, d.ctypes.data, float(dt), _stream(stream)),
                    "pdfx_correct_velocity")

    # Eulerian solves of the coupled loop (FP64 on the device; host arrays).
    def wp_rhs(self, stream=None):
        """Eqs. 12-18 at every node from the fields: (rhs[nn][3][3], L[nn])."""
        rhs, L = np.zeros((self.nn, 9)), np.zeros(self.nn)
        self._check(lib().pdfx_wp_rhs(self.h, rhs.ctypes.data, L.ctypes.data, _stream(stream)),
                    "pdfx_wp_rhs")
        return rhs.reshape(self.nn, 3, 3), L

    def wp_solve(self, rhs, L, wp0=None, tol: float = 1e-13, max_iter: int = 100000, stream=None):
        """Eq. 12 by Galerkin FEM and Jacobi-PCG: (wp[nn][3][3], iterations)."""
        r = np.ascontiguousarray(np.asarray(rhs, dtype=np.float64).reshape(self.nn, 9))
        LL = np.ascontiguousarray(L, dtype=np.float64)
        wp = (np.zeros((self.nn, 9)) if wp0 is None
              else np.array(np.asarray(wp0, dtype=np.float64).reshape(self.nn, 9)))
        it = C.c_int32()
        self._check(lib().pdfx_wp_solve(self.h, r.ctypes.data, LL.ctypes.data, wp.ctypes.data, float(tol),
                                        int(max_iter), C.byref(it), _stream(stream)), "pdfx_wp_solve")
        return wp.reshape(self.nn, 3, 3), it.value

    def update_wp(self, tol: float = 1e-13, max_iter: int = 100000, stream=None) -> int:
        """Eq. 12's update of the fields' wp_ij (slots 14-22); returns the iterations."""
        it = C.c_int32()
        self._check(lib().pdfx_update_wp(self.h, float(tol), int(max_iter), C.byref(it), _stream(stream)),
                    "pdfx_update_wp")
        return it.value

    def pressure_rhs(self, ustar, P, dt: float, Cp: float = 1e-3, stream=None):
        """Eq. 33's nodal source and Eq. 61's increment flux: (src[nn], flux[nn])."""
        u = np.ascontiguousarray(np.asarray(ustar, dtype=np.float64).reshape(self.nn, 3))
        p = np.ascontiguousarray(P, dtype=np.float64)
        src, flux = np.zeros(self.nn), np.zeros(self.nn)
        self._check(lib().pdfx_pressure_rhs(self.h, u.ctypes.data, p.ctypes.data, float(dt), float(Cp),
                                            src.ctypes.data, flux.ctypes.data, _stream(stream)),
                    "pdfx_pressure_rhs")
        return src, flux

    def pressure_solve(self, src, flux, dP0=None, tol: float = 1e-13, max_iter: int = 100000,
                       stream=None):
        """Eq. 33 by Galerkin FEM and Jacobi-PCG: (zero-mean dP[nn], iterations)."""
        s_ = np.ascontiguousarray(src, dtype=np.float64)
        f = np.ascontiguousarray(flux, dtype=np.float64)
        d = np.zeros(self.nn) if dP0 is None else np.array(dP0, dtype=np.float64)
        it = C.c_int32()
        self._check(lib().pdfx_pressure_solve(self.h, s_.ctypes.data, f.ctypes.data, d.ctypes.data,
                                              float(tol), int(max_iter), C.byref(it), _stream(stream)),
                    "pdfx_pressure_solve")
        return d, it.value

    def set_pressure(self, P, stream=None):
        p = np.ascontiguousarray(P, dtype=np.float64)
        self._check(lib().pdfx_set_pressure(self.h, p.ctypes.data, _stream(stream)), "pdfx_set_pressure")

    def pressure(self, stream=None):
        """(P[nn], last dP[nn])."""
        P, dP = np.zeros(self.nn), np.zeros(self.nn)
        self._check(lib().pdfx_get_pressure(self.h, P.ctypes.data, dP.ctypes.data, _stream(stream)),
                    "pdfx_get_pressure")
        return P, dP

    def coupled_step(self, dt: float, Cp: float = 1e-3, tol: float = 1e-13, max_iter: int = 100000,
                     stream=None):
        """One step of the coupled loop in Table 1's order; returns the two solves' iterations."""
        it = (C.c_int32 * 2)()
        self._check(lib().pdfx_coupled_step(self.h, float(dt), float(Cp), float(tol), int(max_iter), it,
                                            _stream(stream)), "pdfx_coupled_step")
        return it[0], it[1]

    def fields(self, stream=None):
        out = np.zeros((self.nn, 32))
        self._check(lib().pdfx_get_fields(self.h, out.ctypes.data, _stream(stream)), "pdfx_get_fields")
        return out

    @property
    def last_dt(self) -> float:
        v = C.c_double()
        self._check(lib().pdfx_last_dt(self.h, C.byref(v)), "pdfx_last_dt")
        return v.value

    def autotune(self, dt: float, stream=None) -> dict:
        blk, se = C.c_int32(0), C.c_int32(0)
        self._check(lib().pdfx_autotune(self.h, float(dt), C.byref(blk), C.byref(se),
                                        _stream(stream)), "pdfx_autotune")
        return self.launch_shapes()

    def launch_shapes(self) -> dict:
        """The advance block size, the re-order period and the binning's size-class split."""
        blk, se, sp = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        self._check(lib().pdfx_get_launch_shapes(self.h, C.byref(blk), C.byref(se), C.byref(sp)),
                    "pdfx_get_launch_shapes")
        return {"adv_block": int(blk.value), "sort_every": int(se.value), "tile_split": int(sp.value)}

    def set_launch_shapes(self, adv_block: int = -1, sort_every: int = -1, tile_split: int = -1):
        """Sets the launch shapes that change no result (-1 keeps the current one)."""
        self._check(lib().pdfx_set_launch_shapes(self.h, int(adv_block), int(sort_every),
                                                 int(tile_split)), "pdfx_set_launch_shapes")

    def step_many(self, dt: float, nsteps: int, use_graph: bool = True, stream=None):
        self._check(lib().pdfx_step_many(self.h, float(dt), int(nsteps), int(bool(use_graph)),
                                         _stream(stream)), "pdfx_step_many")

    def nodal_stats(self, out=None, stream=None):
        if out is None:
            out = np.zeros((self.nn, NS))
        on_dev = not isinstance(out, np.ndarray)
        self._check(lib().pdfx_get_nodal_stats(self.h, _ptr(out), int(on_dev), _stream(stream)),
                    "pdfx_get_nodal_stats")
        return out

    def element_stats(self, stream=None):
        out = np.zeros((self.ne, NS))
        cnt = np.zeros(self.ne, dtype=np.int32)
        self._check(lib().pdfx_get_element_stats(self.h, out.ctypes.data, cnt.ctypes.data, 0,
                                                 _stream(stream)), "pdfx_get_element_stats")
        return out, cnt

    def bins(self, stream=None):
        v = np.zeros((self.ne, self.G))
        g = np.zeros((self.ne, 3), dtype=np.int32)
        self._check(lib().pdfx_get_bins(self.h, v.ctypes.data, g.ctypes.data, 0, _stream(stream)),
                    "pdfx_get_bins")
        return v, g

    def scalar_stats(self, elems, nb: int = 200, stream=None) -> dict:
        """Scalar statistics of probe elements (pdfx_scalar_stats): per element the psi bin
        counts, Eq. 68's phi~, the conditional diffusion and Eq. 67's conditional
        dissipation per unit 1/t_m over nb bins of [0, 1], and <phi>, <phi'^2>, <phi'^3>,
        <phi'^4>, min and max of psi."""
        el = np.ascontiguousarray(elems, dtype=np.int32)
        n = int(el.size)
        out = dict(count=np.zeros((n, nb), np.int32), phit=np.zeros((n, nb)),
                   cdiff=np.zeros((n, nb)), cdiss=np.zeros((n, nb)), mom=np.zeros((n, 6)))
        self._check(lib().pdfx_scalar_stats(self.h, n, el.ctypes.data, int(nb),
                                            out["count"].ctypes.data, out["phit"].ctypes.data,
                                            out["cdiff"].ctypes.data, out["cdiss"].ctypes.data,
                                            out["mom"].ctypes.data, 0, _stream(stream)),
                    "pdfx_scalar_stats")
        return out

    def diag(self, stream=None) -> dict:
        d = Diag()
        self._check(lib().pdfx_get_diag(self.h, C.byref(d), _stream(stream)), "pdfx_get_diag")
        out = {n: int(getattr(d, n)) for n in DIAG_NAMES}
        out["hop_hist"] = [int(v) for v in d.hop_hist]
        out["error"] = int(d.error)
        out["lost_records"] = [list(d.lost_xy[4 * i:4 * i + 4]) for i in range(d.lost_records)]
        out["bad_element"] = int(d.bad_element)
        return out

    def reset_diag(self, stream=None):
        self._check(lib().pdfx_reset_diag(self.h, _stream(stream)), "pdfx_reset_diag")

    def check(self, stream=None) -> int:
        return int(lib().pdfx_check(self.h, _stream(stream)))

    def set_profiling(self, on: bool):
        self._check(lib().pdfx_set_profiling(self.h, int(bool(on))), "pdfx_set_profiling")

    def stage_times(self, stream=None):
        ms = (C.c_double * 8)()
        n = (C.c_int64 * 8)()
        k = lib().pdfx_stage_times(self.h, ms, n, 8, _stream(stream))
        if k < 0:
            raise PdfxError(k, "pdfx_stage_times")
        return [float(ms[i]) for i in range(k)], [int(n[i]) for i in range(k)]

    def element_stats_noalloc(self, st: dict, emom, vcce, gbin, cp, nmom=None, stream=None):
        """Statistics of a device particle state (torch tensors by particle id) into the
        given device outputs, with no device allocation (pdfx_element_stats_noalloc)."""
        n = int(st["u"].shape[0])
        args = [_ptr(st[k]) for k in ("u", "v", "w", "om", "psi", "elem")]
        self._check(lib().pdfx_element_stats_noalloc(self.h, n, *args, _ptr(emom), _ptr(vcce),
                                                      _ptr(gbin), _ptr(cp), _ptr(nmom),
                                                      _stream(stream)),
                    "pdfx_element_stats_noalloc")

    @property
    def kernel_launches(self) -> int:
        return int(lib().pdfx_kernel_launches(self.h))


def measure_fp64_rate(stream=None) -> float:
    """FP64 FMA rate of the current device in FLOP/s (pdfx_measure_fp64_rate)."""
    out = C.c_double(0.0)
    rc = lib().pdfx_measure_fp64_rate(C.byref(out), _stream(stream))
    if rc:
        raise PdfxError(rc, "pdfx_measure_fp64_rate")
    return float(out.value)
