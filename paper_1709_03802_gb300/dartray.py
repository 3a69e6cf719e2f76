"""Thin Python binding of libdartray.so (include/dartray.h).

Argument marshalling only: every step of the sweep runs in the CUDA library.
The functions ``dartray_*`` mirror the C calls one to one; ``DartRay`` wraps a
grid handle for convenience.  Inputs may be numpy arrays (host) or CUDA
torch tensors (device); outputs are numpy arrays unless ``out`` is a CUDA
tensor.  If the library is not built, loading fails with an error -- there is
no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MAX_LAMBDA = 16
ERRORS = {0: "OK", -1: "INVAL", -2: "NOMEM", -3: "CUDA", -4: "QUEUE", -5: "LIMIT", -6: "STATE"}


class DartRayError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class dartray_grid_desc(C.Structure):
    _fields_ = [("nroot", C.c_int32 * 3), ("root_lo", C.c_double * 3), ("root_size", C.c_double),
                ("n_nodes", C.c_int32), ("n_leaf", C.c_int32), ("n_lambda", C.c_int32),
                ("first_child", C.c_void_p), ("leaf_of_node", C.c_void_p), ("kappa_rho", C.c_void_p),
                ("emissivity", C.c_void_p), ("albedo", C.c_void_p), ("g", C.c_void_p),
                ("n_point", C.c_int32), ("point_xyz", C.c_void_p), ("point_lum", C.c_void_p),
                ("inputs_on_device", C.c_int32)]


class dartray_params(C.Structure):
    _fields_ = [("a_rt", C.c_double), ("r_pre", C.c_double), ("f_l", C.c_double), ("c_light", C.c_double),
                ("n_rays_min", C.c_int32), ("n_rays_max", C.c_int32), ("k0", C.c_int32),
                ("k_ray_max", C.c_int32), ("k_sca_cap", C.c_int32), ("n_fwhm", C.c_int32),
                ("merge", C.c_int32), ("max_cross", C.c_int32), ("max_waves", C.c_int32),
                ("src_stride", C.c_int32), ("src_offset", C.c_int32), ("queue_rays", C.c_int64),
                ("src_batch", C.c_int64), ("profile", C.c_int32), ("deposit_direct", C.c_int32),
                ("deposit_records", C.c_int64), ("deterministic", C.c_int32), ("octant", C.c_int32),
                ("graphs", C.c_int32), ("tangent_albedo", C.c_int32)]


_L = MAX_LAMBDA


class dartray_dust(C.Structure):
    _fields_ = [("n_ir", C.c_int32), ("lam_ir", C.c_double * MAX_LAMBDA), ("dlam_ir", C.c_double * MAX_LAMBDA),
                ("n_stellar", C.c_int32), ("dlam_stellar", C.c_double * MAX_LAMBDA), ("scale", C.c_double),
                ("t_min", C.c_double), ("t_max", C.c_double)]


class dartray_stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("rays", "crossings", "splits", "merges", "blocks", "escapes",
                                          "cuts", "lows", "resumes", "waves", "sources")] + \
               [(n, C.c_double * _L) for n in ("emitted", "absorbed", "scattered", "escaped", "blocked",
                                                "cut", "skipped")] + \
               [("f_u", C.c_double), ("l_sca2", C.c_double), ("gpu_ms", C.c_double),
                ("kernel_launches", C.c_int64), ("march_ms", C.c_double), ("march_launches", C.c_int64),
                ("jsca_pixels", C.c_int64), ("flush_ms", C.c_double), ("busy_ms", C.c_double),
               ("restarts", C.c_int64), ("march_sum_ms", C.c_double), ("flushes", C.c_int64),
               ("batches", C.c_int64), ("records", C.c_int64)]

    def to_dict(self, n_lambda=1):
        out = {}
        for name, typ in self._fields_:
            v = getattr(self, name)
            out[name] = np.array(v[:n_lambda]) if hasattr(v, "__len__") else v
        return out


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libdartray.so (building it first if asked and missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"libdartray.so not built ({path}); run __graft_entry__.build()")
        _build.build()
    lib = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "dartray_params_default": ([P], C.c_int),
        "dartray_grid_create": ([P, P, P, P], C.c_int),
        "dartray_direct": ([P, P], C.c_int),
        "dartray_scatter_iter": ([P, P, P], C.c_int),
        "dartray_rfed": ([P, P, P, C.c_int], C.c_int),
        "dartray_jsca_layout": ([P, P, P, P], C.c_int),
        "dartray_jsca": ([P, C.c_int, P, C.c_int], C.c_int),
        "dartray_map": ([P, P, C.c_int32, C.c_int32, C.c_int32, P, C.c_int], C.c_int),
        "dartray_map_noalloc": ([P, P, C.c_int32, C.c_int32, C.c_int32, P, C.c_int], C.c_int),
        "dartray_state_save": ([P, C.c_char_p], C.c_int),
        "dartray_grid_create_batch": ([P, C.c_int32, P, P, P], C.c_int),
        "dartray_model_info": ([P, C.c_int32, P, P, P, P, P], C.c_int),
        "dartray_model_stats": ([P, C.c_int32, P], C.c_int),
        "dartray_autotune": ([P, C.c_int32, P, P], C.c_int),
        "dartray_dust_emission": ([P, P, P, P, P, C.c_int, P], C.c_int),
        "dartray_set_emissivity": ([P, P, C.c_int], C.c_int),
        "dartray_direct_incremental": ([P, P], C.c_int),
        "dartray_map_external": ([P, P, P, P, C.c_double, C.c_int32, C.c_int32, C.c_int32, P, C.c_int], C.c_int),
        "dartray_map_external_vjp": ([P, P, P, P, C.c_double, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, C.c_int],
                                     C.c_int),
        "dartray_set_kappa_rho": ([P, P, C.c_int], C.c_int),
        "dartray_jsca_dg_arm": ([P, P], C.c_int),
        "dartray_jsca_dg": ([P, P, C.c_int], C.c_int),
        "dartray_rfed_tangent": ([P, P, P, C.c_int], C.c_int),
        "dartray_state_load": ([P, C.c_char_p], C.c_int),
        "dartray_grid_destroy": ([P], None),
        "dartray_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


EXPORTED = ("dartray_params_default", "dartray_grid_create", "dartray_direct", "dartray_scatter_iter",
            "dartray_rfed", "dartray_jsca_layout", "dartray_jsca", "dartray_map", "dartray_map_noalloc",
            "dartray_state_save", "dartray_state_load", "dartray_grid_destroy", "dartray_last_error",
            "dartray_grid_create_batch", "dartray_model_info", "dartray_model_stats", "dartray_autotune",
            "dartray_dust_emission", "dartray_set_emissivity", "dartray_direct_incremental",
            "dartray_map_external", "dartray_map_external_vjp", "dartray_set_kappa_rho",
            "dartray_jsca_dg_arm", "dartray_jsca_dg", "dartray_rfed_tangent")


def _check(rc):
    if rc != 0:
        msg = load().dartray_last_error().decode(errors="replace")
        raise DartRayError(rc, msg)


# ---------------------------------------------------------------- raw calls
def dartray_params_default():
    p = dartray_params()
    _check(load().dartray_params_default(C.byref(p)))
    return p


def dartray_grid_create(desc, params, stream=None):
    h = C.c_void_p()
    _check(load().dartray_grid_create(C.byref(desc), C.byref(params) if params is not None else None,
                                      C.c_void_p(stream or 0), C.byref(h)))
    return h


def dartray_grid_create_batch(descs, params, stream=None):
    arr = (dartray_grid_desc * len(descs))(*descs)
    h = C.c_void_p()
    _check(load().dartray_grid_create_batch(arr, len(descs), C.byref(params) if params is not None else None,
                                            C.c_void_p(stream or 0), C.byref(h)))
    return h


def dartray_model_info(h, model):
    l0, p0 = C.c_int64(), C.c_int64()
    nl, act = C.c_int32(), C.c_int32()
    rem = C.c_double()
    _check(load().dartray_model_info(h, int(model), C.byref(l0), C.byref(nl), C.byref(p0), C.byref(rem),
                                     C.byref(act)))
    return dict(leaf_offset=l0.value, n_leaf=nl.value, point_offset=p0.value, remaining=rem.value,
                active=bool(act.value))


def dartray_model_stats(h, model):
    st = dartray_stats()
    _check(load().dartray_model_stats(h, int(model), C.byref(st)))
    return st


def dartray_direct(h):
    st = dartray_stats()
    _check(load().dartray_direct(h, C.byref(st)))
    return st


def dartray_scatter_iter(h):
    st = dartray_stats()
    rem = C.c_double(0)
    _check(load().dartray_scatter_iter(h, C.byref(rem), C.byref(st)))
    return rem.value, st


def dartray_rfed(h, U_ptr, Labs_ptr, dst_is_device):
    _check(load().dartray_rfed(h, U_ptr, Labs_ptr, int(dst_is_device)))


def dartray_jsca_layout(h, n_lambda):
    k = (C.c_int32 * MAX_LAMBDA)()
    off = (C.c_int64 * MAX_LAMBDA)()
    tot = C.c_int64()
    _check(load().dartray_jsca_layout(h, k, off, C.byref(tot)))
    return list(k[:n_lambda]), list(off[:n_lambda]), tot.value


def dartray_jsca(h, which, out_ptr, dst_is_device):
    _check(load().dartray_jsca(h, int(which), out_ptr, int(dst_is_device)))


def dartray_map(h, observer, nside_k, max_sub, use_jsca, out_ptr, dst_is_device):
    obs = (C.c_double * 3)(*[float(v) for v in observer])
    _check(load().dartray_map(h, obs, int(nside_k), int(max_sub), int(use_jsca), out_ptr, int(dst_is_device)))


def dartray_map_noalloc(h, observer, nside_k, max_sub, use_jsca, out_ptr, dst_is_device):
    obs = (C.c_double * 3)(*[float(v) for v in observer])
    _check(load().dartray_map_noalloc(h, obs, int(nside_k), int(max_sub), int(use_jsca), out_ptr,
                                      int(dst_is_device)))


def dartray_state_save(h, path):
    _check(load().dartray_state_save(h, os.fsencode(path)))


def dartray_state_load(h, path):
    _check(load().dartray_state_load(h, os.fsencode(path)))


def dartray_grid_destroy(h):
    load().dartray_grid_destroy(h)


# ---------------------------------------------------------------- helpers
def _is_cuda_tensor(x):
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _ptr(x):
    if x is None:
        return None
    if _is_cuda_tensor(x):
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return C.c_void_p(x.ctypes.data) if x.size else None
    raise TypeError(type(x))


def default_params(**overrides):
    p = dartray_params_default()
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def grid_desc(grid):
    """dartray_grid_desc of a synth.Grid-like object, and the arrays it points
    to (keep them alive while the description is used)."""
    fields = dict(first_child=grid.first_child, leaf_of_node=grid.leaf_of_node, kappa_rho=grid.kappa_rho,
                  emissivity=grid.emissivity, albedo=grid.albedo, g=grid.g, point_xyz=grid.point_xyz,
                  point_lum=grid.point_lum)
    on_dev = _is_cuda_tensor(grid.kappa_rho)
    keep = {}
    for k, v in fields.items():
        if on_dev:
            keep[k] = v.contiguous()
        else:
            dt = np.int32 if k in ("first_child", "leaf_of_node") else np.float32
            keep[k] = np.ascontiguousarray(v, dt)
    d = dartray_grid_desc()
    d.nroot[:] = [int(v) for v in grid.nroot]
    d.root_lo[:] = [float(v) for v in grid.root_lo]
    d.root_size = float(grid.root_size)
    d.n_nodes = int(keep["first_child"].shape[0])
    d.n_leaf = int(grid.n_leaf)
    d.n_lambda = int(grid.n_lambda)
    for k in fields:
        setattr(d, k, _ptr(keep[k]).value if _ptr(keep[k]) is not None else None)
    d.n_point = int(keep["point_xyz"].shape[0])
    d.inputs_on_device = 1 if on_dev else 0
    return d, keep


def _default_stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:
            stream = None
    return stream


class DartRay:
    """One grid on the current CUDA device.

    ``grid`` is a synth.Grid-like object (nroot, root_lo, root_size,
    first_child, leaf_of_node, kappa_rho, emissivity, albedo, g, point_xyz,
    point_lum).  Arrays may be numpy (host) or CUDA tensors (then all of them
    must be, and ``inputs_on_device`` is set).
    """

    def __init__(self, grid, stream=None, **params):
        self.grid = grid
        self.n_leaf = int(grid.n_leaf)
        self.n_lambda = int(grid.n_lambda)
        self.params = default_params(**params)
        d, self._keep = grid_desc(grid)
        self.stream = _default_stream(stream)
        self._h = dartray_grid_create(d, self.params, self.stream)
        self.k_lam, self.off_lam, self.sca_len = dartray_jsca_layout(self._h, self.n_lambda)

    def close(self):
        if getattr(self, "_h", None):
            dartray_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, sample_stride=64):
        """Pick the fastest deposit schedule (dartray_autotune); returns its
        index and the trial times in ms."""
        choice = C.c_int32()
        ms = (C.c_double * 3)()
        _check(load().dartray_autotune(self._h, int(sample_stride), C.byref(choice), ms))
        return choice.value, list(ms)

    def direct(self):
        self.last_stats = dartray_direct(self._h).to_dict(self.n_lambda)
        return self.last_stats

    def scatter_iter(self):
        rem, st = dartray_scatter_iter(self._h)
        self.last_stats = st.to_dict(self.n_lambda)
        return rem, self.last_stats

    def rfed(self, U=None, L_abs=None):
        dev = _is_cuda_tensor(U) or _is_cuda_tensor(L_abs)
        if U is None and not dev:
            U = np.empty((self.n_leaf, self.n_lambda), np.float32)
        if L_abs is None and not dev:
            L_abs = np.empty((self.n_leaf, self.n_lambda), np.float32)
        dartray_rfed(self._h, _ptr(U), _ptr(L_abs), dev)
        return U, L_abs

    def jsca(self, which="total", out=None):
        dev = _is_cuda_tensor(out)
        if out is None:
            out = np.empty(self.sca_len, np.float32)
        dartray_jsca(self._h, 0 if which == "total" else 1, _ptr(out), dev)
        return out

    def rfed_tangent(self, dU=None, dL_abs=None):
        """Forward mode (tangent_albedo=1): dU/d albedo and dL_abs/d albedo
        [n_leaf][n_lambda] (dartray_rfed_tangent), into the given host arrays
        or CUDA tensors (both of one kind) or new host arrays."""
        dev = _is_cuda_tensor(dU) or _is_cuda_tensor(dL_abs)
        if not dev:
            dU = np.empty((self.n_leaf, self.n_lambda), np.float32) if dU is None else dU
            dL_abs = np.empty((self.n_leaf, self.n_lambda), np.float32) if dL_abs is None else dL_abs
        _check(load().dartray_rfed_tangent(self._h, _ptr(dU), _ptr(dL_abs), int(dev)))
        return dU, dL_abs

    def jsca_block(self, l, which="total"):
        a = self.jsca(which)
        npx = 12 * 4 ** self.k_lam[l]
        return a[self.off_lam[l]: self.off_lam[l] + self.n_leaf * npx].reshape(self.n_leaf, npx)

    def map(self, observer, nside_k, max_sub=4, use_jsca=True, out=None):
        dev = _is_cuda_tensor(out)
        if out is None:
            out = np.empty((self.n_lambda, 12 * 4 ** nside_k), np.float32)
        dartray_map(self._h, observer, nside_k, max_sub, use_jsca, _ptr(out), dev)
        return out

    @staticmethod
    def _frame(view, up, origin):
        d3 = C.c_double * 3
        return d3(*map(float, view)), d3(*map(float, up)), (C.c_double * 2)(*map(float, origin))

    def map_external(self, view, up, origin, pixel, nx, ny, use_jsca=True, out=None):
        """Orthographic map for a distant observer (dartray_map_external):
        [n_lambda][ny][nx], into `out` (host array or CUDA tensor) if given."""
        if out is None:
            out = np.empty((self.n_lambda, ny, nx), np.float32)
        v, u, o = self._frame(view, up, origin)
        _check(load().dartray_map_external(self._h, v, u, o, float(pixel), int(nx), int(ny), int(bool(use_jsca)),
                                           _ptr(out), int(_is_cuda_tensor(out))))
        return out

    def map_external_vjp(self, view, up, origin, pixel, nx, ny, dmap, use_jsca=True, out=None, with_albedo=False,
                         with_g=False):
        """d/d kappa_rho of sum(dmap * map) (dartray_map_external_vjp):
        [n_leaf][n_lambda]; dmap and out both host arrays or both CUDA
        tensors.  with_albedo / with_g: also return d/d albedo and d/d g
        [n_lambda] (float64; with_g needs dg_arm(view) before direct())."""
        dev = _is_cuda_tensor(dmap)
        if dev:
            dmap = dmap.contiguous()
            if out is None:
                import torch
                out = torch.empty((self.n_leaf, self.n_lambda), dtype=torch.float32, device=dmap.device)
        else:
            dmap = np.ascontiguousarray(dmap, np.float32)
            if out is None:
                out = np.empty((self.n_leaf, self.n_lambda), np.float32)
        v, u, o = self._frame(view, up, origin)
        ga = np.zeros(self.n_lambda, np.float64)
        gg = np.zeros(self.n_lambda, np.float64)
        _check(load().dartray_map_external_vjp(self._h, v, u, o, float(pixel), int(nx), int(ny), int(bool(use_jsca)),
                                               _ptr(dmap), _ptr(out), _ptr(ga), _ptr(gg) if with_g else None,
                                               int(dev)))
        extra = ((ga,) if with_albedo else ()) + ((gg,) if with_g else ())
        return (out,) + extra if extra else out

    def dg_arm(self, view):
        """Arm the tally of d j_sca / d g for the j_sca pixel holding `view`
        (dartray_jsca_dg_arm); None disarms it.  Takes effect from the next
        direct()."""
        v = None if view is None else (C.c_double * 3)(*map(float, view))
        _check(load().dartray_jsca_dg_arm(self._h, v))

    def dg(self, out=None):
        """The armed tally [n_leaf][n_lambda] (dartray_jsca_dg)."""
        if out is None:
            out = np.empty((self.n_leaf, self.n_lambda), np.float32)
        _check(load().dartray_jsca_dg(self._h, _ptr(out), int(_is_cuda_tensor(out))))
        return out

    def set_kappa_rho(self, kr):
        k = kr.contiguous() if _is_cuda_tensor(kr) else np.ascontiguousarray(kr, np.float32)
        _check(load().dartray_set_kappa_rho(self._h, _ptr(k), int(_is_cuda_tensor(k))))

    def set_emissivity(self, emis):
        e = emis.contiguous() if _is_cuda_tensor(emis) else np.ascontiguousarray(emis, np.float32)
        _check(load().dartray_set_emissivity(self._h, _ptr(e), int(_is_cuda_tensor(e))))

    def direct_incremental(self):
        st = dartray_stats()
        _check(load().dartray_direct_incremental(self._h, C.byref(st)))
        self.last_stats = st.to_dict(self.n_lambda)
        return self.last_stats

    def dust_emission(self, stellar, lam_ir, dlam_ir, dlam_stellar, scale, t_min=2.0, t_max=5000.0):
        """Dust emission of this (dust) grid heated by the absorbed light of
        both grids (dartray_dust_emission): returns T [n_leaf], j [n_leaf][n_ir]
        and the largest relative change of j since the previous call; the
        grid's emissivity becomes that change."""
        d = dartray_dust()
        d.n_ir = self.n_lambda
        d.n_stellar = stellar.n_lambda
        for i in range(self.n_lambda):
            d.lam_ir[i], d.dlam_ir[i] = float(lam_ir[i]), float(dlam_ir[i])
        for i in range(stellar.n_lambda):
            d.dlam_stellar[i] = float(dlam_stellar[i])
        d.scale, d.t_min, d.t_max = float(scale), float(t_min), float(t_max)
        T = np.empty(self.n_leaf, np.float32)
        j = np.empty((self.n_leaf, self.n_lambda), np.float32)
        rel = C.c_double()
        _check(load().dartray_dust_emission(self._h, stellar._h, C.byref(d), _ptr(T), _ptr(j), 0, C.byref(rel)))
        return T, j, rel.value

    def save(self, path):
        dartray_state_save(self._h, path)

    def load(self, path):
        dartray_state_load(self._h, path)


class DartRayBatch(DartRay):
    """Several models traced together in one grid (dartray_grid_create_batch).

    ``grids`` share n_lambda, albedo and g.  rfed() and jsca() return all
    models concatenated; model_rfed(m), model_jsca_block(m, l) and
    model_stats(m) return one model's part."""

    def __init__(self, grids, stream=None, **params):
        self.grids = list(grids)
        self.grid = self.grids[0]
        self.n_leaf = int(sum(g.n_leaf for g in self.grids))
        self.n_lambda = int(self.grid.n_lambda)
        self.params = default_params(**params)
        descs, self._keep = [], []
        for g in self.grids:
            d, k = grid_desc(g)
            descs.append(d)
            self._keep.append(k)
        self.stream = _default_stream(stream)
        self._h = dartray_grid_create_batch(descs, self.params, self.stream)
        self.k_lam, self.off_lam, self.sca_len = dartray_jsca_layout(self._h, self.n_lambda)
        self.info = [dartray_model_info(self._h, m) for m in range(len(self.grids))]

    def model_info(self, m):
        return dartray_model_info(self._h, m)

    def model_stats(self, m):
        return dartray_model_stats(self._h, m).to_dict(self.n_lambda)

    def model_rfed(self, m, U=None, L_abs=None):
        U, L_abs = self.rfed()
        a = self.info[m]["leaf_offset"]
        b = a + self.info[m]["n_leaf"]
        return U[a:b], L_abs[a:b]

    def model_jsca_block(self, m, l, which="total"):
        blk = self.jsca_block(l, which)
        a = self.info[m]["leaf_offset"]
        return blk[a:a + self.info[m]["n_leaf"]]


def dust_self_heating(stellar, dust, lam_ir, dlam_ir, dlam_stellar, scale, f_l=0.01, tol=0.01, max_steps=20,
                      max_iters=12):
    """The dust emission RT with self-heating (Sect. 3.3): ``stellar`` has run
    its sweep; ``dust`` is a grid of the same topology at the dust
    wavelengths.  Step 1: the emission heated by the stellar light alone;
    step 2: its full RT (steps 1-2 of Sect. 2 and scattering iterations to
    f_l); then, until the emission changes by less than ``tol`` everywhere,
    the emission is recomputed with the absorbed dust light added and only
    its change is propagated (no U_LL step; U and j_sca continue).  Returns
    the per-step history (largest relative change, crossings)."""
    hist = []
    T, j, rel = dust.dust_emission(stellar, lam_ir, dlam_ir, dlam_stellar, scale)
    st = dust.direct()
    for step in range(max_steps):
        cross = st["crossings"]
        for _ in range(max_iters):
            rem, s2 = dust.scatter_iter()
            cross += s2["crossings"]
            if rem < f_l:
                break
        T, j, rel = dust.dust_emission(stellar, lam_ir, dlam_ir, dlam_stellar, scale)
        hist.append(dict(step=step, max_rel_change=rel, crossings=cross))
        if rel < tol:
            break
        st = dust.direct_incremental()
    return T, j, hist


def external_map(model, kappa_rho, view, up, origin, pixel, nx, ny, use_jsca=True, albedo=None, g=None):
    """Differentiable orthographic map: kappa_rho (CUDA tensor [n_leaf][n_lambda])
    -> map [n_lambda][ny][nx] of `model` (a DartRay), the radiation field of
    the last sweep held fixed.  Forward and backward are the library's map
    kernel and its reverse march.

    albedo, g: optional tensors [n_lambda] equal to the model's albedo and g;
    passing them (with requires_grad) gives their gradients too -- the map is
    differentiated at those values (for g, model.dg_arm(view) must precede
    the sweep)."""
    import torch

    def same(t, ref, name):
        if t is not None and not np.allclose(t.detach().cpu().numpy(), np.asarray(ref, np.float64), rtol=1e-6, atol=0):
            raise ValueError(f"{name} must hold the model's values (the map is differentiated there)")

    same(albedo, model.grid.albedo, "albedo")
    same(g, model.grid.g, "g")

    class _ExternalMap(torch.autograd.Function):
        @staticmethod
        def forward(ctx, kr, alb, gg):
            kr = kr.detach().contiguous()
            model.set_kappa_rho(kr)
            out = torch.empty((model.n_lambda, ny, nx), dtype=torch.float32, device=kr.device)
            model.map_external(view, up, origin, pixel, nx, ny, use_jsca, out=out)
            ctx.save_for_backward(kr)
            ctx.want = (alb is not None, gg is not None)
            return out

        @staticmethod
        def backward(ctx, gout):
            (kr,) = ctx.saved_tensors
            model.set_kappa_rho(kr)  # the medium the forward map saw
            wa, wg = ctx.want
            res = model.map_external_vjp(view, up, origin, pixel, nx, ny, gout.float().contiguous(), use_jsca,
                                         with_albedo=wa, with_g=wg)
            if not (wa or wg):
                return res, None, None
            res = list(res)
            gk = res.pop(0)
            ga = torch.tensor(res.pop(0), dtype=torch.float32, device=kr.device) if wa else None
            gg = torch.tensor(res.pop(0), dtype=torch.float32, device=kr.device) if wg else None
            return gk, ga, gg

    return _ExternalMap.apply(kappa_rho, albedo, g)


def rfed_albedo(model, albedo):
    """U and L_abs [n_leaf][n_lambda] (CUDA tensors) of `model`, a DartRay
    created with tangent_albedo=1 whose sweep has run, as functions of
    `albedo` (a CUDA tensor [n_lambda] holding the model's albedo): the
    backward pass contracts the upstream gradients with the forward-mode
    derivatives dU/d albedo and dL_abs/d albedo of the library's sweep (each
    wavelength depends on its own albedo only)."""
    import torch

    if not np.allclose(albedo.detach().cpu().numpy(), np.asarray(model.grid.albedo, np.float64), rtol=1e-6, atol=0):
        raise ValueError("albedo must hold the model's values (the sweep ran with them)")

    class _RfedAlbedo(torch.autograd.Function):
        @staticmethod
        def forward(ctx, alb):
            shape = (model.n_leaf, model.n_lambda)
            U = torch.empty(shape, dtype=torch.float32, device=alb.device)
            L = torch.empty_like(U)
            dU = torch.empty_like(U)
            dL = torch.empty_like(U)
            model.rfed(U, L)
            model.rfed_tangent(dU, dL)
            ctx.save_for_backward(dU, dL)
            return U, L

        @staticmethod
        def backward(ctx, gU, gL):
            dU, dL = ctx.saved_tensors
            g = torch.zeros(dU.shape[1], dtype=torch.float64, device=dU.device)
            if gU is not None:
                g += (gU.double() * dU.double()).sum(0)
            if gL is not None:
                g += (gL.double() * dL.double()).sum(0)
            return g.float()

    return _RfedAlbedo.apply(albedo)
