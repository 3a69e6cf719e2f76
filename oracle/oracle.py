"""ctypes wrapper of oracle/dartray_oracle.c (test infrastructure only).

The C file is compiled with the host C compiler into oracle/_build/ on first
use (or by ``build()``).  All arrays handed to the C code are float64 copies
of the float32 grid inputs, so both sides see the same numbers.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dartray_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXL = 16
LEDGER_NAMES = ("emitted", "absorbed", "scattered", "escaped", "blocked", "cut", "skipped")
COUNTER_NAMES = ("rays", "crossings", "splits", "merges", "blocks", "escapes", "cuts", "lows",
                 "resumes", "waves", "sources")


def _compile(src, out):
    cc = os.environ.get("CC", "gcc")
    tmp = out + f".tmp{os.getpid()}"
    cmd = [cc, "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC",
           "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def build(force=False, openmp=False):
    """Compile the oracle shared library (plain C, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    return _compile(_SRC, _LIB_PATH)


def build_variant(replacements, folder):
    """Compile a copy of the oracle with textual replacements (old, new), each
    of which must occur exactly once, into ``folder``.  Tests use it to plant
    a mistake in the oracle and check that a pin catches it; the returned
    path goes to ``Oracle(..., lib_path=...)``."""
    with open(_SRC) as f:
        src = f.read()
    for old, new in replacements:
        if src.count(old) != 1:
            raise ValueError(f"replacement target occurs {src.count(old)} times: {old!r}")
        src = src.replace(old, new)
    os.makedirs(folder, exist_ok=True)
    cpath = os.path.join(folder, "dartray_oracle_variant.c")
    with open(cpath, "w") as f:
        f.write(src)
    return _compile(cpath, os.path.join(folder, "liboracle_variant.so"))


class _Grid(C.Structure):
    _fields_ = [("nroot", C.c_int32 * 3), ("root_lo", C.c_double * 3), ("root_size", C.c_double),
                ("n_nodes", C.c_int32), ("n_leaf", C.c_int32), ("n_lambda", C.c_int32),
                ("first_child", C.c_void_p), ("leaf_of_node", C.c_void_p),
                ("kappa_rho", C.c_void_p), ("emis", C.c_void_p), ("albedo", C.c_void_p),
                ("g", C.c_void_p), ("n_point", C.c_int32), ("point_xyz", C.c_void_p),
                ("point_lum", C.c_void_p)]


class _Params(C.Structure):
    _fields_ = [("a_rt", C.c_double), ("r_pre", C.c_double), ("f_l", C.c_double),
                ("c_light", C.c_double), ("n_rays_min", C.c_int32), ("n_rays_max", C.c_int32),
                ("k0", C.c_int32), ("k_ray_max", C.c_int32), ("k_sca_cap", C.c_int32),
                ("n_fwhm", C.c_int32), ("merge", C.c_int32), ("max_cross", C.c_int32),
                ("max_waves", C.c_int32), ("src_stride", C.c_int32), ("src_offset", C.c_int32),
                ("octant", C.c_int32), ("tangent", C.c_int32)]


class _State(C.Structure):
    _fields_ = [("k_lam", C.c_int32 * MAXL), ("off_lam", C.c_int64 * MAXL), ("sca_len", C.c_int64),
                ("U", C.c_void_p), ("U_LL", C.c_void_p), ("pend_a", C.c_void_p),
                ("pend_b", C.c_void_p), ("cur_is_a", C.c_int32), ("jsca_total", C.c_void_p),
                ("ledger", (C.c_double * 7) * MAXL), ("counters", C.c_int64 * 11),
                ("L_sca2", C.c_double), ("f_u", C.c_double), ("n_src", C.c_int32),
                ("dg", C.c_void_p), ("dg_view", C.c_double * 3), ("dg_on", C.c_int32)]


_variants = {}


def _load(path=None):
    global _lib
    with _lock:
        if path is not None:
            if path not in _variants:
                _variants[path] = _bind(C.CDLL(path))
            return _variants[path]
        if _lib is None:
            _lib = _bind(C.CDLL(build()))
    return _lib


def _bind(lib):
    """Argument and result types of the oracle's C entry points."""
    P = C.c_void_p
    lib.or_pix2vec.argtypes = [C.c_int, C.c_int64, P]
    lib.or_vec2pix.argtypes = [C.c_int, P]
    lib.or_vec2pix.restype = C.c_int64
    lib.or_hg.argtypes = [C.c_double, C.c_double]
    lib.or_hg.restype = C.c_double
    lib.or_k_hp_real.argtypes = [C.c_double, C.c_int]
    lib.or_k_hp_real.restype = C.c_double
    lib.or_k_hp.argtypes = [C.c_double, C.c_int, C.c_int]
    lib.or_locate.argtypes = [P, P, P, P]
    lib.or_trace.argtypes = [P, P, P, C.c_double, C.c_int, P, P, P]
    lib.or_setup.argtypes = [P, P, P]
    lib.or_setup.restype = C.c_int64
    lib.or_direct.argtypes = [P, P, P]
    lib.or_direct_incremental.argtypes = [P, P, P]
    lib.or_scatter_iter.argtypes = [P, P, P, P]
    lib.or_run_phase.argtypes = [P, P, P, C.c_int]
    lib.or_tau.argtypes = [P, C.c_int, P, P]
    lib.or_tau.restype = C.c_double
    lib.or_map.argtypes = [P, P, P, C.c_int, C.c_int, C.c_int, P]
    lib.or_pending_next.argtypes = [P]
    lib.or_pending_next.restype = C.c_void_p
    return lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None and a.size else None


# --------------------------------------------------------------- small pure functions
def pix2vec(k, p):
    lib = _load()
    out = np.zeros(3)
    lib.or_pix2vec(int(k), int(p), _ptr(out))
    return out


def pix2vec_all(k):
    return np.array([pix2vec(k, p) for p in range(12 * 4 ** k)])


def vec2pix(k, v):
    lib = _load()
    v = np.ascontiguousarray(v, np.float64)
    return int(lib.or_vec2pix(int(k), _ptr(v)))


def hg(g, mu):
    return _load().or_hg(float(g), float(mu))


def k_hp_real(g, n_fwhm=5):
    return _load().or_k_hp_real(float(g), int(n_fwhm))


def k_hp(g, n_fwhm=5, cap=3):
    return _load().or_k_hp(float(g), int(n_fwhm), int(cap))


# --------------------------------------------------------------- grid
class _GridHandle:
    """Keeps the float64 copies alive for as long as the C struct is used."""

    def __init__(self, grid):
        self.fc = np.ascontiguousarray(grid.first_child, np.int32)
        self.lon = np.ascontiguousarray(grid.leaf_of_node, np.int32)
        self.kr = np.ascontiguousarray(grid.kappa_rho, np.float64)
        self.em = np.ascontiguousarray(grid.emissivity, np.float64)
        self.al = np.ascontiguousarray(grid.albedo, np.float64)
        self.g = np.ascontiguousarray(grid.g, np.float64)
        self.pxyz = np.ascontiguousarray(grid.point_xyz, np.float64).reshape(-1, 3)
        self.plum = np.ascontiguousarray(grid.point_lum, np.float64).reshape(self.pxyz.shape[0], grid.n_lambda)
        s = _Grid()
        s.nroot[:] = grid.nroot
        s.root_lo[:] = grid.root_lo
        s.root_size = grid.root_size
        s.n_nodes = grid.n_nodes
        s.n_leaf = grid.n_leaf
        s.n_lambda = grid.n_lambda
        s.first_child = _ptr(self.fc)
        s.leaf_of_node = _ptr(self.lon)
        s.kappa_rho = _ptr(self.kr)
        s.emis = _ptr(self.em)
        s.albedo = _ptr(self.al)
        s.g = _ptr(self.g)
        s.n_point = self.pxyz.shape[0]
        s.point_xyz = _ptr(self.pxyz)
        s.point_lum = _ptr(self.plum)
        self.s = s

    @property
    def ref(self):
        return C.byref(self.s)


def locate(grid, p, n):
    lib = _load()
    h = grid if isinstance(grid, _GridHandle) else _GridHandle(grid)
    p = np.ascontiguousarray(p, np.float64)
    n = np.ascontiguousarray(n, np.float64)
    box = np.zeros(4)
    leaf = lib.or_locate(h.ref, _ptr(p), _ptr(n), _ptr(box))
    return leaf, box


def trace(grid, xs, n, d0=0.0, cap=100000):
    lib = _load()
    h = grid if isinstance(grid, _GridHandle) else _GridHandle(grid)
    xs = np.ascontiguousarray(xs, np.float64)
    n = np.ascontiguousarray(n, np.float64)
    leaf = np.zeros(cap, np.int32)
    tin = np.zeros(cap)
    tout = np.zeros(cap)
    cnt = lib.or_trace(h.ref, _ptr(xs), _ptr(n), float(d0), int(cap), _ptr(leaf), _ptr(tin), _ptr(tout))
    if cnt < 0:
        raise OracleError(_ERRORS.get(cnt, f"error {cnt}"))
    return leaf[:cnt], tin[:cnt], tout[:cnt]


def tau_between(grid, a, b, lam=0):
    lib = _load()
    h = grid if isinstance(grid, _GridHandle) else _GridHandle(grid)
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    return lib.or_tau(h.ref, int(lam), _ptr(a), _ptr(b))


# --------------------------------------------------------------- solver
@dataclasses.dataclass
class OracleParams:
    """Parameters of the sweep (defaults are the readings of the paper's
    input-defined values used throughout the tests)."""
    a_rt: float = 0.05
    r_pre: float = 0.3
    f_l: float = 0.01
    c_light: float = 1.0
    n_rays_min: int = 5
    n_rays_max: int = 40
    k0: int = 2
    k_ray_max: int = 13
    k_sca_cap: int = 3
    n_fwhm: int = 5
    merge: int = 1
    max_cross: int = 1 << 22
    max_waves: int = 200
    src_stride: int = 1
    src_offset: int = 0
    octant: int = 0
    tangent_albedo: int = 0  # 1: also d/d albedo of U (forward mode), see Oracle

    def to_c(self, n_lambda=1):
        p = _Params()
        for f in dataclasses.fields(self):
            if f.name != "tangent_albedo":
                setattr(p, f.name, getattr(self, f.name))
        p.tangent = n_lambda if self.tangent_albedo else 0
        return p


class OracleError(RuntimeError):
    pass


_ERRORS = {-1: "out of memory", -2: "crossing cap reached", -3: "wave cap reached",
           -4: "source cell not found", -5: "no progress across a face (inexact grid coordinates)",
           -6: "octant mode: the model is not mirror-symmetric about its centre",
           -7: "the g tally is not available in the octant mode",
           -8: "forward mode: not with the octant mode"}


class Oracle:
    """Stateful FP64 solver mirroring the library calls: direct(),
    scatter_iter(), rfed(), jsca(), map()."""

    def __init__(self, grid, params: OracleParams | None = None, lib_path=None):
        self.params = params or OracleParams()
        self.user_grid = grid
        self.n_user = grid.n_lambda
        if self.params.tangent_albedo:
            # forward mode: wavelengths [n, 2n) are the derivatives of [0, n)
            # with respect to their albedo -- the same extinction, albedo and
            # g, no emission of their own; the source of a derivative is the
            # extra scattered light lost * d(albedo) of its wavelength
            grid = grid.with_lambda(np.concatenate([grid.kappa_rho, grid.kappa_rho], axis=1),
                                    np.concatenate([grid.emissivity, np.zeros_like(grid.emissivity)], axis=1),
                                    np.concatenate([grid.albedo, grid.albedo]), np.concatenate([grid.g, grid.g]))
        self.grid = grid
        self._lib = _load(lib_path)
        self._g = _GridHandle(grid)
        self._p = self.params.to_c(self.n_user)
        self._s = _State()
        n = grid.n_leaf * grid.n_lambda
        self.U = np.zeros(n)
        self.U_LL = np.zeros(n)
        sca_len = self._lib.or_setup(self._g.ref, C.byref(self._p), C.byref(self._s))
        self.pend_a = np.zeros(sca_len)
        self.pend_b = np.zeros(sca_len)
        self.jsca_total = np.zeros(sca_len)
        s = self._s
        s.U, s.U_LL = _ptr(self.U), _ptr(self.U_LL)
        s.pend_a, s.pend_b = self.pend_a.ctypes.data, self.pend_b.ctypes.data
        s.jsca_total = self.jsca_total.ctypes.data
        self.k_lam = [s.k_lam[l] for l in range(grid.n_lambda)]
        self.off_lam = [s.off_lam[l] for l in range(grid.n_lambda)]

    def _check(self, rc):
        if rc:
            raise OracleError(_ERRORS.get(rc, f"error {rc}"))

    def reset_stats(self):
        for l in range(MAXL):
            for i in range(7):
                self._s.ledger[l][i] = 0.0
        for i in range(11):
            self._s.counters[i] = 0

    def stats(self):
        nl = self.n_user
        led = {name: np.array([self._s.ledger[l][i] for l in range(nl)])
               for i, name in enumerate(LEDGER_NAMES)}
        cnt = {name: int(self._s.counters[i]) for i, name in enumerate(COUNTER_NAMES)}
        return led, cnt

    def direct(self):
        self._check(self._lib.or_direct(self._g.ref, C.byref(self._p), C.byref(self._s)))

    def dg_arm(self, view):
        """From the next direct() on, accumulate per cell and wavelength the
        derivative with respect to g of the total j_sca pixel holding `view`
        (the deposited luminosities held fixed); dg() returns it."""
        w = np.asarray(view, np.float64) / np.linalg.norm(view)
        self.dg_buf = np.zeros(self.grid.n_leaf * self.grid.n_lambda)
        self._s.dg = self.dg_buf.ctypes.data
        for a in range(3):
            self._s.dg_view[a] = w[a]
        self._s.dg_on = 1

    def dg(self):
        return self.dg_buf.reshape(self.grid.n_leaf, self.grid.n_lambda)

    def direct_incremental(self):
        """Step 2 for a change of the emissivity, on top of the current U and
        j_sca (dust self-heating iterations, Sect. 3.3)."""
        self._check(self._lib.or_direct_incremental(self._g.ref, C.byref(self._p), C.byref(self._s)))

    def set_emissivity(self, emis):
        """Replace the per-leaf emissivity [n_leaf][n_lambda] (the C side
        reads the float64 copy in place)."""
        self._g.em[...] = np.asarray(emis, np.float64).reshape(self._g.em.shape)

    def run_phase(self, mode):
        self._check(self._lib.or_run_phase(self._g.ref, C.byref(self._p), C.byref(self._s), int(mode)))

    def scatter_iter(self):
        rem = C.c_double(0)
        self._check(self._lib.or_scatter_iter(self._g.ref, C.byref(self._p), C.byref(self._s),
                                              C.byref(rem)))
        return rem.value

    @property
    def f_u(self):
        return self._s.f_u

    @property
    def n_src(self):
        return self._s.n_src

    @property
    def L_sca2(self):
        return self._s.L_sca2

    def rfed(self):
        """U [n_leaf, n_lambda] and absorbed luminosity L_abs = (1-albedo)
        kappa*rho c V U per leaf."""
        g, n = self.grid, self.n_user
        U = self.U.reshape(g.n_leaf, g.n_lambda)[:, :n].copy()
        V = g.leaf_size ** 3
        L_abs = (1.0 - g.albedo[:n].astype(np.float64))[None, :] * g.kappa_rho[:, :n].astype(np.float64) \
            * self.params.c_light * V[:, None] * U
        return U, L_abs

    def rfed_tangent(self):
        """Forward mode (tangent_albedo): dU/d albedo [n_leaf, n_lambda] with
        the blocking, splitting and merging decisions frozen, and
        dL_abs/d albedo = kappa*rho c V ((1 - albedo) dU - U)."""
        assert self.params.tangent_albedo
        g, n = self.grid, self.n_user
        U2 = self.U.reshape(g.n_leaf, g.n_lambda)
        U, dU = U2[:, :n], U2[:, n:].copy()
        k = g.kappa_rho[:, :n].astype(np.float64) * self.params.c_light * (g.leaf_size ** 3)[:, None]
        return dU, k * ((1.0 - g.albedo[:n].astype(np.float64))[None, :] * dU - U)

    def pending_next(self):
        ptr = self._lib.or_pending_next(C.byref(self._s))
        return self.pend_a if ptr == self.pend_a.ctypes.data else self.pend_b

    def jsca(self, l=0, which="total"):
        g = self.grid
        npx = 12 * 4 ** self.k_lam[l]
        src = self.jsca_total if which == "total" else self.pending_next()
        return src[self.off_lam[l]: self.off_lam[l] + g.n_leaf * npx].reshape(g.n_leaf, npx)

    def map(self, observer, nside_k, max_sub=4, use_jsca=True):
        g = self.grid
        out = np.zeros(g.n_lambda * 12 * 4 ** nside_k)
        obs = np.ascontiguousarray(observer, np.float64)
        self._check(self._lib.or_map(self._g.ref, C.byref(self._s), _ptr(obs), int(nside_k),
                                     int(max_sub), int(bool(use_jsca)), _ptr(out)))
        return out.reshape(g.n_lambda, -1)


# --------------------------------------------------------------- dust emission
def planck_lambda(lam_um, T):
    """Synthetic Planck function per unit wavelength (lambda in um, T in K),
    B = lambda^-5 / (exp(c2 / (lambda T)) - 1), c2 = hc/k = 14387.77 um K; the
    physical prefactor 2hc^2 is absorbed in the dust model's scale."""
    x = 14387.77 / (np.asarray(lam_um, np.float64) * np.asarray(T, np.float64))
    with np.errstate(over="ignore"):  # exp(x) beyond the double range: B = 0
        return np.asarray(lam_um, np.float64) ** -5 / np.expm1(x)


def dust_emission(absorbed_power, kabs, volume, lam_um, dlam_um, scale, t_lo=2.0, t_hi=5000.0, iters=200):
    """Equilibrium dust emission (Sect. 3.3, with a synthetic modified
    blackbody in place of grain models): per cell, the temperature T where
    the emitted power 4 pi V sum_i scale kabs_i B(lambda_i, T) dlambda_i
    equals the absorbed power, by bisection in log T; returns T [n_cell] and
    the emissivity j_i = scale kabs_i B(lambda_i, T) [n_cell][n_ir]
    (luminosity per volume per sr per unit wavelength).  Cells that absorb
    nothing, or have no dust, emit nothing."""
    P = np.asarray(absorbed_power, np.float64)
    k = np.asarray(kabs, np.float64)
    V = np.asarray(volume, np.float64)

    def emitted(T):
        return 4 * np.pi * V * (scale * k * planck_lambda(lam_um[None, :], T[:, None]) * dlam_um[None, :]).sum(1)

    lo = np.full(P.shape, np.log(t_lo))
    hi = np.full(P.shape, np.log(t_hi))
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        low = emitted(np.exp(mid)) < P
        lo = np.where(low, mid, lo)
        hi = np.where(low, hi, mid)
    T = np.exp(0.5 * (lo + hi))
    active = (P > 0) & (k.sum(1) > 0)
    j = np.where(active[:, None], scale * k * planck_lambda(lam_um[None, :], T[:, None]), 0.0)
    return np.where(active, T, 0.0), j


def absorbed_power(oracles, dlams):
    """Per-cell absorbed power summed over the wavelengths of one or more
    oracle runs on the same grid: sum of (1 - albedo) kappa*rho c V U dlambda
    (Sect. 3.3: the dust is heated by everything it absorbs)."""
    P = 0.0
    for o, dl in zip(oracles, dlams):
        U, L_abs = o.rfed()
        P = P + (L_abs * np.asarray(dl, np.float64)[None, :]).sum(1)
    return P


def dust_self_heating(stellar, dust, lam_ir, dlam_ir, dlam_stellar, scale, f_l=0.01, tol=0.01, max_steps=20,
                      max_iters=12):
    """The self-heating procedure of Sect. 3.3 on two oracles of one grid
    (stellar wavelengths, dust wavelengths), in the paper's order:
    1. dust emission from the absorbed stellar light;
    2. the dust emission RT (steps 1-3 of Sect. 2);
    3. the emission recomputed from the absorbed stellar and dust light;
    4. its change;
    5. an RT of the change only (no U_LL step; U and j_sca continue);
    6. 3-5 until the change is below tol everywhere.
    Returns T, j and the per-step history."""
    g = dust.grid
    V = g.leaf_size.astype(np.float64) ** 3
    kabs = (1.0 - g.albedo.astype(np.float64))[None, :] * g.kappa_rho.astype(np.float64)
    lam = np.asarray(lam_ir, np.float64)
    dl = np.asarray(dlam_ir, np.float64)
    T, j = dust_emission(absorbed_power([stellar], [dlam_stellar]), kabs, V, lam, dl, scale)
    dust.set_emissivity(j)
    j_prev = j
    dust.direct()
    hist = []
    for step in range(max_steps):
        cross = dust.stats()[1]["crossings"]
        for _ in range(max_iters):
            rem = dust.scatter_iter()
            cross += dust.stats()[1]["crossings"]
            if rem < f_l:
                break
        T, j = dust_emission(absorbed_power([stellar, dust], [dlam_stellar, dl]), kabs, V, lam, dl, scale)
        change = j - j_prev
        with np.errstate(divide="ignore", invalid="ignore"):
            rel = np.where(j_prev > 0, np.abs(change) / j_prev, np.where(j > 0, np.inf, 0.0))
        rel = float(rel.max()) if rel.size else 0.0
        hist.append(dict(step=step, max_rel_change=rel, crossings=cross))
        dust.set_emissivity(np.maximum(change, 0.0))
        j_prev = j
        if rel < tol:
            break
        dust.direct_incremental()
    return T, j, hist


# --------------------------------------------------------------- external maps
def external_frame(view, up):
    """Unit view direction w (model -> observer), image up u (orthogonal to
    w) and right r = u x w."""
    w = np.asarray(view, np.float64) / np.linalg.norm(view)
    u = np.asarray(up, np.float64) - np.dot(up, w) * w
    u /= np.linalg.norm(u)
    return w, u, np.cross(u, w)


def _cell_emission(eta, kr, ds):
    """E = eta (1 - e^{-kr ds}) / kr (eta ds for kr = 0) and dE/dkr."""
    x = kr * ds
    with np.errstate(divide="ignore", invalid="ignore"):
        omT = -np.expm1(-x)
        E = np.where(x > 0, eta * omT / np.where(kr > 0, kr, 1.0), eta * ds)
        dE = np.where(x > 1e-8, eta * (ds * (1 - omT) * kr - omT) / np.where(kr > 0, kr * kr, 1.0),
                      -0.5 * eta * ds * ds)
    return E, dE


class ExternalMapOracle:
    """Orthographic map for a distant observer (Sect. 2, end: I_obs = I_0
    e^-tau along each line of sight, the cells as a continuous medium) and its
    vector-Jacobian product with respect to kappa*rho, the source held fixed;
    plain line-by-line evaluation in double."""

    def __init__(self, oracle, view, up, origin, pixel, nx, ny, use_jsca=True):
        self.o, self.g = oracle, oracle.grid
        self.w, self.u, self.r = external_frame(view, up)
        self.origin, self.px, self.nx, self.ny = np.asarray(origin, np.float64), float(pixel), int(nx), int(ny)
        g = self.g
        self.lo = np.asarray(g.root_lo, np.float64)
        self.hi = self.lo + np.asarray(g.nroot, np.float64) * g.root_size
        # source toward the observer: emissivity plus the total scattered
        # luminosity of the j_sca pixel holding w, per its solid angle, per volume
        V = g.leaf_size.astype(np.float64) ** 3
        self.eta_sca = np.zeros((g.n_leaf, g.n_lambda))
        if use_jsca:
            for l in range(g.n_lambda):
                k = oracle.k_lam[l]
                q = vec2pix(k, self.w)
                self.eta_sca[:, l] = oracle.jsca(l, "total")[:, q] / (4 * np.pi / (12 * 4 ** k)) / V
        self.eta = g.emissivity.astype(np.float64) + self.eta_sca
        self.h = _GridHandle(g)

    def segments(self, i, j):
        """Leaves and chords along pixel (i, j)'s line of sight, front to back."""
        p0 = (self.origin[0] + (i + 0.5) * self.px) * self.r + (self.origin[1] + (j + 0.5) * self.px) * self.u
        d = -self.w
        with np.errstate(divide="ignore"):
            ta, tb = (self.lo - p0) / d, (self.hi - p0) / d
        t0 = np.max(np.where(d != 0, np.minimum(ta, tb), -np.inf))
        t1 = np.min(np.where(d != 0, np.maximum(ta, tb), np.inf))
        inside = np.all((d != 0) | ((p0 >= self.lo) & (p0 < self.hi)))
        if not (t1 > t0) or not inside:
            return np.zeros(0, np.int64), np.zeros(0)
        xs = np.clip(p0 + t0 * d, self.lo, self.hi)
        leaf, tin, tout = trace(self.h, xs, d)
        return leaf.astype(np.int64), tout - tin

    def kappa(self):
        return self.g.kappa_rho.astype(np.float64)

    def pixel(self, i, j, kr=None):
        kr = self.kappa() if kr is None else kr
        leaf, ds = self.segments(i, j)
        out = np.zeros(self.g.n_lambda)
        for l in range(self.g.n_lambda):
            E, _ = _cell_emission(self.eta[leaf, l], kr[leaf, l], ds)
            T = np.exp(-kr[leaf, l] * ds)
            Tf = np.concatenate([[1.0], np.cumprod(T)[:-1]])
            out[l] = (E * Tf).sum()
        return out

    def map(self, kr=None, eta=None):
        m = np.zeros((self.g.n_lambda, self.ny, self.nx))
        saved = self.eta
        if eta is not None:
            self.eta = eta
        try:
            for j in range(self.ny):
                for i in range(self.nx):
                    m[:, j, i] = self.pixel(i, j, kr)
        finally:
            self.eta = saved
        return m

    def vjp_g(self, dmap, dg, kr=None):
        """d/d g_l of sum(dmap * map), the radiation field held fixed: the
        map of the source dg / (Omega V) (dg: the oracle's tally for this
        view, [n_leaf][n_lambda])."""
        g = self.g
        V = g.leaf_size.astype(np.float64) ** 3
        src = np.zeros((g.n_leaf, g.n_lambda))
        for l in range(g.n_lambda):
            src[:, l] = dg[:, l] / (4 * np.pi / (12 * 4 ** self.o.k_lam[l])) / V
        return (dmap * self.map(kr, eta=src)).sum(axis=(1, 2))

    def vjp_albedo(self, dmap, kr=None):
        """d/d albedo_l of sum(dmap * map), the radiation field held fixed:
        j_sca is the albedo times a field-only quantity, so the derivative is
        the map of the scattered light alone divided by the albedo."""
        ms = self.map(kr, eta=self.eta_sca)
        a = self.g.albedo.astype(np.float64)
        return np.where(a > 0, (dmap * ms).sum(axis=(1, 2)) / np.where(a > 0, a, 1.0), 0.0)

    def vjp(self, dmap, kr=None):
        """grad[c][l] = sum over pixels of dmap d map / d kappa_rho[c][l]:
        d SB / d kr_c = T_front dE_c/dkr - ds_c (sum of the contributions of
        the cells behind c)."""
        kr = self.kappa() if kr is None else kr
        grad = np.zeros_like(kr)
        for j in range(self.ny):
            for i in range(self.nx):
                leaf, ds = self.segments(i, j)
                if leaf.size == 0:
                    continue
                for l in range(self.g.n_lambda):
                    E, dE = _cell_emission(self.eta[leaf, l], kr[leaf, l], ds)
                    T = np.exp(-kr[leaf, l] * ds)
                    Tf = np.concatenate([[1.0], np.cumprod(T)[:-1]])
                    contrib = E * Tf
                    behind = np.concatenate([np.cumsum(contrib[::-1])[::-1][1:], [0.0]])
                    np.add.at(grad[:, l], leaf, dmap[l, j, i] * (Tf * dE - ds * behind))
        return grad
