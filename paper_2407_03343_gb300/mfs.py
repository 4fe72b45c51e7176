"""Thin ctypes binding of libmfs (include/mfs.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays to
pointers, checks status codes and raises ``MfsError`` on failure.  If libmfs.so has not
been built, importing the library raises immediately -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmfs.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "mfs.h")

FP64 = 0
MIXED = 1
FP32 = 2
MIXED_PASS = 3   # single-step entry points: the operator of the MIXED GMRES passes
RESIDUAL_AUTO = 0
RESIDUAL_FP64 = 1
RESIDUAL_SOLVE = 2

STATUS = {0: "MFS_OK", -1: "MFS_ERR_ARG", -2: "MFS_ERR_GEOMETRY", -3: "MFS_ERR_UNSUPPORTED",
          -4: "MFS_ERR_STATE", -5: "MFS_ERR_NOT_CONVERGED", -6: "MFS_ERR_NUMERIC", -7: "MFS_ERR_OOM",
          -8: "MFS_ERR_CUDA", -9: "MFS_ERR_TIMEOUT"}


class Params(C.Structure):
    _fields_ = [("n_proxy", C.c_int), ("r_proxy", C.c_double), ("m_basic", C.c_int),
                ("delta_offset", C.c_double), ("alpha1", C.c_int), ("alpha2", C.c_int),
                ("beta1", C.c_double), ("beta2", C.c_double), ("eps_trunc", C.c_double),
                ("nim_a", C.c_double), ("nim_b", C.c_double), ("nim_cut", C.c_double),
                ("nim_max", C.c_int), ("nim_fixed", C.c_int), ("left_precond", C.c_int),
                ("visc", C.c_double), ("build_factors", C.c_int), ("nim_min", C.c_int),
                ("far_dist", C.c_double), ("far_n_eq", C.c_int), ("far_r_eq", C.c_double),
                ("far_r_chk", C.c_double), ("far_eps", C.c_double), ("tensor_step1", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int),
                ("restart", C.c_int), ("max_refine", C.c_int), ("inner_tol", C.c_double),
                ("residual", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("refinements", C.c_int), ("rel_residual", C.c_double),
                ("seconds", C.c_double), ("converged", C.c_int)]


class Sizes(C.Structure):
    _fields_ = [("P", C.c_int), ("n_contacts", C.c_int), ("n_colloc", C.c_int),
                ("n_proxy_total", C.c_int), ("n_image_nodes", C.c_int), ("n_unknowns", C.c_int),
                ("n_factors", C.c_int), ("pairs_fp", C.c_longlong), ("pairs_near_fp", C.c_longlong),
                ("pairs_far_eq", C.c_longlong), ("n_factors_shared", C.c_int), ("n_factors_reused", C.c_int)]


class Timing(C.Structure):
    _fields_ = [("kernel_launches", C.c_longlong), ("pair_launches", C.c_longlong), ("pair_ms", C.c_double),
                ("pair_interactions", C.c_longlong), ("pair_proxy", C.c_longlong),
                ("pair_image_nodes", C.c_longlong), ("pair_kind", C.c_int), ("gemv_launches", C.c_longlong),
                ("gemv_ms", C.c_double), ("gemv_bytes", C.c_double),
                ("by_kind_launches", C.c_longlong * 3), ("by_kind_ms", C.c_double * 3),
                ("by_kind_proxy", C.c_longlong * 3), ("by_kind_image_nodes", C.c_longlong * 3),
                ("krylov_launches", C.c_longlong), ("krylov_ms", C.c_double), ("krylov_bytes", C.c_double),
                ("far_launches", C.c_longlong), ("far_ms", C.c_double), ("far_pairs", C.c_longlong),
                ("tc_launches", C.c_longlong), ("tc_columns", C.c_longlong),
                ("pair_issued_flops", C.c_double), ("pair_shared_rhs", C.c_longlong)]


class PairShapes(C.Structure):
    _fields_ = [("all_nodes_per_thread", C.c_int), ("all_parts", C.c_int), ("near_nodes_per_thread", C.c_int),
                ("near_parts", C.c_int), ("far_nodes_per_thread", C.c_int), ("far_parts", C.c_int),
                ("far_packed", C.c_int), ("all_ms", C.c_double), ("near_ms", C.c_double), ("far_ms", C.c_double)]


class MfsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib():
    """Load libmfs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    sig = {
        "mfs_default_params": (None, [C.POINTER(Params)]),
        "mfs_default_solve_opts": (None, [C.POINTER(SolveOpts)]),
        "mfs_create": (C.c_int, [C.POINTER(P), C.c_int, P]),
        "mfs_destroy": (None, [P]),
        "mfs_last_error": (C.c_char_p, [P]),
        "mfs_set_spheres": (C.c_int, [P, C.c_int, _D, _D]),
        "mfs_set_rigid_velocities": (C.c_int, [P, _D, _D]),
        "mfs_set_rigid_velocities_device": (C.c_int, [P, P, P]),
        "mfs_set_forces_torques": (C.c_int, [P, _D, _D]),
        "mfs_get_rigid_velocities": (C.c_int, [P, _D, _D]),
        "mfs_set_background_flow": (C.c_int, [P, _D, _D, _D]),
        "mfs_build": (C.c_int, [P, C.POINTER(Params)]),
        "mfs_sizes": (C.c_int, [P, C.POINTER(Sizes)]),
        "mfs_discretise_host": (C.c_int, [C.c_int, _D, C.c_double, C.POINTER(Params), _I, _I, _D, _D, _I, _D, _I]),
        "mfs_solve": (C.c_int, [P, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
        "mfs_get_forces_torques": (C.c_int, [P, _D, _D]),
        "mfs_get_forces_torques_device": (C.c_int, [P, P, P]),
        "mfs_eval_velocity": (C.c_int, [P, C.c_int, _D, _D]),
        "mfs_get_strengths": (C.c_int, [P, _D, _D, _I]),
        "mfs_get_collocation": (C.c_int, [P, _D, _D, _I]),
        "mfs_get_rhs": (C.c_int, [P, _D]),
        "mfs_apply_operator": (C.c_int, [P, C.c_int, _D, _D]),
        "mfs_apply_precond": (C.c_int, [P, C.c_int, _D, _D]),
        "mfs_apply_pairs": (C.c_int, [P, C.c_int, _D, _D, _D]),
        "mfs_apply_precond_noalloc": (C.c_int, [P, P, P]),
        "mfs_batch_solve": (C.c_int, [C.c_int, C.POINTER(P), C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
        "mfs_batch_solve_rhs": (C.c_int, [C.c_int, C.POINTER(P), C.POINTER(P), C.POINTER(P),
                                          C.POINTER(SolveOpts), C.POINTER(SolveInfo), C.POINTER(P), C.POINTER(P)]),
        "mfs_batch_solve_rhs_device": (C.c_int, [C.c_int, C.POINTER(P), C.POINTER(P), C.POINTER(P),
                                                 C.POINTER(SolveOpts), C.POINTER(SolveInfo), C.POINTER(P), C.POINTER(P)]),
        "mfs_set_profiling": (C.c_int, [P, C.c_int]),
        "mfs_probe_alu_peak": (C.c_int, [C.c_int, C.c_int, _D, _D]),
        "mfs_tune_pairs": (C.c_int, [P, C.POINTER(PairShapes)]),
        "mfs_set_memory_limit": (C.c_int, [P, C.c_ulonglong]),
        "mfs_memory_in_use": (C.c_int, [P, C.POINTER(C.c_ulonglong)]),
        "mfs_get_timing": (C.c_int, [P, C.POINTER(Timing), C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def declared_functions():
    """Names of the functions include/mfs.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mfs_[a-z0-9_]+)\s*\(", txt)))


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(_I) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def default_params(**kw) -> Params:
    p = Params()
    lib().mfs_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def default_solve_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib().mfs_default_solve_opts(C.byref(o))
    for k, v in kw.items():
        if k not in [f[0] for f in SolveOpts._fields_]:
            raise KeyError(k)
        if k == "precision" and isinstance(v, str):
            v = {"fp64": FP64, "mixed": MIXED, "fp32": FP32}[v]
        if k == "residual" and isinstance(v, str):
            v = {"auto": RESIDUAL_AUTO, "fp64": RESIDUAL_FP64, "solve": RESIDUAL_SOLVE}[v]
        setattr(o, k, v)
    return o


class Context:
    """One solver context on one GPU (mirrors mfs_create ... mfs_destroy)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self._L = lib()
        self._h = C.c_void_p()
        st = self._L.mfs_create(C.byref(self._h), int(device), C.c_void_p(stream) if stream else None)
        if st != 0:
            raise MfsError(st, "mfs_create failed")
        self.P = 0

    def close(self):
        if self._h:
            self._L.mfs_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st, allow=()):
        if st != 0 and st not in allow:
            raise MfsError(st, self._L.mfs_last_error(self._h).decode())
        return st

    # -- problem set-up
    def set_spheres(self, centres, radius=1.0):
        """P sphere centres (P, 3) of one common radius (mfs_set_spheres)."""
        c = _f64(centres).reshape(-1, 3)
        P = c.shape[0]
        r = _f64(np.broadcast_to(np.asarray(radius, dtype=np.float64), (P,)).copy())
        self._check(self._L.mfs_set_spheres(self._h, P, _dp(c), _dp(r)))
        self.P = P

    def build(self, params: Params | None = None, **kw):
        """Discretise and factor the one-body blocks (mfs_build); keywords override the defaults."""
        p = params if params is not None else default_params(**kw)
        self._check(self._L.mfs_build(self._h, C.byref(p)))

    def sizes(self) -> Sizes:
        """Node, source and unknown counts of the built discretisation (mfs_sizes)."""
        s = Sizes()
        self._check(self._L.mfs_sizes(self._h, C.byref(s)))
        return s

    def set_rigid_velocities(self, v, omega):
        """Rigid velocities v and omega, each (P, 3): the next solve is the resistance problem."""
        v = _f64(v, (self.P, 3))
        w = _f64(omega, (self.P, 3))
        self._check(self._L.mfs_set_rigid_velocities(self._h, _dp(v), _dp(w)))

    def set_rigid_velocities_device(self, v_ptr: int, omega_ptr: int):
        """As set_rigid_velocities, from device pointers of 3P doubles each."""
        self._check(self._L.mfs_set_rigid_velocities_device(self._h, C.c_void_p(v_ptr), C.c_void_p(omega_ptr)))

    def set_forces_torques(self, F, T):
        """Prescribe forces and torques: the next solve is the mobility problem."""
        F = _f64(F, (self.P, 3))
        T = _f64(T, (self.P, 3))
        self._check(self._L.mfs_set_forces_torques(self._h, _dp(F), _dp(T)))

    def rigid_velocities(self):
        """(V, Omega) found by the last mobility solve, each (P, 3)."""
        v = np.zeros((self.P, 3))
        w = np.zeros((self.P, 3))
        self._check(self._L.mfs_get_rigid_velocities(self._h, _dp(v), _dp(w)))
        return v, w

    def set_background_flow(self, U=None, E=None, Omega=None):
        """Background flow U + E x + Omega x x (each term optional; no arguments clears it)."""
        a = _f64(U, (3,)) if U is not None else None
        b = _f64(E, (3, 3)) if E is not None else None
        c = _f64(Omega, (3,)) if Omega is not None else None
        self._check(self._L.mfs_set_background_flow(self._h, _dp(a), _dp(b), _dp(c)))

    # -- solve and outputs
    def solve(self, opts: SolveOpts | None = None, allow_not_converged=False, **kw) -> SolveInfo:
        """GMRES solve with refinement (mfs_solve); keywords override the default options."""
        o = opts if opts is not None else default_solve_opts(**kw)
        info = SolveInfo()
        allow = (-5,) if allow_not_converged else ()
        self._check(self._L.mfs_solve(self._h, C.byref(o), C.byref(info)), allow)
        return info

    def forces_torques(self):
        """(F, T), each (P, 3): force and torque each sphere exerts on the fluid."""
        F = np.zeros((self.P, 3))
        T = np.zeros((self.P, 3))
        self._check(self._L.mfs_get_forces_torques(self._h, _dp(F), _dp(T)))
        return F, T

    def forces_torques_device(self, F_ptr: int, T_ptr: int):
        """As forces_torques, into device buffers of 3P doubles each."""
        self._check(self._L.mfs_get_forces_torques_device(self._h, C.c_void_p(F_ptr), C.c_void_p(T_ptr)))

    def eval_velocity(self, x):
        """Disturbance velocity u(x) at points x (n, 3), from the solved strengths."""
        x = _f64(x).reshape(-1, 3)
        u = np.zeros_like(x)
        self._check(self._L.mfs_eval_velocity(self._h, x.shape[0], _dp(x), _dp(u)))
        return u

    def strengths(self, with_positions=False):
        """Source strengths lambda in the library order (optionally with positions and types)."""
        s = self.sizes()
        lam = np.zeros(s.n_unknowns)
        nv = s.n_unknowns // 3
        pos = np.zeros((nv, 3)) if with_positions else None
        typ = np.zeros(nv, dtype=np.int32) if with_positions else None
        self._check(self._L.mfs_get_strengths(self._h, _dp(lam), _dp(pos), _ip(typ)))
        return (lam, pos, typ) if with_positions else lam

    def source_layout(self):
        """Positions (n_sources, 3) and types (0 Stokeslet, 1 rotlet, 2 dipole) of all vector sources."""
        s = self.sizes()
        nv = s.n_unknowns // 3
        pos = np.zeros((nv, 3))
        typ = np.zeros(nv, dtype=np.int32)
        self._check(self._L.mfs_get_strengths(self._h, None, _dp(pos), _ip(typ)))
        return pos, typ

    def collocation(self):
        """Collocation nodes (n, 3), area weights (n) and owner sphere (n)."""
        s = self.sizes()
        x = np.zeros((s.n_colloc, 3))
        w = np.zeros(s.n_colloc)
        o = np.zeros(s.n_colloc, dtype=np.int32)
        self._check(self._L.mfs_get_collocation(self._h, _dp(x), _dp(w), _ip(o)))
        return x, w, o

    def rhs(self):
        """Scaled boundary data W b at the collocation nodes (3 n)."""
        s = self.sizes()
        b = np.zeros(3 * s.n_colloc)
        self._check(self._L.mfs_get_rhs(self._h, _dp(b)))
        return b

    def apply_operator(self, mu, precision=FP64):
        """G_hat mu (the preconditioned operator) in the given precision."""
        mu = _f64(mu)
        out = np.zeros_like(mu)
        self._check(self._L.mfs_apply_operator(self._h, int(precision), _dp(mu), _dp(out)))
        return out

    def apply_precond(self, mu, precision=FP64):
        """lambda_hat = B^+ mu for every sphere (step 1)."""
        mu = _f64(mu)
        out = np.zeros(self.sizes().n_unknowns)
        self._check(self._L.mfs_apply_precond(self._h, int(precision), _dp(mu), _dp(out)))
        return out

    def apply_precond_noalloc(self, d_mu_ptr: int, d_lambda_hat_ptr: int):
        """Step 1 on caller-owned device buffers, without any device allocation."""
        self._check(self._L.mfs_apply_precond_noalloc(self._h, C.c_void_p(d_mu_ptr), C.c_void_p(d_lambda_hat_ptr)))

    def set_profiling(self, on=True):
        """Record CUDA events around the pair and GEMV launches of this context."""
        self._check(self._L.mfs_set_profiling(self._h, 1 if on else 0))

    def timing(self, reset=False) -> Timing:
        """Launch counts, device times and work counters since the last reset."""
        t = Timing()
        self._check(self._L.mfs_get_timing(self._h, C.byref(t), 1 if reset else 0))
        return t

    def tune_pairs(self) -> PairShapes:
        """Time the candidate tile shapes of the pair kernels and keep the fastest (mfs_tune_pairs)."""
        r = PairShapes()
        self._check(self._L.mfs_tune_pairs(self._h, C.byref(r)))
        return r

    def set_memory_limit(self, nbytes: int):
        """Cap the device memory this context may hold (0 = no cap); see mfs_set_memory_limit."""
        self._check(self._L.mfs_set_memory_limit(self._h, int(nbytes)))

    def memory_in_use(self) -> int:
        """Device bytes the context holds under the cap's accounting."""
        b = C.c_ulonglong(0)
        self._check(self._L.mfs_memory_in_use(self._h, C.byref(b)))
        return int(b.value)

    def apply_pairs(self, lam_hat, mu, precision=FP64):
        """mu + W sum over other spheres of G lambda_hat (steps 2 and 3)."""
        lam_hat = _f64(lam_hat)
        mu = _f64(mu)
        out = np.zeros_like(mu)
        self._check(self._L.mfs_apply_pairs(self._h, int(precision), _dp(lam_hat), _dp(mu), _dp(out)))
        return out


def probe_alu_peak(device: int = 0, kind: str = "fp32"):
    """Measured FFMA (kind "fp32") or DFMA ("fp64") peak of the device: (TFLOP/s, ms of the launch)."""
    t = C.c_double(0)
    ms = C.c_double(0)
    st = lib().mfs_probe_alu_peak(int(device), {"fp32": 0, "fp64": 1}[kind], C.byref(t), C.byref(ms))
    if st != 0:
        raise MfsError(st, "mfs_probe_alu_peak failed")
    return t.value, ms.value


def discretise_host(centres, radius=1.0, params: Params | None = None, **kw):
    """The discretisation of build() computed on the host without a GPU: returns the collocation
    nodes (n, 3), weights (n), owners (n), source positions (m, 3) and types (m)."""
    L = lib()
    c = _f64(centres).reshape(-1, 3)
    p = params if params is not None else default_params(**kw)
    nc, ns = C.c_int(0), C.c_int(0)
    st = L.mfs_discretise_host(c.shape[0], _dp(c), float(radius), C.byref(p), C.byref(nc), C.byref(ns),
                               None, None, None, None, None)
    if st != 0:
        raise MfsError(st, "mfs_discretise_host failed")
    x = np.zeros((nc.value, 3))
    w = np.zeros(nc.value)
    owner = np.zeros(nc.value, dtype=np.int32)
    pos = np.zeros((ns.value, 3))
    typ = np.zeros(ns.value, dtype=np.int32)
    st = L.mfs_discretise_host(c.shape[0], _dp(c), float(radius), C.byref(p), None, None, _dp(x), _dp(w), _ip(owner),
                               _dp(pos), _ip(typ))
    if st != 0:
        raise MfsError(st, "mfs_discretise_host failed")
    return x, w, owner, pos, typ


def batch_solve(contexts, opts: SolveOpts | None = None, allow_not_converged=False, **kw):
    """mfs_batch_solve over several built contexts; returns the list of SolveInfo."""
    L = lib()
    n = len(contexts)
    arr = (C.c_void_p * n)(*[c._h.value for c in contexts])
    infos = (SolveInfo * n)()
    o = opts if opts is not None else default_solve_opts(**kw)
    st = L.mfs_batch_solve(n, arr, C.byref(o), infos)
    if st != 0 and not (allow_not_converged and st == -5):
        bad = [i for i in range(n) if infos[i].converged == 0]
        msg = L.mfs_last_error(contexts[bad[0]]._h).decode() if bad else ""
        raise MfsError(st, f"batch solve failed ({len(bad)} problems): {msg}")
    return list(infos)


def batch_solve_rhs(contexts, velocities, opts: SolveOpts | None = None, allow_not_converged=False, **kw):
    """Several right-hand sides, contexts may repeat: velocities[i] = (v_i, omega_i) host arrays.
    Returns (infos, [(F_i, T_i)])."""
    L = lib()
    n = len(contexts)
    keep = []
    vs = (C.c_void_p * n)()
    ws = (C.c_void_p * n)()
    Fs = (C.c_void_p * n)()
    Ts = (C.c_void_p * n)()
    outs = []
    for i, (c, (v, w)) in enumerate(zip(contexts, velocities)):
        v = _f64(v, (c.P, 3))
        w = _f64(w, (c.P, 3))
        F = np.zeros((c.P, 3))
        T = np.zeros((c.P, 3))
        keep += [v, w]
        outs.append((F, T))
        vs[i], ws[i], Fs[i], Ts[i] = v.ctypes.data, w.ctypes.data, F.ctypes.data, T.ctypes.data
    arr = (C.c_void_p * n)(*[c._h.value for c in contexts])
    infos = (SolveInfo * n)()
    o = opts if opts is not None else default_solve_opts(**kw)
    st = L.mfs_batch_solve_rhs(n, arr, vs, ws, C.byref(o), infos, Fs, Ts)
    if st != 0 and not (allow_not_converged and st == -5):
        raise MfsError(st, L.mfs_last_error(contexts[0]._h).decode())
    return list(infos), outs


def batch_solve_rhs_device(contexts, v_ptrs, w_ptrs, F_ptrs, T_ptrs, opts: SolveOpts | None = None,
                           allow_not_converged=False, **kw):
    """Device-pointer variant of batch_solve_rhs (pointers as integers)."""
    L = lib()
    n = len(contexts)
    arr = (C.c_void_p * n)(*[c._h.value for c in contexts])
    infos = (SolveInfo * n)()
    o = opts if opts is not None else default_solve_opts(**kw)
    mk = lambda ps: (C.c_void_p * n)(*ps)
    st = L.mfs_batch_solve_rhs_device(n, arr, mk(v_ptrs), mk(w_ptrs), C.byref(o), infos, mk(F_ptrs), mk(T_ptrs))
    if st != 0 and not (allow_not_converged and st == -5):
        raise MfsError(st, L.mfs_last_error(contexts[0]._h).decode())
    return list(infos)
