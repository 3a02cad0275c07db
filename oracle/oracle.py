"""ctypes wrapper of the plain FP64 CPU oracle (lbm_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
bench's CPU-baseline leg.  The product path never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.cpp")
LIB = os.path.join(HERE, "liblbm_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no fast-math, no FMA contraction;
    OpenMP over the elements of a level, see set_threads).
    ORACLE_LIB_OVERRIDE names a prebuilt oracle library to load instead (used to
    check that the pins catch planted mistakes)."""
    if os.environ.get("ORACLE_LIB_OVERRIDE"):
        return os.environ["ORACLE_LIB_OVERRIDE"]
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-shared",
                               "-fPIC", SRC, "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P, I64, I, D = C.c_void_p, C.c_int64, C.c_int, C.c_double
        L.orc_create.restype = P
        L.orc_create.argtypes = [I, I, P, P, D, D, P, I, P, I64, I, C.c_char_p, I]
        L.orc_dual_create.restype = P
        L.orc_dual_create.argtypes = [I, I, P, P, D, D, D, P, P, I, P, I64, I, C.c_char_p, I]
        L.orc_destroy.argtypes = [P]
        L.orc_dual_destroy.argtypes = [P]
        L.orc_counts.argtypes = [P, P, I]
        L.orc_level_omega.restype = D
        L.orc_level_omega.argtypes = [P, I]
        for name in ("orc_init", "orc_dual_init"):
            getattr(L, name).argtypes = [P, P, P, P, P]
        L.orc_set_force.argtypes = [P, P]
        L.orc_set_outlet.argtypes = [P, I]
        L.orc_dual_set_outlet.argtypes = [P, I]
        L.orc_set_inlet_profile.argtypes = [P, I]
        L.orc_dual_set_inlet_profile.argtypes = [P, I]
        L.orc_set_link_q.argtypes = [P, I64, P, P, P]
        L.orc_dual_set_link_q.argtypes = [P, I64, P, P, P]
        L.orc_dual_set_force.argtypes = [P, P, P]
        L.orc_step.argtypes = [P, I64]
        L.orc_dual_step.argtypes = [P, I64]
        L.orc_fill_ghosts.argtypes = [P]
        L.orc_moments.argtypes = [P, P, P, P]
        L.orc_get_f.argtypes = [P, P]
        L.orc_set_f.argtypes = [P, P]
        L.orc_dual_set_f.argtypes = [P, P, P]
        L.orc_ghost_count.restype = I64
        L.orc_ghost_count.argtypes = [P]
        L.orc_ghosts.argtypes = [P, P, P]
        L.orc_reduce.argtypes = [P, P]
        L.orc_dual_reduce.argtypes = [P, P, P]
        L.orc_compact_velocity.argtypes = [I, P, P, P, P]
        L.orc_set_threads.argtypes = [I]
        L.orc_set_threads.restype = I
        L.orc_op.argtypes = [P, I, I]
        L.orc_op.restype = I
        L.orc_nlev.argtypes = [P]
        L.orc_nlev.restype = I
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def set_threads(n: int = 0) -> int:
    """Threads the oracle's element loops use (n <= 0: the OpenMP default, all
    cores unless OMP_NUM_THREADS says otherwise); returns the count in use.
    Results are the same for every count."""
    return int(lib().orc_set_threads(int(n)))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class OracleError(RuntimeError):
    pass


class Oracle:
    """One multilevel simulation held by the oracle.  With dual=True every value
    carries a tangent (forward-mode derivative along omega_dot and F_dot).
    n_levels > 0 fixes the number of levels from the coarsest one present; the
    levels beyond those the treeIDs span hold no element (an empty refined
    region)."""

    def __init__(self, mesh, stencil, omega_c, time_mode=0, rho0=1.0, u_in=(0.0, 0.0, 0.0),
                 use_force=False, dual=False, omega_dot=0.0, u_in_dot=(0.0, 0.0, 0.0), outlet=0,
                 inlet_profile=0, n_levels=0):
        L = lib()
        self.mesh, self.stencil, self.dual = mesh, stencil, dual
        self.d = 2 if stencil == 9 else 3
        self.Q = stencil
        self.ns = 3 if self.d == 2 else 6
        self.n = mesh.n
        self._keep = [np.ascontiguousarray(mesh.tree_ids, dtype=np.int64),
                      np.array(list(mesh.extent) + [1] * (3 - len(mesh.extent)), dtype=np.int32),
                      np.array(list(mesh.bc) + [0] * (6 - len(mesh.bc)), dtype=np.int32),
                      np.array(list(u_in) + [0.0] * (3 - len(u_in)), dtype=np.float64),
                      np.array(list(u_in_dot) + [0.0] * (3 - len(u_in_dot)), dtype=np.float64)]
        tid, ext, bc, uin, uin_dot = self._keep
        err = C.create_string_buffer(512)
        if dual:
            h = L.orc_dual_create(stencil, time_mode, _p(ext), _p(bc), omega_c, omega_dot, rho0, _p(uin),
                                  _p(uin_dot), int(use_force), _p(tid), self.n, int(n_levels), err, 512)
        else:
            h = L.orc_create(stencil, time_mode, _p(ext), _p(bc), omega_c, rho0, _p(uin), int(use_force),
                             _p(tid), self.n, int(n_levels), err, 512)
        if not h:
            raise OracleError(err.value.decode())
        self.h = h
        # outlet extrapolation: 0 linear (Sec. 2.3), 1 zero-gradient
        if (L.orc_dual_set_outlet if dual else L.orc_set_outlet)(h, int(outlet)) != 0:
            raise OracleError("outlet must be 0 (linear) or 1 (zero-gradient)")
        # inlet velocity profile: 0 uniform, 1 parabolic across the channel (mean 1)
        if (L.orc_dual_set_inlet_profile if dual else L.orc_set_inlet_profile)(h, int(inlet_profile)) != 0:
            raise OracleError("inlet_profile must be 0 (uniform) or 1 (parabolic)")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            (lib().orc_dual_destroy if self.dual else lib().orc_destroy)(h)
            self.h = None

    # ------------------------------------------------------------------
    def set_link_q(self, user_elem, direction, q):
        """Wall distance q in (0, 1] of obstacle links (user element index,
        direction i with x - c_i solid): the wall lies at x - q c_i."""
        ue = np.ascontiguousarray(user_elem, dtype=np.int64)
        dr = np.ascontiguousarray(direction, dtype=np.int32)
        qq = np.ascontiguousarray(q, dtype=np.float64)
        fn = lib().orc_dual_set_link_q if self.dual else lib().orc_set_link_q
        if fn(self.h, len(ue), _p(ue), _p(dr), _p(qq)) != 0:
            raise OracleError("set_link_q: not an obstacle link, or q outside (0, 1]")

    def counts(self):
        out = np.zeros((16, 6), dtype=np.int64)
        n = lib().orc_counts(self.h, _p(out), 16)
        return out[:n]

    def level_omega(self, li):
        return lib().orc_level_omega(self.h, li)

    def init(self, rho, u, S=None, df=None):
        rho = _f64(rho, (self.n,))
        u = _f64(u, (self.n, self.d))
        S = _f64(S, (self.n, self.ns))
        df = _f64(df, (self.n, self.Q))
        fn = lib().orc_dual_init if self.dual else lib().orc_init
        fn(self.h, _p(rho), _p(u), _p(S), _p(df))

    def set_force(self, F, F_dot=None):
        F = _f64(F, (self.n, self.d))
        if self.dual:
            lib().orc_dual_set_force(self.h, _p(F), _p(_f64(F_dot, (self.n, self.d))))
        else:
            lib().orc_set_force(self.h, _p(F))

    def step(self, n=1):
        (lib().orc_dual_step if self.dual else lib().orc_step)(self.h, int(n))

    def fill_ghosts(self):
        lib().orc_fill_ghosts(self.h)

    OP_GFF, OP_MOM_A, OP_GFC_A, OP_SC, OP_MOM_B, OP_GFC_B = range(6)

    def op(self, op, level):
        """One op of the recursive step (see orc_op), for drivers that put
        their own work between the ops."""
        if lib().orc_op(self.h, int(op), int(level)) != 0:
            raise OracleError(f"op {op} does not apply on level {level}")

    def nlev(self):
        return int(lib().orc_nlev(self.h))

    def moments(self):
        rho = np.zeros(self.n)
        u = np.zeros((self.n, self.d))
        S = np.zeros((self.n, self.ns))
        lib().orc_moments(self.h, _p(rho), _p(u), _p(S))
        return rho, u, S

    def get_f(self):
        f = np.zeros((self.n, self.Q))
        lib().orc_get_f(self.h, _p(f))
        return f

    def set_f(self, f, f_dot=None):
        """Set the fluid pdfs (dual twin: with tangents f_dot, default zero)."""
        f = _f64(f, (self.n, self.Q))
        if self.dual:
            lib().orc_dual_set_f(self.h, _p(f), _p(_f64(f_dot, (self.n, self.Q))))
        else:
            lib().orc_set_f(self.h, _p(f))

    def ghosts(self):
        n = lib().orc_ghost_count(self.h)
        info = np.zeros((n, 6), dtype=np.int64)
        f = np.zeros((n, self.Q))
        lib().orc_ghosts(self.h, _p(info), _p(f))
        return info, f

    def reduce(self):
        out = np.zeros(8)
        if self.dual:
            dot = np.zeros(8)
            lib().orc_dual_reduce(self.h, _p(out), _p(dot))
            return out, dot
        lib().orc_reduce(self.h, _p(out))
        return out


def compact_velocity(d, signs, u4, S4):
    """Compact quadratic velocity at one ghost (global frame inputs)."""
    s = np.ascontiguousarray(signs, dtype=np.int32)
    u4 = _f64(u4, (4, d))
    S4 = _f64(S4, (4, 3 if d == 2 else 6))
    out = np.zeros(d)
    if lib().orc_compact_velocity(d, _p(s), _p(u4), _p(S4), _p(out)) != 0:
        raise OracleError("bad dimension")
    return out
