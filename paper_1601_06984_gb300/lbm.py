"""Thin ctypes binding of liblbm (include/lbm.h).

Argument marshalling only: every step of the method runs inside liblbm's CUDA
kernels.  PyTorch supplies the device workspace and the CUDA stream.  There is
no CPU fallback: if liblbm.so is missing or was built for another machine,
importing the library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_OK = 0
STATUS = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_MESH", -3: "LBM_ERR_CUDA", -4: "LBM_ERR_OOM",
          -5: "LBM_ERR_STATE", -6: "LBM_ERR_NUMERIC", -7: "LBM_ERR_INTERNAL"}
FP64, FP32DEV, BF16DEV = 0, 1, 2
TIME_LINEAR, TIME_TWO_LAYER, TIME_DIFFUSIVE = 0, 1, 2
OUTLET_LINEAR, OUTLET_ZERO_GRADIENT = 0, 1
INLET_UNIFORM, INLET_PARABOLIC = 0, 1
EXPORTS = ["lbm_build_mesh", "lbm_mesh_info", "lbm_device_bytes", "lbm_bind", "lbm_init", "lbm_set_force",
           "lbm_step", "lbm_fill_ghosts", "lbm_moments", "lbm_reduce", "lbm_get_state", "lbm_set_state", "lbm_ghost_count",
           "lbm_get_ghosts", "lbm_sfc_partition", "lbm_kernel_launches", "lbm_timing_enable", "lbm_timing_read",
           "lbm_reduce_noalloc", "lbm_set_params", "lbm_adjoint_bytes", "lbm_adjoint", "lbm_last_error",
           "lbm_destroy", "lbm_obstacle_links", "lbm_set_link_q", "lbm_alu_peak", "lbm_halo_plan"]


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class lbm_params(C.Structure):
    _fields_ = [("stencil", C.c_int32), ("precision", C.c_int32), ("time_mode", C.c_int32),
                ("extent", C.c_int32 * 3), ("bc", C.c_int32 * 6), ("omega_coarse", C.c_double),
                ("rho0", C.c_double), ("u_in", C.c_double * 3), ("use_force", C.c_int32),
                ("outlet", C.c_int32), ("inlet_profile", C.c_int32), ("bouzidi", C.c_int32),
                ("n_levels", C.c_int32), ("check_every", C.c_int32), ("mass_band", C.c_double),
                ("adjoint_tape", C.c_int32)]


_lib = None


def lib():
    """Load liblbm.so (raises OSError if it is absent: build it with build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} not found: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        P, I64, I32, U64 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64
        sig = {
            "lbm_build_mesh": [P, P, I64, C.POINTER(lbm_params), C.POINTER(P)],
            "lbm_mesh_info": [P, P, I32, P],
            "lbm_device_bytes": [P, C.POINTER(U64)],
            "lbm_bind": [P, P, U64, P],
            "lbm_init": [P, P, P, P, P],
            "lbm_set_force": [P, P],
            "lbm_step": [P, I64],
            "lbm_fill_ghosts": [P],
            "lbm_moments": [P, P, P, P],
            "lbm_reduce": [P, P],
            "lbm_get_state": [P, P],
            "lbm_set_state": [P, P],
            "lbm_ghost_count": [P, C.POINTER(I64)],
            "lbm_get_ghosts": [P, P, P],
            "lbm_sfc_partition": [P, I64, I32, I32, P, P, P, P],
            "lbm_kernel_launches": [P, C.POINTER(I64)],
            "lbm_timing_enable": [P, I32],
            "lbm_timing_read": [P, P, P, I32],
            "lbm_reduce_noalloc": [P, P],
            "lbm_set_params": [P, C.c_double, P],
            "lbm_adjoint_bytes": [P, I64, I32, C.POINTER(U64)],
            "lbm_adjoint": [P, I64, I32, I32, P, U64, P, P, P, P, P],
            "lbm_obstacle_links": [P, P, P, I64, C.POINTER(I64)],
            "lbm_set_link_q": [P, P, I64],
            "lbm_alu_peak": [I32, P, U64, P],
            "lbm_halo_plan": [P, P, I32, I32, P, P, I64, P, P, I64],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.lbm_last_error.argtypes = [P]
        L.lbm_last_error.restype = C.c_char_p
        L.lbm_destroy.argtypes = [P]
        L.lbm_destroy.restype = None
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _arr(a, dtype, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(ctx, status):
    if status != LBM_OK:
        msg = lib().lbm_last_error(ctx).decode() if ctx else ""
        raise LBMError(status, msg)


# ---------------------------------------------------------------- C-named wrappers
def lbm_build_mesh(tree_ids, levels, params: lbm_params):
    tid = _arr(tree_ids, np.int64)
    lv = _arr(levels, np.int8)
    ctx = C.c_void_p()
    st = lib().lbm_build_mesh(_p(tid), _p(lv), tid.shape[0], C.byref(params), C.byref(ctx))
    if st != LBM_OK:
        msg = lib().lbm_last_error(ctx).decode() if ctx else ""
        if ctx:
            lib().lbm_destroy(ctx)
        raise LBMError(st, msg)
    return ctx


def lbm_sfc_partition(tree_ids, d, nparts):
    tid = _arr(tree_ids, np.int64)
    n = tid.shape[0]
    order = np.zeros(n, np.int64)
    w = np.zeros(n, np.int64)
    cum = np.zeros(n, np.int64)
    part = np.zeros(n, np.int32)
    _check(None, lib().lbm_sfc_partition(_p(tid), n, d, nparts, _p(order), _p(w), _p(cum), _p(part)))
    return order, w, cum, part


def lbm_alu_peak(precision, device="cuda"):
    """Measured multiply-add rate (GFLOP/s) of the device for FP64 or FP32
    (precision FP64 / FP32DEV)."""
    import torch
    dev = torch.device(device)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    scratch = torch.empty(16 * sms * 256 * 8, dtype=torch.uint8, device=dev)
    out = C.c_double()
    with torch.cuda.device(dev):
        _check(None, lib().lbm_alu_peak(int(precision), C.c_void_p(scratch.data_ptr()), scratch.numel(),
                                        C.byref(out)))
    return float(out.value)


def lbm_reduce_noalloc(sim):
    """FP64 reductions of a bound simulation through the entry point that
    allocates nothing (its scratch is a static device array of the library)."""
    out = np.zeros(8)
    _check(sim.ctx, lib().lbm_reduce_noalloc(sim.ctx, _p(out)))
    return out


# ---------------------------------------------------------------- convenience
class Sim:
    """One multilevel simulation in liblbm.  mesh: an object with tree_ids,
    levels, extent, bc (e.g. workloads.Mesh).  device=None builds the mesh on
    the host only (no GPU needed); otherwise a torch CUDA device."""

    def __init__(self, mesh, stencil, omega_c, precision=FP64, time_mode=TIME_LINEAR, rho0=1.0,
                 u_in=(0.0, 0.0, 0.0), use_force=False, device="cuda", stream=None, outlet=OUTLET_LINEAR,
                 inlet_profile=INLET_UNIFORM, bouzidi=False, n_levels=0, check_every=0, mass_band=0.0,
                 adjoint_tape=0):
        self.d = 2 if stencil == 9 else 3
        self.Q = stencil
        self.ns = 3 if self.d == 2 else 6
        self.n = int(len(mesh.tree_ids))
        p = lbm_params()
        p.stencil, p.precision, p.time_mode = stencil, precision, time_mode
        ext = list(mesh.extent) + [1] * (3 - len(mesh.extent))
        bc = list(mesh.bc) + [0] * (6 - len(mesh.bc))
        for a in range(3):
            p.extent[a] = int(ext[a])
            p.u_in[a] = float((list(u_in) + [0.0] * 3)[a])
        for f in range(6):
            p.bc[f] = int(bc[f])
        p.omega_coarse, p.rho0, p.use_force = float(omega_c), float(rho0), int(bool(use_force))
        p.outlet = int(outlet)
        p.inlet_profile = int(inlet_profile)
        p.bouzidi = int(bool(bouzidi))
        p.n_levels, p.check_every, p.mass_band = int(n_levels), int(check_every), float(mass_band)
        p.adjoint_tape = int(adjoint_tape)
        self.params = p
        self.ctx = lbm_build_mesh(mesh.tree_ids, mesh.levels, p)
        self.ws = None
        self.stream = None
        if device is not None:
            self.bind(device, stream)

    def bind(self, device="cuda", stream=None):
        import torch
        nbytes = C.c_uint64()
        _check(self.ctx, lib().lbm_device_bytes(self.ctx, C.byref(nbytes)))
        self.ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.ws.device)
        _check(self.ctx, lib().lbm_bind(self.ctx, C.c_void_p(self.ws.data_ptr()), nbytes.value,
                                        C.c_void_p(self.stream.cuda_stream)))

    def close(self):
        if getattr(self, "ctx", None):
            lib().lbm_destroy(self.ctx)
            self.ctx = None
        self.ws = None

    def __del__(self):
        self.close()

    # -- queries
    def halo_plan(self, part, nparts, rank):
        """Sec. 3.1/3.2 halo plan of part `rank` for the owner array part[n]
        (caller order): {sending part: caller indices to receive (ascending)}
        and the rows (lbm_get_ghosts order) of the ghosts the part fills."""
        part = _arr(part, np.int32, (self.n,))
        counts = np.zeros(nparts, np.int64)
        ng = C.c_int64()
        _check(self.ctx, lib().lbm_halo_plan(self.ctx, _p(part), int(nparts), int(rank), _p(counts), None, 0,
                                             C.byref(ng), None, 0))
        recv = np.zeros(int(counts.sum()), np.int64)
        ghosts = np.zeros(ng.value, np.int64)
        _check(self.ctx, lib().lbm_halo_plan(self.ctx, _p(part), int(nparts), int(rank), _p(counts), _p(recv),
                                             len(recv), C.byref(ng), _p(ghosts), len(ghosts)))
        start = np.concatenate([[0], np.cumsum(counts)])
        return {p: recv[start[p]:start[p + 1]] for p in range(nparts) if counts[p] > 0}, ghosts

    def mesh_info(self):
        info = np.zeros((32, 10), np.int64)
        nl = C.c_int32()
        _check(self.ctx, lib().lbm_mesh_info(self.ctx, _p(info), 32, C.byref(nl)))
        return info[: nl.value]

    def obstacle_links(self):
        """(caller element index [m], direction [m]) of the links x -> x - c_i
        into solid cells, in the order lbm_set_link_q expects."""
        n = C.c_int64()
        _check(self.ctx, lib().lbm_obstacle_links(self.ctx, None, None, 0, C.byref(n)))
        elem = np.zeros(n.value, np.int64)
        dr = np.zeros(n.value, np.int8)
        _check(self.ctx, lib().lbm_obstacle_links(self.ctx, _p(elem), _p(dr), n.value, C.byref(n)))
        return elem, dr

    def set_link_q(self, q):
        """Wall distance q in (0, 1] per obstacle link (wall at x - q c_i)."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        _check(self.ctx, lib().lbm_set_link_q(self.ctx, _p(q), len(q)))

    def device_bytes(self):
        nbytes = C.c_uint64()
        _check(self.ctx, lib().lbm_device_bytes(self.ctx, C.byref(nbytes)))
        return int(nbytes.value)

    def kernel_launches(self):
        n = C.c_int64()
        _check(self.ctx, lib().lbm_kernel_launches(self.ctx, C.byref(n)))
        return int(n.value)

    def timing_enable(self, mode=1):
        """0 off; 1 every kernel timed, steps launched kernel by kernel; 2 steps
        replay the captured graphs, which time the finest level's
        stream-collide launches (read back: the most recent replay)."""
        _check(self.ctx, lib().lbm_timing_enable(self.ctx, int(mode)))

    TIMED_KINDS = ("interior", "list", "boundary", "gff", "moments", "gfc", "outlet", "sc_span")

    def timing_read(self):
        """Launches and summed device ms since enabled, arrays [level, kind]
        with kind 0 = interior-brick stream-collide, 1 = neighbour-list
        stream-collide, 2 = boundary-brick stream-collide, 3 = GhostFromFiner,
        4 = source moments, 5 = GhostFromCoarser, 6 = outlet values."""
        k = len(self.TIMED_KINDS)
        n = np.zeros(16 * k, np.int64)
        ms = np.zeros(16 * k)
        _check(self.ctx, lib().lbm_timing_read(self.ctx, _p(n), _p(ms), 16 * k))
        nl = len(self.mesh_info())
        return n[: k * nl].reshape(nl, k), ms[: k * nl].reshape(nl, k)

    # -- state
    def init(self, rho, u, S=None, df=None):
        rho = _arr(rho, np.float64, (self.n,))
        u = _arr(u, np.float64, (self.n, self.d))
        S = _arr(S, np.float64, (self.n, self.ns))
        df = _arr(df, np.float64, (self.n, self.Q))
        _check(self.ctx, lib().lbm_init(self.ctx, _p(rho), _p(u), _p(S), _p(df)))

    def set_force(self, F):
        F = _arr(F, np.float64, (self.n, self.d))
        _check(self.ctx, lib().lbm_set_force(self.ctx, _p(F)))

    def step(self, n=1):
        _check(self.ctx, lib().lbm_step(self.ctx, int(n)))

    def fill_ghosts(self):
        _check(self.ctx, lib().lbm_fill_ghosts(self.ctx))

    def moments(self, out=None):
        if out is None:
            out = (np.empty(self.n), np.empty((self.n, self.d)), np.empty((self.n, self.ns)))
        rho, u, S = out
        _check(self.ctx, lib().lbm_moments(self.ctx, _p(rho), _p(u), _p(S)))
        return rho, u, S

    def get_state(self):
        f = np.empty((self.n, self.Q))
        _check(self.ctx, lib().lbm_get_state(self.ctx, _p(f)))
        return f

    def set_state(self, f):
        f = _arr(f, np.float64, (self.n, self.Q))
        _check(self.ctx, lib().lbm_set_state(self.ctx, _p(f)))

    def ghosts(self):
        n = C.c_int64()
        _check(self.ctx, lib().lbm_ghost_count(self.ctx, C.byref(n)))
        info = np.zeros((n.value, 6), np.int64)
        f = np.zeros((n.value, self.Q))
        if n.value:
            _check(self.ctx, lib().lbm_get_ghosts(self.ctx, _p(info), _p(f)))
        return info, f

    def ghost_count(self):
        n = C.c_int64()
        _check(self.ctx, lib().lbm_ghost_count(self.ctx, C.byref(n)))
        return int(n.value)

    def reduce(self):
        out = np.zeros(8)
        _check(self.ctx, lib().lbm_reduce(self.ctx, _p(out)))
        return out

    def set_params(self, omega_c, u_in=None):
        uin = None if u_in is None else _arr(list(u_in) + [0.0] * (3 - len(u_in)), np.float64)
        _check(self.ctx, lib().lbm_set_params(self.ctx, float(omega_c), _p(uin)))

    def adjoint_bytes(self, n_coarse, K=20):
        nbytes = C.c_uint64()
        _check(self.ctx, lib().lbm_adjoint_bytes(self.ctx, int(n_coarse), int(K), C.byref(nbytes)))
        return int(nbytes.value)

    def adjoint(self, n_coarse, K=20, objective=0, want_force=True, want_f0=False):
        """Discrete adjoint of n_coarse steps from the current state (gradients
        at fixed initial pdfs).  Returns (J, dJ/dF [n, d] or None, dJ/domega_c,
        dJ/du_in [3]) and, with want_f0, dJ/d(initial pdfs) [n, Q] last."""
        import torch
        nbytes = C.c_uint64()
        _check(self.ctx, lib().lbm_adjoint_bytes(self.ctx, int(n_coarse), int(K), C.byref(nbytes)))
        ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.ws.device)
        J = C.c_double()
        dF = np.zeros((self.n, self.d)) if want_force else None
        dw = C.c_double()
        du = np.zeros(3)
        df0 = np.zeros((self.n, self.Q)) if want_f0 else None
        _check(self.ctx, lib().lbm_adjoint(self.ctx, int(n_coarse), int(K), int(objective),
                                           C.c_void_p(ws.data_ptr()), nbytes.value, C.byref(J), _p(dF),
                                           C.byref(dw), _p(du), _p(df0)))
        del ws
        if want_f0:
            return J.value, dF, dw.value, du, df0
        return J.value, dF, dw.value, du
