"""Python binding of the C ABI in include/lbrbc.h (argument marshalling only).

Every time step runs in the CUDA kernels of ``_lib/liblbrbc.so``; this module
never computes any part of the method.  If the library has not been built, or
cannot be loaded, every entry point raises: there is no CPU fallback.

Functions with the C names (``lbrbc_create`` ...) take and return ctypes
values; the ``Sim`` class wraps them for numpy / torch callers.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbrbc.so")

LBRBC_OK, LBRBC_ERR_ARG, LBRBC_ERR_CUDA, LBRBC_ERR_NUMERIC = 0, 1, 2, 3
LBRBC_ERR_TIMEOUT, LBRBC_ERR_STATE, LBRBC_ERR_UNSUPPORTED = 4, 5, 6
BC = {"periodic": 0, "wall": 1, "open": 2}
SCHEME = {"new": 0, "verhaeghe": 1, "patel_ju": 2, "anti_bb": 3}
PRECISION = {"fp32": 0, "fp64": 1}
LAYOUT = {"auto": 0, "dense": 1, "sparse": 2}
CLASS_FLUID, CLASS_BOUND, CLASS_SOLID = 0, 1, 2
EV_DISSOLVE, EV_PRECIPITATE = 1, 2


class lbrbc_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("flow_q", ctypes.c_int), ("solute_q", ctypes.c_int), ("bc", ctypes.c_int * 3),
        ("scheme", ctypes.c_int), ("phase_change", ctypes.c_int), ("precision", ctypes.c_int),
        ("event_log_capacity", ctypes.c_int),
        ("tau_flow", ctypes.c_double), ("magic_flow", ctypes.c_double), ("tau_solute", ctypes.c_double),
        ("magic_solute", ctypes.c_double), ("rest_fraction", ctypes.c_double), ("k_r", ctypes.c_double),
        ("c_eq", ctypes.c_double), ("molar_volume", ctypes.c_double), ("c_init", ctypes.c_double),
        ("rho_init", ctypes.c_double), ("c_dirichlet", ctypes.c_double), ("c_inlet", ctypes.c_double),
        ("u_inlet", ctypes.c_double), ("rho_outlet", ctypes.c_double), ("layout", ctypes.c_int),
    ]


class lbrbc_init(ctypes.Structure):
    _fields_ = [(n, ctypes.POINTER(ctypes.c_double)) for n in
                ("k_field", "c_init", "u_init", "phi_init", "inlet_ux")]


class LbrbcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("lbrbc status %d: %s" % (status, msg))
        self.status = status


_lib = None

EXPORTED = ["lbrbc_create", "lbrbc_step", "lbrbc_fields", "lbrbc_classes", "lbrbc_mass_ledger",
            "lbrbc_mass_ledger_noalloc", "lbrbc_noalloc_size_check",
            "lbrbc_events", "lbrbc_adjoint", "lbrbc_profile_step", "lbrbc_info", "lbrbc_launch_counts", "lbrbc_layout_info", "lbrbc_check", "lbrbc_last_error",
            "lbrbc_destroy", "lbrbc_batch_create", "lbrbc_batch_step", "lbrbc_batch_autotune", "lbrbc_batch_schedule",
            "lbrbc_batch_info", "lbrbc_batch_domain", "lbrbc_batch_last_error", "lbrbc_batch_destroy"]


def load(path: str = LIB_PATH):
    """Load the compiled library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("liblbrbc.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, dp = ctypes.c_void_p, P(ctypes.c_double)
    lib.lbrbc_create.restype = ctypes.c_int
    lib.lbrbc_create.argtypes = [P(lbrbc_params), P(ctypes.c_uint8), P(lbrbc_init), P(vp)]
    lib.lbrbc_step.restype = ctypes.c_int
    lib.lbrbc_step.argtypes = [vp, ctypes.c_int64, vp]
    lib.lbrbc_fields.restype = ctypes.c_int
    lib.lbrbc_fields.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int]
    lib.lbrbc_classes.restype = ctypes.c_int
    lib.lbrbc_classes.argtypes = [vp, P(ctypes.c_uint8)]
    lib.lbrbc_mass_ledger.restype = ctypes.c_int
    lib.lbrbc_mass_ledger.argtypes = [vp, dp]
    lib.lbrbc_mass_ledger_noalloc.restype = ctypes.c_int
    lib.lbrbc_mass_ledger_noalloc.argtypes = [vp, dp]
    lib.lbrbc_noalloc_size_check.restype = ctypes.c_int
    lib.lbrbc_noalloc_size_check.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_char_p,
                                             ctypes.c_int32]
    lib.lbrbc_events.restype = ctypes.c_int
    lib.lbrbc_events.argtypes = [vp, P(ctypes.c_int64), ctypes.c_int64, P(ctypes.c_int64), P(ctypes.c_int64),
                                 P(ctypes.c_int32)]
    lib.lbrbc_adjoint.restype = ctypes.c_int
    lib.lbrbc_adjoint.argtypes = [vp, ctypes.c_int64, dp, dp, dp, dp]
    lib.lbrbc_profile_step.restype = ctypes.c_int
    lib.lbrbc_profile_step.argtypes = [vp, ctypes.c_int64, vp, dp, P(ctypes.c_int64)]
    lib.lbrbc_info.restype = ctypes.c_int
    lib.lbrbc_info.argtypes = [vp, P(ctypes.c_int64)]
    lib.lbrbc_layout_info.restype = ctypes.c_int
    lib.lbrbc_layout_info.argtypes = [vp, P(ctypes.c_int64)]
    lib.lbrbc_launch_counts.restype = ctypes.c_int
    lib.lbrbc_launch_counts.argtypes = [vp, P(ctypes.c_int64)]
    lib.lbrbc_check.restype = ctypes.c_int
    lib.lbrbc_check.argtypes = [vp]
    lib.lbrbc_last_error.restype = ctypes.c_char_p
    lib.lbrbc_last_error.argtypes = [vp]
    lib.lbrbc_destroy.restype = None
    lib.lbrbc_destroy.argtypes = [vp]
    lib.lbrbc_batch_create.restype = ctypes.c_int
    lib.lbrbc_batch_create.argtypes = [ctypes.c_int32, P(lbrbc_params), P(P(ctypes.c_uint8)), P(lbrbc_init), P(vp)]
    lib.lbrbc_batch_step.restype = ctypes.c_int
    lib.lbrbc_batch_step.argtypes = [vp, ctypes.c_int64, vp]
    lib.lbrbc_batch_autotune.restype = ctypes.c_int
    lib.lbrbc_batch_autotune.argtypes = [vp, ctypes.c_int32, vp, P(ctypes.c_int64), dp]
    lib.lbrbc_batch_schedule.restype = ctypes.c_int
    lib.lbrbc_batch_schedule.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    lib.lbrbc_batch_info.restype = ctypes.c_int
    lib.lbrbc_batch_info.argtypes = [vp, P(ctypes.c_int64)]
    lib.lbrbc_batch_domain.restype = vp
    lib.lbrbc_batch_domain.argtypes = [vp, ctypes.c_int32]
    lib.lbrbc_batch_last_error.restype = ctypes.c_char_p
    lib.lbrbc_batch_last_error.argtypes = [vp]
    lib.lbrbc_batch_destroy.restype = None
    lib.lbrbc_batch_destroy.argtypes = [vp]
    _lib = lib
    return lib


def _check(lib, handle, st):
    if st != LBRBC_OK:
        raise LbrbcError(st, lib.lbrbc_last_error(handle).decode())


# Thin wrappers with the C names -------------------------------------------------
def lbrbc_create(params: lbrbc_params, mask: np.ndarray, init: lbrbc_init | None = None):
    lib = load()
    h = ctypes.c_void_p()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    st = lib.lbrbc_create(ctypes.byref(params), m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                          ctypes.byref(init) if init is not None else None, ctypes.byref(h))
    _check(lib, None, st)
    return h


def lbrbc_step(handle, n: int, stream: int | None = None):
    lib = load()
    _check(lib, handle, lib.lbrbc_step(handle, int(n), ctypes.c_void_p(stream) if stream else None))


def lbrbc_fields(handle, u=None, rho=None, c=None, phi=None, device: bool = False):
    """Pointers as ints (device) or numpy float64 arrays (host)."""
    lib = load()

    def ptr(a):
        if a is None:
            return None
        if isinstance(a, int):
            return ctypes.c_void_p(a)
        return ctypes.c_void_p(a.ctypes.data)

    _check(lib, handle, lib.lbrbc_fields(handle, ptr(u), ptr(rho), ptr(c), ptr(phi), int(device)))


def lbrbc_classes(handle, out: np.ndarray):
    lib = load()
    _check(lib, handle, lib.lbrbc_classes(handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))


def lbrbc_mass_ledger(handle):
    lib = load()
    out = np.zeros(6)
    _check(lib, handle, lib.lbrbc_mass_ledger(handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def lbrbc_mass_ledger_noalloc(handle):
    """Same values as lbrbc_mass_ledger, computed without device allocation."""
    lib = load()
    out = np.zeros(6)
    _check(lib, handle, lib.lbrbc_mass_ledger_noalloc(handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def lbrbc_noalloc_size_check(n_cells: int, max_blocks: int = 4096, cells_per_block: int = 65536):
    """(status, message) of the size rule of lbrbc_mass_ledger_noalloc (host only)."""
    lib = load()
    buf = ctypes.create_string_buffer(256)
    st = lib.lbrbc_noalloc_size_check(int(n_cells), int(max_blocks), int(cells_per_block), buf, len(buf))
    return st, buf.value.decode()


def lbrbc_events(handle):
    lib = load()
    n = ctypes.c_int64()
    _check(lib, handle, lib.lbrbc_events(handle, ctypes.byref(n), 0, None, None, None))
    k = n.value
    st, nd, kd = np.zeros(k, np.int64), np.zeros(k, np.int64), np.zeros(k, np.int32)
    if k:
        P = ctypes.POINTER
        _check(lib, handle, lib.lbrbc_events(handle, ctypes.byref(n), k, st.ctypes.data_as(P(ctypes.c_int64)),
                                             nd.ctypes.data_as(P(ctypes.c_int64)),
                                             kd.ctypes.data_as(P(ctypes.c_int32))))
    return st, nd, kd


def lbrbc_adjoint(handle, n_steps: int, field: bool = False, N: int = 0):
    """(J, dJ/dk_r, dJ/dc_eq, dJ/dk_r(cell) or None) over the next n_steps steps."""
    lib = load()
    J, dk, dc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    kf = np.zeros(N) if field else None
    _check(lib, handle, lib.lbrbc_adjoint(handle, int(n_steps), ctypes.byref(J), ctypes.byref(dk), ctypes.byref(dc),
                                          kf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if field else None))
    return J.value, dk.value, dc.value, kf


def lbrbc_profile_step(handle, n: int, stream: int | None = None):
    """(ms per step of [fluid, boundary, fluid-end, phase-change] kernels, launches per step)."""
    lib = load()
    ms = np.zeros(4)
    nl = ctypes.c_int64()
    _check(lib, handle, lib.lbrbc_profile_step(handle, int(n), ctypes.c_void_p(stream) if stream else None,
                                               ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(nl)))
    return ms, nl.value


def lbrbc_info(handle):
    lib = load()
    out = (ctypes.c_int64 * 3)()
    _check(lib, handle, lib.lbrbc_info(handle, out))
    return dict(fluid_cells=out[0], boundary_cells=out[1], launches_per_step=out[2])


def lbrbc_launch_counts(handle):
    lib = load()
    out = (ctypes.c_int64 * 2)()
    _check(lib, handle, lib.lbrbc_launch_counts(handle, out))
    return dict(per_step=out[0], per_event_step=out[1])


def lbrbc_layout_info(handle):
    lib = load()
    out = (ctypes.c_int64 * 4)()
    _check(lib, handle, lib.lbrbc_layout_info(handle, out))
    return dict(layout={1: "dense", 2: "sparse"}.get(out[0], str(out[0])), stored_cells=out[1], repacks=out[2],
                population_bytes=out[3])


def lbrbc_check(handle):
    lib = load()
    _check(lib, handle, lib.lbrbc_check(handle))


def lbrbc_last_error(handle=None) -> str:
    return load().lbrbc_last_error(handle).decode()


def lbrbc_destroy(handle):
    if handle:
        load().lbrbc_destroy(handle)


def _current_device() -> int:
    """CUDA device current in this thread (the one lbrbc_create used)."""
    try:
        import torch

        return int(torch.cuda.current_device()) if torch.cuda.is_available() else 0
    except Exception:
        return 0


# Convenience wrapper -------------------------------------------------------------
DEFAULTS = dict(dim=3, nx=8, ny=8, nz=8, flow_q=19, solute_q=7, bc=("periodic", "periodic", "periodic"),
                scheme="new", phase_change=0, precision="fp32", event_log_capacity=0, tau_flow=0.8,
                magic_flow=-1.0, tau_solute=0.8, magic_solute=-1.0, rest_fraction=-1.0, k_r=0.0, c_eq=0.0,
                molar_volume=1.0, c_init=0.0, rho_init=1.0, c_dirichlet=0.0, c_inlet=0.0, u_inlet=0.0,
                rho_outlet=1.0, layout="auto")


def make_params(p: dict) -> lbrbc_params:
    """ctypes parameter block from a dict (missing keys take DEFAULTS).  When
    the dict names no layout, the environment variable LBRBC_LAYOUT (auto,
    dense or sparse) chooses it, so a whole test run can be repeated on
    either population layout."""
    q = dict(DEFAULTS)
    if "layout" not in p and os.environ.get("LBRBC_LAYOUT"):
        q["layout"] = os.environ["LBRBC_LAYOUT"]
    q.update(p)
    s = lbrbc_params()
    for k in ("dim", "nx", "ny", "nz", "flow_q", "solute_q", "phase_change", "event_log_capacity"):
        setattr(s, k, int(q[k]))
    if q["dim"] == 2:
        s.nz = 1
    for a in range(3):
        s.bc[a] = BC[q["bc"][a]] if isinstance(q["bc"][a], str) else int(q["bc"][a])
    s.scheme = SCHEME[q["scheme"]] if isinstance(q["scheme"], str) else int(q["scheme"])
    s.precision = PRECISION[q["precision"]] if isinstance(q["precision"], str) else int(q["precision"])
    s.layout = LAYOUT[q["layout"]] if isinstance(q["layout"], str) else int(q["layout"])
    for k in ("tau_flow", "magic_flow", "tau_solute", "magic_solute", "rest_fraction", "k_r", "c_eq",
              "molar_volume", "c_init", "rho_init", "c_dirichlet", "c_inlet", "u_inlet", "rho_outlet"):
        setattr(s, k, float(q[k]))
    return s


def _host(a):
    """numpy view of an array-like input; torch tensors (on any device) are
    copied to the host first (the library copies every input at creation)."""
    if hasattr(a, "detach") and hasattr(a, "cpu"):
        return a.detach().cpu().numpy()
    return a


class Sim:
    """One GPU simulation.  ``mask``: uint8 [z, y, x] (0 fluid, 1 reactive
    solid, 2 Dirichlet solid); optional init fields; numpy arrays or torch
    tensors."""

    def __init__(self, params: dict, mask, k_field=None, c_init=None, u_init=None, phi_init=None,
                 inlet_ux=None):
        self._lib = load()
        self._p = make_params(params)
        self.shape = (self._p.nz, self._p.ny, self._p.nx)
        self.N = int(np.prod(self.shape))
        m = np.ascontiguousarray(np.asarray(_host(mask), dtype=np.uint8).reshape(-1))
        if m.size != self.N:
            raise ValueError("mask size %d != grid %d" % (m.size, self.N))
        self._keep = {}
        ini = lbrbc_init()
        for name, arr, n in (("k_field", k_field, self.N), ("c_init", c_init, self.N), ("u_init", u_init, 3 * self.N),
                             ("phi_init", phi_init, self.N), ("inlet_ux", inlet_ux, self._p.ny * self._p.nz)):
            if arr is None:
                continue
            a = np.ascontiguousarray(np.asarray(_host(arr), dtype=np.float64).reshape(-1))
            if a.size != n:
                raise ValueError("%s has %d entries, expected %d" % (name, a.size, n))
            self._keep[name] = a
            setattr(ini, name, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        self._h = lbrbc_create(self._p, m, ini)
        self.device = _current_device()

    def step(self, n: int = 1, stream: int | None = None):
        lbrbc_step(self._h, n, stream)

    def fields(self, device: bool = False):
        """(u[z, y, x, 3], rho, c, phi) of the current state: numpy arrays on
        the host, or with device=True float64 torch tensors on the
        simulation's GPU, filled there by the library (no host copy)."""
        s = self.shape
        if device:
            import torch

            dev = torch.device("cuda", self.device)
            u = torch.empty(s + (3,), dtype=torch.float64, device=dev)
            rho, c, phi = (torch.empty(s, dtype=torch.float64, device=dev) for _ in range(3))
            self.fields_device(u, rho, c, phi)
            return u, rho, c, phi
        u = np.zeros(3 * self.N)
        rho, c, phi = np.zeros(self.N), np.zeros(self.N), np.zeros(self.N)
        lbrbc_fields(self._h, u, rho, c, phi)
        return u.reshape(s + (3,)), rho.reshape(s), c.reshape(s), phi.reshape(s)

    def fields_device(self, u=None, rho=None, c=None, phi=None):
        """Write into device buffers given as torch tensors (float64, cuda)."""
        ptr = lambda t: None if t is None else int(t.data_ptr())
        lbrbc_fields(self._h, ptr(u), ptr(rho), ptr(c), ptr(phi), device=True)

    def classes(self):
        out = np.zeros(self.N, np.uint8)
        lbrbc_classes(self._h, out)
        return out.reshape(self.shape)

    def ledger(self) -> dict:
        o = lbrbc_mass_ledger(self._h)
        return dict(solute=o[0], solid_over_vm=o[1], unpaid=o[2], dirichlet_in=o[3], reacted=o[4], step=int(o[5]))

    def events(self):
        st, nd, kd = lbrbc_events(self._h)
        return np.stack([st, nd, kd.astype(np.int64)], axis=1) if len(st) else np.zeros((0, 3), np.int64)

    def check(self):
        lbrbc_check(self._h)

    def adjoint(self, n_steps: int, field: bool = False):
        """Reacted mass over the next n_steps and its gradients (see lbrbc_adjoint)."""
        J, dk, dc, kf = lbrbc_adjoint(self._h, n_steps, field, self.N)
        return J, dk, dc, (kf.reshape(self.shape) if field else None)

    def profile(self, n: int, stream: int | None = None):
        return lbrbc_profile_step(self._h, n, stream)

    def info(self) -> dict:
        return lbrbc_info(self._h)

    def layout_info(self) -> dict:
        return lbrbc_layout_info(self._h)

    def launch_counts(self) -> dict:
        return lbrbc_launch_counts(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lbrbc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent 3D domains stepped together (one launch per kernel phase
    for the whole batch).  ``cases``: list of (params dict, mask, init dict)."""

    def __init__(self, cases):
        self._lib = load()
        n = len(cases)
        self._params = (lbrbc_params * n)()
        self._masks = (ctypes.POINTER(ctypes.c_uint8) * n)()
        self._inits = (lbrbc_init * n)()
        self._keep = []
        self.shapes = []
        for i, (p, mask, init) in enumerate(cases):
            self._params[i] = make_params(p)
            m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(-1))
            self._keep.append(m)
            self._masks[i] = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
            self.shapes.append((self._params[i].nz, self._params[i].ny, self._params[i].nx))
            for name, arr in (init or {}).items():
                a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(-1))
                self._keep.append(a)
                setattr(self._inits[i], name, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        h = ctypes.c_void_p()
        st = self._lib.lbrbc_batch_create(n, self._params, self._masks, self._inits, ctypes.byref(h))
        if st != LBRBC_OK:
            raise LbrbcError(st, self._lib.lbrbc_batch_last_error(None).decode())
        self._h = h

    def _chk(self, st):
        if st != LBRBC_OK:
            raise LbrbcError(st, self._lib.lbrbc_batch_last_error(self._h).decode())

    def step(self, n: int = 1, stream: int | None = None):
        self._chk(self._lib.lbrbc_batch_step(self._h, int(n), ctypes.c_void_p(stream) if stream else None))

    def autotune(self, pairs: int = 5, stream: int | None = None):
        ch = (ctypes.c_int64 * 3)()
        ms = ctypes.c_double()
        self._chk(self._lib.lbrbc_batch_autotune(self._h, int(pairs), ctypes.c_void_p(stream) if stream else None,
                                                 ch, ctypes.byref(ms)))
        return dict(tile_policy=ch[0], order=ch[1], blocks_per_sm=ch[2], ms_per_step=ms.value)

    def schedule(self, policy: int, order: int = 0, blocks_per_sm: int = 4):
        """Fix the schedule (the numbers autotune reports) without timing."""
        self._chk(self._lib.lbrbc_batch_schedule(self._h, int(policy), int(order), int(blocks_per_sm)))

    def info(self):
        out = (ctypes.c_int64 * 2)()
        self._chk(self._lib.lbrbc_batch_info(self._h, out))
        return dict(domains=out[0], fluid_cells=out[1])

    def domain(self, i: int):
        """Borrowed lbrbc_sim handle of domain i (fields, ledger, classes)."""
        h = self._lib.lbrbc_batch_domain(self._h, int(i))
        if not h:
            raise IndexError(i)
        return ctypes.c_void_p(h)

    def fields(self, i: int):
        N = int(np.prod(self.shapes[i]))
        u, rho, c, phi = np.zeros(3 * N), np.zeros(N), np.zeros(N), np.zeros(N)
        lbrbc_fields(self.domain(i), u, rho, c, phi)
        s = self.shapes[i]
        return u.reshape(s + (3,)), rho.reshape(s), c.reshape(s), phi.reshape(s)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbrbc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reacted_mass(params: dict, mask, n_steps: int, k_field=None, c_eq=None, **init):
    """Reacted mass over n_steps of a fresh simulation as a differentiable
    torch function of the per-cell rate field k_field (torch tensor shaped
    like the mask) and c_eq (0-d torch tensor).  The backward pass returns
    the discrete adjoint gradients computed by lbrbc_adjoint."""
    import torch

    class _ReactedMass(torch.autograd.Function):
        @staticmethod
        def forward(ctx, kf, ceq):
            p = dict(params)
            p["c_eq"] = float(ceq.detach().cpu())
            sim = Sim(p, mask, k_field=kf.detach().cpu().double().numpy(), **init)
            J, dk, dc, dkf = sim.adjoint(n_steps, field=True)
            sim.close()
            ctx.save_for_backward(torch.as_tensor(dkf, dtype=kf.dtype, device=kf.device),
                                  torch.as_tensor(dc, dtype=ceq.dtype, device=ceq.device))
            return torch.as_tensor(J, dtype=kf.dtype, device=kf.device)

        @staticmethod
        def backward(ctx, g):
            dkf, dc = ctx.saved_tensors
            return g * dkf, g * dc

    return _ReactedMass.apply(k_field, c_eq)
