"""FP64 CPU oracle of the coupled LBM step with the general local reactive
boundary condition (arXiv 2306.10794).

TEST INFRASTRUCTURE ONLY: this package exists so that ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` can check
the CUDA path against a plain, slow, obviously correct statement of the
method.  The product library never imports, links or executes anything here,
and nothing here imports the product package.

The arithmetic lives in ``lbrbc_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module only compiles it and marshals arguments
through ctypes.  Every function of the C file cites the section / equation of
the paper it follows.  Parity status of each part is listed in the module
``oracle.analytic`` docstring and in the test files that pin it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbrbc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbrbc_oracle.so")
_lock = threading.Lock()
_lib = None

BC = {"periodic": 0, "wall": 1, "open": 2}
SCHEME = {"new": 0, "verhaeghe": 1, "patel_ju": 2, "anti_bb": 3}
FLUID, BOUND, SOLID = 0, 1, 2
EV_DISSOLVE, EV_PRECIPITATE = 1, 2


class _Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("flow_q", ctypes.c_int), ("solute_q", ctypes.c_int), ("bc", ctypes.c_int * 3),
        ("scheme", ctypes.c_int), ("phase_change", ctypes.c_int),
        ("tau_flow", ctypes.c_double), ("magic_flow", ctypes.c_double),
        ("tau_solute", ctypes.c_double), ("magic_solute", ctypes.c_double),
        ("rest_fraction", ctypes.c_double), ("k_r", ctypes.c_double), ("c_eq", ctypes.c_double),
        ("molar_volume", ctypes.c_double), ("c_init", ctypes.c_double), ("rho_init", ctypes.c_double),
        ("c_dirichlet", ctypes.c_double), ("c_inlet", ctypes.c_double), ("u_inlet", ctypes.c_double),
        ("rho_outlet", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, no FMA contraction) into oracle/_build."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.POINTER
    dp, u8p, lp, ip = P(ctypes.c_double), P(ctypes.c_uint8), P(ctypes.c_long), P(ctypes.c_int)
    lib.orc_create.restype = ctypes.c_void_p
    lib.orc_create.argtypes = [P(_Params), u8p, dp, dp, dp, dp, dp]
    lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
    lib.orc_set_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.orc_adjoint.restype = ctypes.c_int
    lib.orc_adjoint.argtypes = [ctypes.c_void_p, ctypes.c_long, dp, dp, dp, dp]
    lib.orc_fields.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
    lib.orc_classes.argtypes = [ctypes.c_void_p, u8p]
    lib.orc_normals.argtypes = [ctypes.c_void_p, dp]
    lib.orc_ledger.argtypes = [ctypes.c_void_p, dp]
    lib.orc_reacted.argtypes = [ctypes.c_void_p, dp]
    lib.orc_event_count.restype = ctypes.c_long
    lib.orc_event_count.argtypes = [ctypes.c_void_p]
    lib.orc_events.argtypes = [ctypes.c_void_p, lp, lp, ip]
    lib.orc_destroy.argtypes = [ctypes.c_void_p]
    lib.orc_lattice.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ip, dp, dp, ip]
    lib.orc_equilibrium.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_double, dp, dp]
    lib.orc_rbc.restype = ctypes.c_double
    lib.orc_rbc.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    _lib = lib
    return lib


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


DEFAULTS = dict(dim=3, nx=8, ny=8, nz=8, flow_q=19, solute_q=7, bc=("periodic", "periodic", "periodic"),
                scheme="new", phase_change=0, tau_flow=0.8, magic_flow=-1.0, tau_solute=0.8,
                magic_solute=-1.0, rest_fraction=-1.0, k_r=0.0, c_eq=0.0, molar_volume=1.0,
                c_init=0.0, rho_init=1.0, c_dirichlet=0.0, c_inlet=0.0, u_inlet=0.0, rho_outlet=1.0)


def _params(p: dict) -> _Params:
    q = dict(DEFAULTS)
    q.update(p)
    s = _Params()
    for k in ("dim", "nx", "ny", "nz", "flow_q", "solute_q", "phase_change"):
        setattr(s, k, int(q[k]))
    if q["dim"] == 2:
        s.nz = 1
    for a in range(3):
        s.bc[a] = BC[q["bc"][a]] if isinstance(q["bc"][a], str) else int(q["bc"][a])
    s.scheme = SCHEME[q["scheme"]] if isinstance(q["scheme"], str) else int(q["scheme"])
    for k in ("tau_flow", "magic_flow", "tau_solute", "magic_solute", "rest_fraction", "k_r", "c_eq",
              "molar_volume", "c_init", "rho_init", "c_dirichlet", "c_inlet", "u_inlet", "rho_outlet"):
        setattr(s, k, float(q[k]))
    return s


class OracleSim:
    """One oracle simulation.  ``mask`` is a uint8 array indexed [z, y, x]
    (x fastest): 0 fluid, 1 reactive solid, 2 Dirichlet solid."""

    def __init__(self, params: dict, mask, k_field=None, c_init=None, u_init=None, phi_init=None,
                 inlet_ux=None):
        lib = _load()
        self.params = dict(DEFAULTS)
        self.params.update(params)
        self._p = _params(params)
        self.shape = (self._p.nz, self._p.ny, self._p.nx)
        self.N = int(np.prod(self.shape))
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(-1))
        if m.size != self.N:
            raise ValueError("mask size %d != grid %d" % (m.size, self.N))

        def opt(a, n):
            if a is None:
                return None
            a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
            if a.size != n:
                raise ValueError("optional field has %d entries, expected %d" % (a.size, n))
            return a

        self._keep = [opt(k_field, self.N), opt(c_init, self.N), opt(u_init, 3 * self.N),
                      opt(phi_init, self.N), opt(inlet_ux, self._p.ny * self._p.nz)]
        self._h = lib.orc_create(ctypes.byref(self._p), m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                 *[_dptr(a) for a in self._keep])
        if not self._h:
            raise ValueError("oracle rejected the lattice / rest-fraction combination")
        self._lib = lib

    def step(self, n: int = 1):
        self._lib.orc_step(self._h, int(n))

    def adjoint(self, n: int, field: bool = False):
        """Advance n steps and return (J, dJ/dk_r, dJ/dc_eq, dJ/dk(x) or None):
        J the reacted mass over those steps, the gradients by the oracle's
        discrete adjoint (phase change must be off)."""
        J, dk, dc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        g = np.zeros(self.N) if field else None
        rc = self._lib.orc_adjoint(self._h, int(n), ctypes.byref(J), ctypes.byref(dk), ctypes.byref(dc), _dptr(g))
        if rc:
            raise ValueError("oracle adjoint needs phase change off and n >= 1 (status %d)" % rc)
        return J.value, dk.value, dc.value, (g.reshape(self.shape) if field else None)

    def set_threads(self, n: int):
        """Run the per-cell loop as n z-slabs on n host threads (for timing
        the oracle on all cores; fields are unchanged, the ledger sums are
        added per slab)."""
        self._lib.orc_set_threads(self._h, int(n))

    def fields(self):
        """(u[z,y,x,3], rho, c, phi) of the current post-collision state."""
        u = np.zeros(3 * self.N)
        rho, c, phi = np.zeros(self.N), np.zeros(self.N), np.zeros(self.N)
        self._lib.orc_fields(self._h, _dptr(u), _dptr(rho), _dptr(c), _dptr(phi))
        s = self.shape
        return u.reshape(s + (3,)), rho.reshape(s), c.reshape(s), phi.reshape(s)

    def classes(self):
        out = np.zeros(self.N, dtype=np.uint8)
        self._lib.orc_classes(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
        return out.reshape(self.shape)

    def normals(self):
        out = np.zeros(3 * self.N)
        self._lib.orc_normals(self._h, _dptr(out))
        return out.reshape(self.shape + (3,))

    def ledger(self) -> dict:
        out = np.zeros(7)
        self._lib.orc_ledger(self._h, _dptr(out))
        return dict(solute=out[0], solid_over_vm=out[1], unpaid=out[2], dirichlet_in=out[3],
                    open_in=out[4], reacted=out[5], step=int(out[6]))

    def reacted(self):
        """Per-cell reacted mass M_b of the last step (mass injected into the fluid)."""
        out = np.zeros(self.N)
        self._lib.orc_reacted(self._h, _dptr(out))
        return out.reshape(self.shape)

    def events(self):
        """Array of (step, node, kind) rows in the order they were applied."""
        n = self._lib.orc_event_count(self._h)
        st, nd = np.zeros(n, dtype=np.int64), np.zeros(n, dtype=np.int64)
        kd = np.zeros(n, dtype=np.int32)
        if n:
            self._lib.orc_events(self._h, st.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                 nd.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                 kd.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return np.stack([st, nd, kd.astype(np.int64)], axis=1) if n else np.zeros((0, 3), dtype=np.int64)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lattice(q: int, dim: int, rest_fraction: float = -1.0):
    """(e[q,3], w[q], cs2, opp[q]) of the oracle's velocity set."""
    lib = _load()
    e = np.zeros(3 * q, dtype=np.int32)
    w = np.zeros(q)
    opp = np.zeros(q, dtype=np.int32)
    cs2 = ctypes.c_double()
    ip = ctypes.POINTER(ctypes.c_int)
    if lib.orc_lattice(q, dim, rest_fraction, e.ctypes.data_as(ip), _dptr(w), ctypes.byref(cs2),
                       opp.ctypes.data_as(ip)):
        raise ValueError("no such lattice")
    return e.reshape(q, 3), w, cs2.value, opp


def equilibrium(q: int, dim: int, density: float, u, solute: bool, rest_fraction: float = -1.0):
    lib = _load()
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(3))
    out = np.zeros(q)
    if lib.orc_equilibrium(q, dim, rest_fraction, int(solute), density, _dptr(u), _dptr(out)):
        raise ValueError("no such lattice")
    return out


def rbc(k: float, w: float, c_eq: float, g_tilde: float, infinite: bool = False) -> float:
    return _load().orc_rbc(k, w, c_eq, g_tilde, int(infinite))
