"""ctypes wrapper for the FP64 CPU oracle (``oracle/tlbm_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow statement of the thermal
lattice Boltzmann step of Xu & Li (§2.2, Eqs. (5)-(7), (10)-(11)).  Only the test
suite, the smoke check and the benchmark's CPU baseline may import this module;
the CUDA library and its Python binding never do.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tlbm_oracle.c")
_HDR = os.path.join(_HERE, "tlbm_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libtlbm_oracle.so")
_lock = threading.Lock()
_lib = None

D2Q9_D2Q5 = 0
D3Q19_D3Q7 = 1
RB = 0
SIDE_HEATED = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_LIB)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-Wall", "-Wno-unused-function", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("walls", C.c_int), ("periodic_mask", C.c_int), ("u_is_ma", C.c_int),
        ("a_T", C.c_double), ("nu", C.c_double), ("alpha", C.c_double), ("gbeta", C.c_double),
        ("s_rho", C.c_double), ("s_e", C.c_double), ("s_eps", C.c_double), ("s_j", C.c_double),
        ("s_q", C.c_double), ("s_pi", C.c_double), ("s_m", C.c_double),
        ("q_e", C.c_double), ("q_v", C.c_double),
        ("body_force", C.c_double * 3), ("Th", C.c_double), ("Tc", C.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            L.tlbmo_default_params.argtypes = [C.POINTER(Params)]
            L.tlbmo_create.restype = C.c_void_p
            L.tlbmo_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                       C.c_double, C.c_double, C.POINTER(Params)]
            L.tlbmo_destroy.argtypes = [C.c_void_p]
            L.tlbmo_derived.restype = C.c_int
            L.tlbmo_derived.argtypes = [C.c_void_p, dp, C.c_int]
            L.tlbmo_init.argtypes = [C.c_void_p, C.c_uint64, C.c_double]
            L.tlbmo_step.argtypes = [C.c_void_p, C.c_int64]
            L.tlbmo_time.restype = C.c_int64
            L.tlbmo_time.argtypes = [C.c_void_p]
            L.tlbmo_get_populations.argtypes = [C.c_void_p, dp, dp]
            L.tlbmo_set_populations.argtypes = [C.c_void_p, dp, dp]
            L.tlbmo_macros.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
            L.tlbmo_nusselt.restype = C.c_double
            L.tlbmo_nusselt.argtypes = [C.c_void_p]
            L.tlbmo_energy.argtypes = [C.c_void_p, dp, dp]
            L.tlbmo_set_threads.argtypes = [C.c_int]
            L.tlbmo_get_threads.restype = C.c_int
            L.tlbmo_velocity_set.restype = C.c_int
            L.tlbmo_velocity_set.argtypes = [C.c_int, ip, dp, ip, dp, dp]
            L.tlbmo_forcing_moments.argtypes = [C.c_int, dp, dp, dp]
            L.tlbmo_flow_meq.argtypes = [C.c_int, C.c_double, dp, dp]
            L.tlbmo_thermal_geq.argtypes = [C.c_int, C.c_double, C.c_double, dp, dp]
            L.tlbmo_collide_node.argtypes = [C.c_void_p, dp, dp, dp, dp]
            L.tlbmo_uniform.restype = C.c_double
            L.tlbmo_uniform.argtypes = [C.c_uint64, C.c_uint64]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(**kw) -> Params:
    """Oracle parameter block; unspecified doubles stay NaN (= derive default)."""
    p = Params()
    lib().tlbmo_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "body_force":
            for a in range(3):
                p.body_force[a] = float(v[a])
        else:
            setattr(p, k, v)
    return p


def velocity_set(which: int):
    """which: 0 D2Q9, 1 D2Q5, 2 D3Q19, 3 D3Q7 -> (e[q,3], w[q], opp[q], M[q,q], Minv[q,q])."""
    L = lib()
    e = np.zeros(19 * 3, dtype=np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, dtype=np.int32)
    M = np.zeros(19 * 19)
    Mi = np.zeros(19 * 19)
    ip = C.POINTER(C.c_int)
    q = L.tlbmo_velocity_set(which, e.ctypes.data_as(ip), _dp(w), opp.ctypes.data_as(ip), _dp(M), _dp(Mi))
    return (e[: 3 * q].reshape(q, 3).copy(), w[:q].copy(), opp[:q].copy(),
            M[: q * q].reshape(q, q).copy(), Mi[: q * q].reshape(q, q).copy())


def forcing_moments(lattice: int, u, F) -> np.ndarray:
    q = 9 if lattice == D2Q9_D2Q5 else 19
    out = np.zeros(q)
    lib().tlbmo_forcing_moments(lattice, _dp(np.asarray(u, dtype=np.float64).copy()),
                                _dp(np.asarray(F, dtype=np.float64).copy()), _dp(out))
    return out


def flow_meq(lattice: int, rho: float, u) -> np.ndarray:
    q = 9 if lattice == D2Q9_D2Q5 else 19
    out = np.zeros(q)
    lib().tlbmo_flow_meq(lattice, float(rho), _dp(np.asarray(u, dtype=np.float64).copy()), _dp(out))
    return out


def thermal_geq(lattice: int, a_T: float, T: float, u) -> np.ndarray:
    q = 5 if lattice == D2Q9_D2Q5 else 7
    out = np.zeros(q)
    lib().tlbmo_thermal_geq(lattice, float(a_T), float(T), _dp(np.asarray(u, dtype=np.float64).copy()), _dp(out))
    return out


def uniform(seed: int, idx: int) -> float:
    return lib().tlbmo_uniform(seed, idx)


def set_threads(n: int) -> None:
    lib().tlbmo_set_threads(int(n))


def get_threads() -> int:
    return lib().tlbmo_get_threads()


class Sim:
    """One oracle instance: nx x ny (x nz) cell, FP64, pre-collision state."""

    def __init__(self, nx, ny, nz=1, lattice=D2Q9_D2Q5, Ra=1e5, Pr=0.71, Ma=0.1, **params):
        self.lattice = lattice
        self.nx, self.ny = nx, ny
        self.nz = nz if lattice == D3Q19_D3Q7 else 1
        self.qf = 9 if lattice == D2Q9_D2Q5 else 19
        self.qg = 5 if lattice == D2Q9_D2Q5 else 7
        self.N = self.nx * self.ny * self.nz
        self._p = make_params(**params)
        self._h = lib().tlbmo_create(nx, ny, self.nz, lattice, Ra, Pr, Ma, C.byref(self._p))
        if not self._h:
            raise ValueError("oracle rejected the arguments")

    def close(self):
        if getattr(self, "_h", None):
            lib().tlbmo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx) if self.lattice == D3Q19_D3Q7 else (self.ny, self.nx)

    def derived(self) -> dict:
        out = np.zeros(64)
        n = lib().tlbmo_derived(self._h, _dp(out), 64)
        v = out[:n]
        d = dict(U=v[0], H=v[1], nu=v[2], alpha=v[3], gbeta=v[4], a_T=v[5], omega=v[6])
        d["S"] = v[7:7 + self.qf].copy()
        d["Q"] = v[7 + self.qf:7 + self.qf + self.qg].copy()
        return d

    def init(self, seed: int, noise_amp: float):
        lib().tlbmo_init(self._h, seed, noise_amp)

    def step(self, n: int = 1):
        lib().tlbmo_step(self._h, int(n))

    @property
    def time(self) -> int:
        return lib().tlbmo_time(self._h)

    def get_populations(self):
        f = np.zeros((self.qf,) + self.shape)
        g = np.zeros((self.qg,) + self.shape)
        lib().tlbmo_get_populations(self._h, _dp(f), _dp(g))
        return f, g

    def set_populations(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape((self.qf,) + self.shape)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape((self.qg,) + self.shape)
        lib().tlbmo_set_populations(self._h, _dp(f), _dp(g))

    def macros(self) -> dict:
        a = {k: np.zeros(self.shape) for k in ("rho", "ux", "uy", "uz", "T")}
        lib().tlbmo_macros(self._h, _dp(a["rho"]), _dp(a["ux"]), _dp(a["uy"]), _dp(a["uz"]), _dp(a["T"]))
        return a

    def nusselt(self) -> float:
        return lib().tlbmo_nusselt(self._h)

    def energy(self):
        e = C.c_double()
        m = C.c_double()
        lib().tlbmo_energy(self._h, C.byref(e), C.byref(m))
        return e.value, m.value

    def collide_node(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        fo = np.zeros(self.qf)
        go = np.zeros(self.qg)
        lib().tlbmo_collide_node(self._h, _dp(f), _dp(g), _dp(fo), _dp(go))
        return fo, go
