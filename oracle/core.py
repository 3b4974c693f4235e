"""ctypes wrapper of the FP64 C oracle (``oracle/relres_oracle.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  ``build_oracle()``
compiles the C file with gcc (OpenMP) into ``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

from . import params as P

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "relres_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the C oracle (plain gcc, -O2, OpenMP).  Returns the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-D_GNU_SOURCE",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build_oracle()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            L.oracle_u_tilde.argtypes = [dp, dp, C.c_long, dp, dp]
            L.oracle_pair_forces.argtypes = [C.c_int, dp, dp, ip, C.c_int, dp, ip, ip, dp, dp,
                                             dp, C.c_int]
            L.oracle_pair_forces.restype = C.c_int
            L.oracle_pair_forces_rows.argtypes = [C.c_int, dp, dp, ip, C.c_int, dp, ip, ip,
                                                  C.c_int, ip, dp, dp, C.c_int]
            L.oracle_pair_forces_rows.restype = C.c_int
            L.oracle_u_tilde_d2.argtypes = [dp, dp, C.c_long, dp]
            L.oracle_pair_param_grads.argtypes = [C.c_int, dp, dp, ip, C.c_int, dp, dp, ip, ip, dp,
                                                  C.c_double, dp, C.c_int]
            L.oracle_pair_param_grads.restype = C.c_int
            L.oracle_pair_hvp.argtypes = [C.c_int, dp, dp, ip, C.c_int, dp, ip, ip, dp, dp, C.c_int]
            L.oracle_pair_hvp.restype = C.c_int
            L.oracle_bonded.argtypes = [C.c_int, dp, dp, C.c_int, ip, ip, dp, dp, C.c_int, ip,
                                        ip, dp, dp, C.c_int, ip, ip, dp, dp, dp]
            L.oracle_bonded.restype = C.c_int
            L.oracle_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
            L.oracle_splitmix64.restype = C.c_uint64
            L.oracle_csvr_alpha.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double,
                                            C.c_double, C.c_uint64, C.c_uint64]
            L.oracle_csvr_alpha.restype = C.c_double
            L.oracle_md.argtypes = [C.c_int, dp, dp, dp, dp, ip, C.c_int, dp, ip, ip, C.c_void_p,
                                    C.c_int, C.c_double, C.c_double, C.c_double, C.c_uint64,
                                    C.c_uint64, dp, C.c_int]
            L.oracle_md.restype = C.c_int
            _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int)) if a is not None else None


def u_tilde(row, r):
    """Eq. 20 for one type-pair record at distances r: returns (u, du/dr)."""
    row = _d(row)
    r = _d(np.atleast_1d(r))
    u = np.empty_like(r)
    du = np.empty_like(r)
    lib().oracle_u_tilde(_dp(row), _dp(r), r.size, _dp(u), _dp(du))
    return u, du


def pair_forces(pos, box, types, table, n_types, excl=None, n_threads=0):
    """All-pairs Eq. 20 forces (N x 3), energy and virial (xx yy zz xy xz yz)."""
    pos = _d(pos)
    box = _d(box)
    types = _i(types)
    table = _d(table)
    n = pos.shape[0]
    f = np.zeros((n, 3))
    e = np.zeros(1)
    w = np.zeros(6)
    eo, ei = (None, None) if excl is None else (_i(excl[0]), _i(excl[1]))
    lib().oracle_pair_forces(n, _dp(pos), _dp(box), _ip(types), n_types, _dp(table), _ip(eo),
                             _ip(ei), _dp(f), _dp(e), _dp(w), int(n_threads))
    return f, float(e[0]), w


def pair_forces_rows(pos, box, types, table, n_types, rows, excl=None, n_threads=0):
    """Eq. 20 forces (len(rows) x 3) and half pair energies of the listed atoms
    against all atoms: the same sum as pair_forces, for a subset of rows."""
    pos = _d(pos)
    box = _d(box)
    types = _i(types)
    table = _d(table)
    rows = _i(rows)
    f = np.zeros((len(rows), 3))
    e = np.zeros(len(rows))
    eo, ei = (None, None) if excl is None else (_i(excl[0]), _i(excl[1]))
    lib().oracle_pair_forces_rows(pos.shape[0], _dp(pos), _dp(box), _ip(types), n_types,
                                  _dp(table), _ip(eo), _ip(ei), len(rows), _ip(rows), _dp(f),
                                  _dp(e), int(n_threads))
    return f, e


def u_tilde_d2(row, r):
    """Second r-derivative of Eq. 20 for one record at the distances r."""
    row = _d(row)
    r = _d(np.atleast_1d(r))
    out = np.zeros_like(r)
    lib().oracle_u_tilde_d2(_dp(row), _dp(r), r.size, _dp(out))
    return out


def pair_param_grads(pos, box, types, table, dtable, n_types, g_energy=0.0, g_forces=None, excl=None,
                     n_threads=0):
    """d L / d (eps_fg, sig_fg, eps_cg, sig_cg) of every record (n_types^2 x 4)
    for L with dL/dE_pair = g_energy and dL/dF_i = g_forces[i] (or None)."""
    pos = _d(pos)
    box = _d(box)
    types = _i(types)
    table = _d(table)
    dtable = _d(dtable)
    gf = None if g_forces is None else _d(g_forces)
    out = np.zeros(n_types * n_types * 4)
    eo, ei = (None, None) if excl is None else (_i(excl[0]), _i(excl[1]))
    lib().oracle_pair_param_grads(pos.shape[0], _dp(pos), _dp(box), _ip(types), n_types, _dp(table),
                                  _dp(dtable), _ip(eo), _ip(ei), None if gf is None else _dp(gf),
                                  float(g_energy), _dp(out), int(n_threads))
    return out.reshape(n_types * n_types, 4)


def pair_hvp(pos, box, types, table, n_types, v, excl=None, n_threads=0):
    """Hessian of the pair energy times v (n x 3): sum_j h_ij (v_i - v_j)."""
    pos = _d(pos)
    box = _d(box)
    types = _i(types)
    table = _d(table)
    v = _d(v)
    out = np.zeros_like(pos)
    eo, ei = (None, None) if excl is None else (_i(excl[0]), _i(excl[1]))
    lib().oracle_pair_hvp(pos.shape[0], _dp(pos), _dp(box), _ip(types), n_types, _dp(table), _ip(eo),
                          _ip(ei), _dp(v), _dp(out), int(n_threads))
    return out


def table_derivs_for(system, shift: bool = True):
    """Derivative records (n_types^2, 4, 26) matching ``table_for``."""
    return P.table_derivs(system.eps_fg, system.sig_fg, system.is_hybrid, system.radii,
                          mixing=system.mixing, group_comp=system.group_comp, shift=shift)


class _Topo(C.Structure):
    _fields_ = [
        ("nb", C.c_int), ("bonds", C.c_void_p), ("btype", C.c_void_p),
        ("bond_k", C.c_void_p), ("bond_r0", C.c_void_p),
        ("na", C.c_int), ("angles", C.c_void_p), ("atype", C.c_void_p),
        ("ang_k", C.c_void_p), ("ang_t0", C.c_void_p),
        ("nd", C.c_int), ("dihs", C.c_void_p), ("dtype", C.c_void_p), ("dih_k", C.c_void_p),
    ]


def _topo_arrays(topo):
    """Contiguous copies of a topology dict (see paper_2104_10231_gb300.systems)."""
    t = {}
    t["bonds"] = _i(topo["bonds"]).reshape(-1)
    t["btype"] = _i(topo["bond_type"])
    t["bond_k"] = _d(topo["bond_k"])
    t["bond_r0"] = _d(topo["bond_r0"])
    t["angles"] = _i(topo["angles"]).reshape(-1)
    t["atype"] = _i(topo["angle_type"])
    t["ang_k"] = _d(topo["angle_k"])
    t["ang_t0"] = _d(topo["angle_theta0"])
    t["dihs"] = _i(topo["dihedrals"]).reshape(-1)
    t["dtype"] = _i(topo["dihedral_type"])
    t["dih_k"] = _d(np.asarray(topo["dihedral_k"]).reshape(-1)) if len(topo["dihedral_k"]) else _d(np.zeros(4))
    for k in ("bond_k", "bond_r0", "ang_k", "ang_t0"):
        if t[k].size == 0:
            t[k] = _d(np.zeros(1))
    return t


def bonded(pos, box, topo):
    """Bonded forces (N x 3) and energies (bond, angle, dihedral)."""
    pos = _d(pos)
    box = _d(box)
    n = pos.shape[0]
    t = _topo_arrays(topo)
    f = np.zeros((n, 3))
    e = np.zeros(3)
    lib().oracle_bonded(n, _dp(pos), _dp(box), len(t["btype"]), _ip(t["bonds"]), _ip(t["btype"]),
                        _dp(t["bond_k"]), _dp(t["bond_r0"]), len(t["atype"]), _ip(t["angles"]),
                        _ip(t["atype"]), _dp(t["ang_k"]), _dp(t["ang_t0"]), len(t["dtype"]),
                        _ip(t["dihs"]), _ip(t["dtype"]), _dp(t["dih_k"]), _dp(f), _dp(e))
    return f, e


def splitmix64(seed: int, counter: int) -> int:
    return int(lib().oracle_splitmix64(C.c_uint64(seed), C.c_uint64(counter)))


def csvr_alpha(ke, ke_target, n_f, dt, tau, seed, step) -> float:
    return float(lib().oracle_csvr_alpha(ke, ke_target, n_f, dt, tau, C.c_uint64(seed),
                                         C.c_uint64(step)))


def md(pos, vel, box, masses, types, table, n_types, excl, topo, n_steps, dt,
       t_target=0.0, tau=100.0, seed=0, step0=0, n_threads=0):
    """Velocity Verlet (+ CSVR if t_target > 0).  Returns (pos, vel, thermo)
    with thermo[s] = (E_pair, E_bonded, KE) after step s."""
    pos = _d(pos).copy()
    vel = _d(vel).copy()
    box = _d(box)
    masses = _d(masses)
    types = _i(types)
    table = _d(table)
    n = pos.shape[0]
    eo, ei = (None, None) if excl is None else (_i(excl[0]), _i(excl[1]))
    t = _topo_arrays(topo)
    st = _Topo(len(t["btype"]), t["bonds"].ctypes.data, t["btype"].ctypes.data,
               t["bond_k"].ctypes.data, t["bond_r0"].ctypes.data, len(t["atype"]),
               t["angles"].ctypes.data, t["atype"].ctypes.data, t["ang_k"].ctypes.data,
               t["ang_t0"].ctypes.data, len(t["dtype"]), t["dihs"].ctypes.data,
               t["dtype"].ctypes.data, t["dih_k"].ctypes.data)
    thermo = np.zeros((n_steps, 3))
    rc = lib().oracle_md(n, _dp(pos), _dp(vel), _dp(box), _dp(masses), _ip(types), n_types,
                         _dp(table), _ip(eo), _ip(ei), C.byref(st), n_steps, dt, t_target, tau,
                         C.c_uint64(seed), C.c_uint64(step0), _dp(thermo), int(n_threads))
    if rc != 0:
        raise RuntimeError("oracle_md failed")
    return pos, vel, thermo


def table_for(system, shift: bool = True):
    """Type-pair table for a synthetic system (see paper_2104_10231_gb300.systems):
    FG mixing per the system, CG parameters by Eq. 13 from the group
    compositions, Eq. 14 for ordinary types."""
    return P.pair_table(system.eps_fg, system.sig_fg, system.is_hybrid, system.radii,
                        mixing=system.mixing, group_comp=system.group_comp, shift=shift)
