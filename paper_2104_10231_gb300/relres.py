"""Thin ctypes binding of librelres (include/relres.h).

Argument marshalling only: every computation runs in the CUDA library.  The
functions keep the C names (``relres_create``, ``relres_build_neighbors``,
``relres_compute``, ``relres_step`` ...) and raise ``RelresError`` when the C
call returns a non-OK status.  Device buffers are passed as raw pointers
(``tensor.data_ptr()`` of CUDA tensors); the CUDA stream as its handle.

The library is loaded from this package directory (built in-tree by
``paper_2104_10231_gb300.build``); a missing library is an error, never a
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librelres.so")

RELRES_OK = 0
STATUS_NAMES = {0: "RELRES_OK", 1: "RELRES_ERR_ARG", 2: "RELRES_ERR_CUDA", 3: "RELRES_ERR_BOX",
                4: "RELRES_ERR_LIST_OVERFLOW", 5: "RELRES_ERR_NONFINITE", 6: "RELRES_ERR_STATE",
                7: "RELRES_ERR_NOMEM"}
RELRES_MIX_GEOMETRIC, RELRES_MIX_LB = 0, 1
RELRES_PREC_FP64, RELRES_PREC_FP32 = 0, 1
RELRES_ACC_FP32, RELRES_ACC_COMPENSATED, RELRES_ACC_FP64 = 0, 1, 2
RELRES_MAX_TYPES = 8
RELRES_THERMO_COLS = 10
RELRES_PAIR_FIELDS = 26

EXPORTED = ["relres_prepare_table", "relres_cg_params", "relres_chain_cg_grads", "relres_create", "relres_set_topology",
            "relres_build_neighbors", "relres_compute", "relres_step", "relres_set_step_counter",
            "relres_get_stats", "relres_set_timing", "relres_get_timings", "relres_last_error",
            "relres_destroy", "relres_pair_forces_static", "relres_set_graphs", "relres_set_params",
            "relres_backward", "relres_set_pair_config", "relres_batch_create", "relres_batch_step",
            "relres_batch_last_error", "relres_batch_destroy", "relres_set_timing_sampled",
            "relres_set_list_caps", "relres_set_prune", "relres_measure_rates", "relres_get_list",
            "relres_eval_recip", "relres_set_force_accumulation", "relres_batch_get_info",
            "relres_batch_set_mode"]
RELRES_STATIC_MAX_ATOMS = 16384
RELRES_BATCH_SHARED_MAX_ATOMS = 16384
TIMING_CLASSES = ["drift", "rebuild", "lists", "pair", "finish", "thermo", "pair_ev", "prune"]


class RelresError(RuntimeError):
    def __init__(self, status, message=""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class relres_params(C.Structure):
    _fields_ = [("n_types", C.c_int), ("eps_fg", _dp), ("sig_fg", _dp), ("is_hybrid", _ip),
                ("mixing", C.c_int), ("eps_cg", _dp), ("sig_cg", _dp), ("group_comp", _ip),
                ("r_si", C.c_double), ("r_so", C.c_double), ("r_ci", C.c_double),
                ("r_co", C.c_double), ("radii_pair", _dp), ("shift", C.c_int),
                ("skin", C.c_double), ("precision", C.c_int)]


class relres_topology(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("type", _ip), ("mass_by_type", _dp),
                ("excl_offsets", _ip), ("excl_index", _ip),
                ("n_bonds", C.c_int), ("bonds", _ip), ("bond_type", _ip), ("n_bond_types", C.c_int),
                ("bond_k", _dp), ("bond_r0", _dp),
                ("n_angles", C.c_int), ("angles", _ip), ("angle_type", _ip),
                ("n_angle_types", C.c_int), ("angle_k", _dp), ("angle_theta0", _dp),
                ("n_dihedrals", C.c_int), ("dihedrals", _ip), ("dihedral_type", _ip),
                ("n_dihedral_types", C.c_int), ("dihedral_k", _dp)]


class relres_stats(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("n_hybrid", C.c_int), ("cap_fg", C.c_int),
                ("cap_cg", C.c_int), ("max_fg", C.c_int), ("max_cg", C.c_int),
                ("mean_fg", C.c_double), ("mean_cg", C.c_double),
                ("list_radius_fg", C.c_double), ("list_radius_cg", C.c_double),
                ("skin_cg", C.c_double), ("grid_fg", C.c_int * 3), ("grid_cg", C.c_int * 3),
                ("n_builds", C.c_longlong), ("n_steps", C.c_longlong), ("has_cg", C.c_int),
                ("n_launches", C.c_longlong), ("pair_tpa", C.c_int), ("pair_block", C.c_int),
                ("prune_delta", C.c_double), ("n_prunes", C.c_longlong), ("mean_fg_pruned", C.c_double),
                ("mean_cg_pruned", C.c_double), ("step_segments", C.c_int), ("force_acc", C.c_int),
                ("n_segments", C.c_int), ("n_segment_protos", C.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["grid_fg"] = list(self.grid_fg)
        d["grid_cg"] = list(self.grid_cg)
        return d


_lib = None


class relres_rates(C.Structure):
    _fields_ = [("ffma_per_clk_sm", C.c_double), ("dfma_per_clk_sm", C.c_double),
                ("conv64_per_clk_sm", C.c_double), ("copy_gbs", C.c_double), ("fp32_tflops", C.c_double),
                ("fp64_tflops", C.c_double), ("sm_count", C.c_int), ("clock_mhz", C.c_int)]


def load():
    """Load librelres.so from the package directory (raises if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2104_10231_gb300.build` (needs nvcc)")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    L.relres_prepare_table.argtypes = [C.POINTER(relres_params), _dp, C.c_int]
    L.relres_cg_params.argtypes = [C.c_int, _dp, _dp, C.c_int, _ip, _ip, _dp, _dp]
    L.relres_chain_cg_grads.argtypes = [C.POINTER(relres_params), _dp, _dp, _dp, _dp]
    L.relres_create.argtypes = [C.POINTER(vp), C.POINTER(relres_params), vp]
    L.relres_set_topology.argtypes = [vp, C.POINTER(relres_topology)]
    L.relres_build_neighbors.argtypes = [vp, vp, _dp]
    L.relres_compute.argtypes = [vp, vp, vp, vp, vp]
    L.relres_step.argtypes = [vp, C.c_int, C.c_double, vp, vp, C.c_double, C.c_double,
                              C.c_uint64, C.c_int, vp]
    L.relres_set_step_counter.argtypes = [vp, C.c_longlong]
    L.relres_get_stats.argtypes = [vp, C.POINTER(relres_stats)]
    L.relres_set_timing.argtypes = [vp, C.c_int]
    L.relres_set_timing_sampled.argtypes = [vp, C.c_uint, C.c_int]
    L.relres_set_list_caps.argtypes = [vp, C.c_int, C.c_int]
    L.relres_set_prune.argtypes = [vp, C.c_double]
    L.relres_measure_rates.argtypes = [vp, C.c_size_t, vp, C.POINTER(relres_rates)]
    L.relres_get_list.argtypes = [vp, C.c_int, _ip, _ip, C.c_longlong, C.POINTER(C.c_longlong)]
    L.relres_eval_recip.argtypes = [vp, vp, vp, C.c_int, vp]
    L.relres_set_graphs.argtypes = [vp, C.c_int]
    L.relres_set_params.argtypes = [vp, C.POINTER(relres_params)]
    L.relres_set_pair_config.argtypes = [vp, C.c_int]
    L.relres_set_force_accumulation.argtypes = [vp, C.c_int]
    L.relres_batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int, vp]
    L.relres_batch_step.argtypes = [vp, C.c_int, C.c_double, C.POINTER(vp), C.POINTER(vp), _dp, C.c_double,
                                    C.POINTER(C.c_uint64), C.c_int, C.POINTER(vp)]
    L.relres_batch_get_info.argtypes = [vp, C.POINTER(C.c_int)]
    L.relres_batch_set_mode.argtypes = [vp, C.c_int]
    L.relres_batch_last_error.argtypes = [vp]
    L.relres_batch_last_error.restype = C.c_char_p
    L.relres_batch_destroy.argtypes = [vp]
    L.relres_batch_destroy.restype = None
    L.relres_backward.argtypes = [vp, vp, vp, C.c_double, vp, _dp, _dp, _dp, _dp, _dp]
    L.relres_get_timings.argtypes = [vp, _dp, C.POINTER(C.c_longlong), C.c_int]
    L.relres_pair_forces_static.argtypes = [C.POINTER(relres_params), C.c_int, vp, vp, _dp, vp, vp, vp,
                                            vp, vp, vp]
    L.relres_last_error.argtypes = [vp]
    L.relres_last_error.restype = C.c_char_p
    L.relres_destroy.argtypes = [vp]
    L.relres_destroy.restype = None
    for name in EXPORTED:
        if name not in ("relres_last_error", "relres_destroy", "relres_batch_last_error", "relres_batch_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(status, ctx=None):
    if status != RELRES_OK:
        msg = ""
        if ctx is not None:
            msg = (load().relres_last_error(ctx) or b"").decode()
        raise RelresError(status, msg)


def _ptr(x):
    """Raw device pointer of a CUDA tensor (or None / int)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


# ------------------------------------------------------------- marshalling

class _Keep:
    """Holds the numpy arrays a ctypes struct points into."""

    def __init__(self):
        self.arrays = []

    def d(self, a):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.arrays.append(a)
        return a.ctypes.data_as(_dp)

    def i(self, a):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=np.int32)
        self.arrays.append(a)
        return a.ctypes.data_as(_ip)


def make_params(eps_fg, sig_fg, is_hybrid, radii, skin, mixing=RELRES_MIX_LB, group_comp=None,
                eps_cg=None, sig_cg=None, shift=True, precision=RELRES_PREC_FP32,
                radii_pair=None):
    keep = _Keep()
    p = relres_params()
    p.n_types = len(eps_fg)
    p.eps_fg = keep.d(eps_fg)
    p.sig_fg = keep.d(sig_fg)
    p.is_hybrid = keep.i(is_hybrid)
    p.mixing = int(mixing)
    p.eps_cg = keep.d(None if eps_cg is None else np.asarray(eps_cg).reshape(-1))
    p.sig_cg = keep.d(None if sig_cg is None else np.asarray(sig_cg).reshape(-1))
    p.group_comp = keep.i(None if group_comp is None else np.asarray(group_comp).reshape(-1))
    p.r_si, p.r_so, p.r_ci, p.r_co = (float(x) for x in radii)
    p.radii_pair = keep.d(None if radii_pair is None else np.asarray(radii_pair).reshape(-1))
    p.shift = 1 if shift else 0
    p.skin = float(skin)
    p.precision = int(precision)
    p._keep = keep
    return p


def make_topology(types, mass_by_type, excl=None, topo=None):
    keep = _Keep()
    t = relres_topology()
    t.n_atoms = len(types)
    t.type = keep.i(types)
    t.mass_by_type = keep.d(mass_by_type)
    if excl is not None:
        t.excl_offsets = keep.i(excl[0])
        t.excl_index = keep.i(excl[1])
    if topo is not None:
        t.n_bonds = len(topo["bond_type"])
        if t.n_bonds:
            t.bonds = keep.i(np.asarray(topo["bonds"]).reshape(-1))
            t.bond_type = keep.i(topo["bond_type"])
            t.n_bond_types = len(topo["bond_k"])
            t.bond_k = keep.d(topo["bond_k"])
            t.bond_r0 = keep.d(topo["bond_r0"])
        t.n_angles = len(topo["angle_type"])
        if t.n_angles:
            t.angles = keep.i(np.asarray(topo["angles"]).reshape(-1))
            t.angle_type = keep.i(topo["angle_type"])
            t.n_angle_types = len(topo["angle_k"])
            t.angle_k = keep.d(topo["angle_k"])
            t.angle_theta0 = keep.d(topo["angle_theta0"])
        t.n_dihedrals = len(topo["dihedral_type"])
        if t.n_dihedrals:
            t.dihedrals = keep.i(np.asarray(topo["dihedrals"]).reshape(-1))
            t.dihedral_type = keep.i(topo["dihedral_type"])
            t.n_dihedral_types = len(topo["dihedral_k"])
            t.dihedral_k = keep.d(np.asarray(topo["dihedral_k"]).reshape(-1))
    t._keep = keep
    return t


def params_for(system, precision=RELRES_PREC_FP32, shift=True):
    """relres_params of a ``systems.System``: FG mixing of the system, CG pair
    parameters derived by the library from the group compositions (Eq. 13)."""
    mixing = RELRES_MIX_LB if system.mixing == "lb" else RELRES_MIX_GEOMETRIC
    return make_params(system.eps_fg, system.sig_fg, system.is_hybrid, system.radii, system.skin,
                       mixing=mixing, group_comp=system.group_comp, shift=shift,
                       precision=precision)


def topology_for(system):
    return make_topology(system.types, system.mass_by_type, system.excl, system.topo)


# ------------------------------------------------------------- C entry points

def relres_measure_rates(d_scratch, stream=None):
    """Measured FP32/FP64 FMA and 64-bit conversion rates (per clock per SM)
    and copy bandwidth of this GPU; d_scratch: a CUDA tensor (bytes), large."""
    out = relres_rates()
    nbytes = d_scratch.numel() * d_scratch.element_size()
    st = C.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(load().relres_measure_rates(_ptr(d_scratch), nbytes, st, C.byref(out)))
    return {k: getattr(out, k) for k, _ in out._fields_}


def relres_eval_recip(d_x, d_out32, d_out64, stream=None):
    """The pair kernels' reciprocals on the FP64 CUDA tensor d_x (n): FP32 1/x
    into d_out32 (n floats), FP64 1/x and 1/sqrt(x) into d_out64 (2n)."""
    st = C.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(load().relres_eval_recip(_ptr(d_x), _ptr(d_out32), _ptr(d_out64), int(d_x.numel()), st))


def relres_prepare_table(params):
    n = params.n_types * params.n_types * RELRES_PAIR_FIELDS
    out = np.zeros(n)
    _check(load().relres_prepare_table(C.byref(params), out.ctypes.data_as(_dp), n))
    return out.reshape(params.n_types * params.n_types, RELRES_PAIR_FIELDS)


def relres_cg_params(eps_fg, sig_fg, mixing, comp_i, comp_j):
    keep = _Keep()
    e = C.c_double()
    s = C.c_double()
    _check(load().relres_cg_params(len(eps_fg), keep.d(eps_fg), keep.d(sig_fg), int(mixing),
                                   keep.i(comp_i), keep.i(comp_j), C.byref(e), C.byref(s)))
    return e.value, s.value


def relres_chain_cg_grads(params, g_eps_cg, g_sig_cg, g_eps_fg, g_sig_fg):
    """Chain rule through Eq. 13 (host-only): returns (g_eps_fg, g_sig_fg)
    [n_types] plus the contributions of g_eps_cg, g_sig_cg [n_types, n_types]
    when the CG parameters follow the FG ones (params: group_comp, no
    explicit eps_cg)."""
    ge = np.array(g_eps_fg, dtype=np.float64, copy=True).reshape(-1)
    gs = np.array(g_sig_fg, dtype=np.float64, copy=True).reshape(-1)
    ec = np.ascontiguousarray(g_eps_cg, dtype=np.float64).reshape(-1)
    sc = np.ascontiguousarray(g_sig_cg, dtype=np.float64).reshape(-1)
    nt = params.n_types
    if ge.size != nt or gs.size != nt or ec.size != nt * nt or sc.size != nt * nt:
        raise ValueError("relres_chain_cg_grads: FG gradients need n_types entries, CG ones n_types^2")
    _check(load().relres_chain_cg_grads(C.byref(params), ec.ctypes.data_as(_dp), sc.ctypes.data_as(_dp),
                                        ge.ctypes.data_as(_dp), gs.ctypes.data_as(_dp)))
    return ge, gs


def relres_create(params, stream=None):
    ctx = C.c_void_p()
    _check(load().relres_create(C.byref(ctx), C.byref(params), stream))
    return ctx


def relres_set_topology(ctx, topo):
    _check(load().relres_set_topology(ctx, C.byref(topo)), ctx)


def relres_build_neighbors(ctx, d_pos, box):
    b = np.ascontiguousarray(box, dtype=np.float64)
    _check(load().relres_build_neighbors(ctx, _ptr(d_pos), b.ctypes.data_as(_dp)), ctx)


def relres_compute(ctx, d_pos, d_forces, d_energy=None, d_virial=None):
    _check(load().relres_compute(ctx, _ptr(d_pos), _ptr(d_forces), _ptr(d_energy),
                                 _ptr(d_virial)), ctx)


def relres_step(ctx, n_steps, dt_fs, d_pos, d_vel, t_target=0.0, tau_fs=100.0, seed=0,
                thermo_every=0, d_thermo=None):
    _check(load().relres_step(ctx, int(n_steps), float(dt_fs), _ptr(d_pos), _ptr(d_vel),
                              float(t_target), float(tau_fs), C.c_uint64(seed),
                              int(thermo_every), _ptr(d_thermo)), ctx)


def relres_set_step_counter(ctx, step):
    _check(load().relres_set_step_counter(ctx, int(step)), ctx)


def relres_get_stats(ctx):
    st = relres_stats()
    _check(load().relres_get_stats(ctx, C.byref(st)), ctx)
    return st.as_dict()


def relres_set_timing(ctx, enable):
    _check(load().relres_set_timing(ctx, 1 if enable else 0), ctx)


def relres_set_pair_config(ctx, config):
    _check(load().relres_set_pair_config(ctx, int(config)), ctx)


def relres_set_params(ctx, params):
    _check(load().relres_set_params(ctx, C.byref(params)), ctx)


def relres_backward(ctx, n_types, d_pos, d_grad_forces, grad_energy, d_grad_pos=None):
    """Backward pass of the pair interaction; returns the host gradients
    {"grad_c": (n_types^2, 4), "eps_fg", "sig_fg": (n_types,), "eps_cg",
    "sig_cg": (n_types, n_types)} and writes dL/dx into d_grad_pos."""
    nt = int(n_types)
    gc = np.zeros(nt * nt * 4)
    de = np.zeros(nt)
    ds = np.zeros(nt)
    dec = np.zeros(nt * nt)
    dsc = np.zeros(nt * nt)
    _check(load().relres_backward(ctx, _ptr(d_pos), _ptr(d_grad_forces), float(grad_energy), _ptr(d_grad_pos),
                                  gc.ctypes.data_as(_dp), de.ctypes.data_as(_dp), ds.ctypes.data_as(_dp),
                                  dec.ctypes.data_as(_dp), dsc.ctypes.data_as(_dp)), ctx)
    return {"grad_c": gc.reshape(nt * nt, 4), "eps_fg": de, "sig_fg": ds, "eps_cg": dec.reshape(nt, nt),
            "sig_cg": dsc.reshape(nt, nt)}


def relres_set_graphs(ctx, enable):
    _check(load().relres_set_graphs(ctx, 1 if enable else 0), ctx)


def relres_get_timings(ctx):
    """{class: (total_ms, launches)} for the kernel classes of relres.h."""
    n = len(TIMING_CLASSES)
    ms = np.zeros(n)
    cnt = (C.c_longlong * n)()
    _check(load().relres_get_timings(ctx, ms.ctypes.data_as(_dp), cnt, n), ctx)
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(TIMING_CLASSES)}


def relres_pair_forces_static(params, n_atoms, d_type, d_pos, box, d_forces, d_energy=None,
                              d_virial=None, d_excl_offsets=None, d_excl_index=None, stream=None):
    """All-pairs RelRes pair forces without any device allocation (scratch in a
    static device array of the library); for callers that cannot allocate."""
    b = np.ascontiguousarray(box, dtype=np.float64)
    _check(load().relres_pair_forces_static(C.byref(params), int(n_atoms), _ptr(d_type), _ptr(d_pos),
                                            b.ctypes.data_as(_dp), _ptr(d_excl_offsets),
                                            _ptr(d_excl_index), _ptr(d_forces), _ptr(d_energy),
                                            _ptr(d_virial), stream))


def relres_last_error(ctx):
    return (load().relres_last_error(ctx) or b"").decode()


def relres_destroy(ctx):
    if ctx:
        load().relres_destroy(ctx)


class Context:
    """Owns one relres context (and the marshalled host arrays it was made
    from).  ``stream`` is a torch.cuda.Stream or None (current stream)."""

    def __init__(self, params, topology=None, stream=None):
        import torch

        self.params = params
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = relres_create(params, C.c_void_p(self.stream.cuda_stream))
        self.topology = None
        if topology is not None:
            self.set_topology(topology)

    def set_topology(self, topology):
        self.topology = topology
        relres_set_topology(self.ctx, topology)

    def build_neighbors(self, d_pos, box):
        relres_build_neighbors(self.ctx, d_pos, box)

    def compute(self, d_pos, d_forces, d_energy=None, d_virial=None):
        relres_compute(self.ctx, d_pos, d_forces, d_energy, d_virial)

    def step(self, n_steps, dt_fs, d_pos, d_vel, t_target=0.0, tau_fs=100.0, seed=0,
             thermo_every=0, d_thermo=None):
        relres_step(self.ctx, n_steps, dt_fs, d_pos, d_vel, t_target, tau_fs, seed,
                    thermo_every, d_thermo)

    def stats(self):
        return relres_get_stats(self.ctx)

    def set_timing(self, enable):
        relres_set_timing(self.ctx, enable)

    def set_timing_sampled(self, classes, every):
        """Time only the named classes (TIMING_CLASSES names), every k-th step."""
        mask = 0
        for name in classes:
            mask |= 1 << TIMING_CLASSES.index(name)
        _check(load().relres_set_timing_sampled(self.ctx, mask, int(every)), self.ctx)

    def set_graphs(self, enable):
        relres_set_graphs(self.ctx, enable)

    def set_list_caps(self, cap_fg, cap_cg):
        _check(load().relres_set_list_caps(self.ctx, int(cap_fg), int(cap_cg)), self.ctx)

    def get_list(self, which):
        """Entries of one list as an (n, 2) int array of atom pairs (i, j):
        which = 0 FG, 1 CG, 2 pruned FG, 3 pruned CG."""
        import numpy as np

        n = C.c_longlong(0)
        _check(load().relres_get_list(self.ctx, int(which), None, None, 0, C.byref(n)), self.ctx)
        pi = np.zeros(max(1, n.value), dtype=np.int32)
        pj = np.zeros(max(1, n.value), dtype=np.int32)
        _check(load().relres_get_list(self.ctx, int(which), pi.ctypes.data_as(_ip), pj.ctypes.data_as(_ip),
                                      n.value, C.byref(n)), self.ctx)
        return np.stack([pi[: n.value], pj[: n.value]], axis=1)

    def set_prune(self, delta):
        """Pruning margin of the lists in Angstrom (<= 0: no pruning)."""
        _check(load().relres_set_prune(self.ctx, float(delta)), self.ctx)

    def set_pair_config(self, config):
        relres_set_pair_config(self.ctx, config)

    def set_force_accumulation(self, mode):
        """RELRES_ACC_FP32, RELRES_ACC_COMPENSATED or RELRES_ACC_FP64: how the FP32
        pair kernels sum each atom's pair forces."""
        _check(load().relres_set_force_accumulation(self.ctx, int(mode)), self.ctx)

    def set_params(self, params):
        self.params = params
        relres_set_params(self.ctx, params)

    def backward(self, d_pos, d_grad_forces, grad_energy, d_grad_pos=None):
        return relres_backward(self.ctx, self.params.n_types, d_pos, d_grad_forces, grad_energy, d_grad_pos)

    def timings(self):
        return relres_get_timings(self.ctx)

    def close(self):
        if self.ctx:
            relres_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent replicas (Context objects, any sizes) advanced together:
    relres_batch_step runs every block of steps of all of them as one CUDA
    graph.  The contexts stay owned by the caller; close the batch first."""

    def __init__(self, contexts, stream=None):
        self.contexts = list(contexts)
        arr = (C.c_void_p * len(self.contexts))(*[c.ctx for c in self.contexts])
        self._arr = arr
        h = C.c_void_p()
        st = None if stream is None else C.c_void_p(stream.cuda_stream)
        _check(load().relres_batch_create(C.byref(h), arr, len(self.contexts), st))
        self.handle = h

    def step(self, n_steps, dt_fs, d_pos, d_vel, t_target, tau_fs=100.0, seeds=None, thermo_every=0,
             d_thermo=None):
        n = len(self.contexts)
        vp = C.c_void_p
        pos = (vp * n)(*[_ptr(x) for x in d_pos])
        vel = (vp * n)(*[_ptr(x) for x in d_vel])
        tt = np.asarray(t_target, dtype=np.float64).reshape(n)
        sd = (C.c_uint64 * n)(*[int(x) for x in (seeds if seeds is not None else range(n))])
        th = None if d_thermo is None else (vp * n)(*[_ptr(x) for x in d_thermo])
        st = load().relres_batch_step(self.handle, int(n_steps), float(dt_fs), pos, vel,
                                      tt.ctypes.data_as(_dp), float(tau_fs), sd, int(thermo_every), th)
        if st != RELRES_OK:
            msg = (load().relres_batch_last_error(self.handle) or b"").decode()
            raise RelresError(st, msg)

    def set_mode(self, mode):
        """-1: small compatible replicas share launches, the rest own branches;
        0: every replica on its own branch; 1: every replica in shared launches."""
        _check(load().relres_batch_set_mode(self.handle, int(mode)))

    def n_shared(self):
        """Replicas the last step ran in shared launches (-1: no step yet)."""
        v = C.c_int(-1)
        _check(load().relres_batch_get_info(self.handle, C.byref(v)))
        return v.value

    def close(self):
        if self.handle:
            load().relres_batch_destroy(self.handle)
            self.handle = None
