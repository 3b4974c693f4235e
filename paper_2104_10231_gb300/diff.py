"""Differentiable RelRes pair interaction for PyTorch.

``RelResPair(...)(pos, eps_fg, sig_fg, eps_cg, sig_cg)`` returns the pair
energy E (Eq. 20 summed over all non-excluded pairs, Eq. 3) and the pair
forces F = -dE/dx of one configuration, computed by librelres on the GPU.
Backpropagation goes through the library's backward kernel
(``relres_backward``): dL/dx (a Hessian-vector product of E with dL/dF, plus
dL/dE times dE/dx) and dL/d(eps_fg, sig_fg) per type (through the mixing
rule), dL/d(eps_cg, sig_cg) per type pair (independent variables).

``RelResPair(...)(pos, eps_fg, sig_fg)`` (CG parameters omitted; the model
knows the group compositions) makes the CG parameters of every hybrid type
pair follow Eq. 13 from the FG ones: the leaves are the FG parameters only,
and their gradients include the path through the CG parameters
(``relres_chain_cg_grads``, the chain rule through Eq. 13 in the library).

Neighbour lists are kept by the library and rebuilt when an atom moved more
than half the skin; nothing else is stored between the passes.

Only argument marshalling happens here: parameter values go to the library
with ``relres_set_params``; every arithmetic step runs in librelres.
"""
from __future__ import annotations

import numpy as np
import torch

from . import relres as R


def cg_table(eps_fg, sig_fg, is_hybrid, group_comp, mixing=R.RELRES_MIX_LB):
    """CG pair parameters of every hybrid type pair by Eq. 13 (through the
    library's relres_cg_params); zero for pairs with an ordinary type (Eq. 14)."""
    nt = len(eps_fg)
    ec = np.zeros((nt, nt))
    sc = np.zeros((nt, nt))
    for a in range(nt):
        for b in range(nt):
            if is_hybrid[a] and is_hybrid[b]:
                ec[a, b], sc[a, b] = R.relres_cg_params(eps_fg, sig_fg, mixing, group_comp[a], group_comp[b])
    return ec, sc


class RelResPair:
    """Owns a librelres context with a pair-only topology (types, masses,
    exclusions; no bonded terms) for one system size."""

    def __init__(self, types, mass_by_type, excl, is_hybrid, radii, skin, eps_fg, sig_fg, eps_cg, sig_cg,
                 mixing=R.RELRES_MIX_LB, shift=True, precision=R.RELRES_PREC_FP64, stream=None, group_comp=None):
        self.n_types = len(is_hybrid)
        self.is_hybrid = np.asarray(is_hybrid, np.int32)
        # group compositions [n_types, n_types] (Eq. 13), for calls without CG parameters
        self.group_comp = None if group_comp is None else np.asarray(group_comp, np.int32).reshape(
            self.n_types, self.n_types)
        self.radii = tuple(float(x) for x in radii)
        self.skin = float(skin)
        self.mixing = mixing
        self.shift = shift
        self.precision = precision
        params = self._params(eps_fg, sig_fg, eps_cg, sig_cg)
        self.ctx = R.Context(params, R.make_topology(types, mass_by_type, excl, None), stream=stream)
        self.box = None

    @classmethod
    def for_system(cls, system, precision=R.RELRES_PREC_FP64, stream=None):
        """Context for a ``systems.System`` with its own parameters; the CG
        parameters start at their Eq. 13 values."""
        mixing = R.RELRES_MIX_LB if system.mixing == "lb" else R.RELRES_MIX_GEOMETRIC
        ec, sc = cg_table(system.eps_fg, system.sig_fg, system.is_hybrid, system.group_comp, mixing)
        obj = cls(system.types, system.mass_by_type, system.excl, system.is_hybrid, system.radii, system.skin,
                  system.eps_fg, system.sig_fg, ec, sc, mixing=mixing, precision=precision, stream=stream,
                  group_comp=system.group_comp)
        obj.cg0 = (ec, sc)
        return obj

    def _params(self, eps_fg, sig_fg, eps_cg, sig_cg):
        return R.make_params(np.asarray(eps_fg, np.float64), np.asarray(sig_fg, np.float64), self.is_hybrid,
                             self.radii, self.skin, mixing=self.mixing,
                             eps_cg=np.asarray(eps_cg, np.float64).reshape(-1),
                             sig_cg=np.asarray(sig_cg, np.float64).reshape(-1), shift=self.shift,
                             precision=self.precision)

    def set_params(self, eps_fg, sig_fg, eps_cg, sig_cg):
        self.ctx.set_params(self._params(eps_fg, sig_fg, eps_cg, sig_cg))

    def bind(self, pos, box):
        """Build the lists for a first configuration of this system (device
        positions, N x 3 float64) in a box."""
        self.box = np.asarray(box, np.float64)
        self.ctx.build_neighbors(pos, self.box)

    def __call__(self, pos, eps_fg, sig_fg, eps_cg=None, sig_cg=None):
        """(E, F) at device positions pos (N x 3 float64) and the given
        parameters (tensors: eps_fg, sig_fg [n_types]; eps_cg, sig_cg
        [n_types, n_types], or both omitted to take them from Eq. 13)."""
        if self.box is None:
            raise RuntimeError("RelResPair.bind(pos, box) first")
        if eps_cg is None and sig_cg is None:
            if self.group_comp is None:
                raise ValueError("CG parameters omitted: the model needs group compositions (Eq. 13)")
            return _RelResPairEq13Fn.apply(self, pos, eps_fg, sig_fg)
        if eps_cg is None or sig_cg is None:
            raise ValueError("give both eps_cg and sig_cg, or neither")
        return _RelResPairFn.apply(self, pos, eps_fg, sig_fg, eps_cg, sig_cg)

    def cg_from_fg(self, eps_fg, sig_fg):
        """Eq. 13 CG parameters (eps_cg, sig_cg [n_types, n_types]) of FG
        parameters given as arrays (through the library)."""
        return cg_table(eps_fg, sig_fg, self.is_hybrid, self.group_comp, self.mixing)

    def close(self):
        self.ctx.close()


def _host(t):
    return t.detach().to("cpu", dtype=torch.float64).numpy()


class _RelResPairFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, owner, pos, eps_fg, sig_fg, eps_cg, sig_cg):
        params = [_host(t) for t in (eps_fg, sig_fg, eps_cg, sig_cg)]
        owner.set_params(*params)
        pos = pos.detach().contiguous()
        f = torch.empty_like(pos)
        e = torch.zeros(4, dtype=torch.float64, device=pos.device)
        owner.ctx.compute(pos, f, e)
        ctx.owner = owner
        ctx.params = params
        ctx.save_for_backward(pos)
        ctx.param_meta = [(t.dtype, t.device, t.shape) for t in (eps_fg, sig_fg, eps_cg, sig_cg)]
        # the context holds no bonded terms: e[3] is the pair energy E_FG + E_CG
        return e[3], f

    @staticmethod
    def backward(ctx, g_energy, g_forces):
        (pos,) = ctx.saved_tensors
        owner = ctx.owner
        owner.set_params(*ctx.params)
        ge = 0.0 if g_energy is None else float(g_energy)
        gf = None if g_forces is None else g_forces.detach().to(torch.float64).contiguous()
        gx = torch.empty_like(pos)
        out = owner.ctx.backward(pos, gf, ge, gx)
        grads = []
        for key, (dtype, device, shape) in zip(("eps_fg", "sig_fg", "eps_cg", "sig_cg"), ctx.param_meta):
            grads.append(torch.as_tensor(out[key].reshape(shape), dtype=dtype, device=device))
        return (None, gx, *grads)


class _RelResPairEq13Fn(torch.autograd.Function):
    """(E, F) with CG parameters that follow Eq. 13 from the FG leaves."""

    @staticmethod
    def forward(ctx, owner, pos, eps_fg, sig_fg):
        ef, sf = _host(eps_fg), _host(sig_fg)
        ec, sc = owner.cg_from_fg(ef, sf)
        owner.set_params(ef, sf, ec, sc)
        pos = pos.detach().contiguous()
        f = torch.empty_like(pos)
        e = torch.zeros(4, dtype=torch.float64, device=pos.device)
        owner.ctx.compute(pos, f, e)
        ctx.owner = owner
        ctx.params = [ef, sf, ec, sc]
        ctx.save_for_backward(pos)
        ctx.param_meta = [(t.dtype, t.device, t.shape) for t in (eps_fg, sig_fg)]
        return e[3], f

    @staticmethod
    def backward(ctx, g_energy, g_forces):
        (pos,) = ctx.saved_tensors
        owner = ctx.owner
        ef, sf, ec, sc = ctx.params
        owner.set_params(ef, sf, ec, sc)
        ge = 0.0 if g_energy is None else float(g_energy)
        gf = None if g_forces is None else g_forces.detach().to(torch.float64).contiguous()
        gx = torch.empty_like(pos)
        out = owner.ctx.backward(pos, gf, ge, gx)
        p = R.make_params(ef, sf, owner.is_hybrid, owner.radii, owner.skin, mixing=owner.mixing,
                          group_comp=owner.group_comp, shift=owner.shift, precision=owner.precision)
        d_eps, d_sig = R.relres_chain_cg_grads(p, out["eps_cg"], out["sig_cg"], out["eps_fg"], out["sig_fg"])
        grads = [torch.as_tensor(g.reshape(shape), dtype=dtype, device=device)
                 for g, (dtype, device, shape) in zip((d_eps, d_sig), ctx.param_meta)]
        return (None, gx, *grads)
