"""GPU parity of the differentiable RelRes pair interaction (relres_backward
through the torch.autograd.Function of paper_2104_10231_gb300.diff) against
the oracle's gradients (direct differentiation of Eq. 11 and Eq. 17-19, pinned
by finite differences in test_oracle_grad.py), and against central finite
differences of the GPU forward itself.

Inputs are seeded synthetic configurations; the CG parameters come from the
oracle's Eq. 13 and are given to both sides as explicit values."""
import math

import numpy as np
import pytest

from oracle import core as O
from oracle import params as P
from paper_2104_10231_gb300 import relres as R
from paper_2104_10231_gb300 import systems as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T

    assert T.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2104_10231_gb300.build import build_library

    build_library()
    R.load()
    return T


def _model(torch, s, ec, sc, precision):
    from paper_2104_10231_gb300 import diff

    mixing = R.RELRES_MIX_LB if s.mixing == "lb" else R.RELRES_MIX_GEOMETRIC
    m = diff.RelResPair(s.types, s.mass_by_type, s.excl, s.is_hybrid, s.radii, s.skin, s.eps_fg, s.sig_fg,
                        ec, sc, mixing=mixing, precision=precision)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    m.bind(pos, s.box)
    return m


def _leaves(torch, s, ec, sc):
    t = lambda a: torch.tensor(np.asarray(a, np.float64), requires_grad=True)
    return t(s.eps_fg), t(s.sig_fg), t(ec), t(sc)


def _oracle_grads(s, ec, sc, pos, g_energy, g_forces):
    eps, sig = s.eps_fg.astype(float), s.sig_fg.astype(float)
    tab = P.pair_table(eps, sig, s.is_hybrid, s.radii, s.mixing, eps_cg=ec, sig_cg=sc)
    dtab = P.table_derivs(eps, sig, s.is_hybrid, s.radii, s.mixing, eps_cg=ec, sig_cg=sc)
    g = O.pair_param_grads(pos, s.box, s.types, tab, dtab, s.n_types, g_energy, g_forces, s.excl)
    d_eps, d_sig, d_ecg, d_scg = P.chain_to_types(g, eps, sig, s.mixing)
    f, e, _ = O.pair_forces(pos, s.box, s.types, tab, s.n_types, s.excl)
    dx = -g_energy * f
    if g_forces is not None:
        dx = dx - O.pair_hvp(pos, s.box, s.types, tab, s.n_types, g_forces, s.excl)
    return (d_eps, d_sig, d_ecg, d_scg), dx, f, e


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def _compare(torch, s, precision, tol_p, tol_x, with_energy=True, with_forces=True, seed=0):
    ec, sc = P.cg_table_eq13(s.eps_fg, s.sig_fg, s.is_hybrid, s.group_comp, s.mixing)
    m = _model(torch, s, ec, sc, precision)
    # fitting target: oracle forces of perturbed parameters
    tab_ref = P.pair_table(s.eps_fg * 1.1, s.sig_fg * 0.98, s.is_hybrid, s.radii, s.mixing,
                           eps_cg=ec * 0.9, sig_cg=sc * 1.02)
    f_ref, _, _ = O.pair_forces(s.pos, s.box, s.types, tab_ref, s.n_types, s.excl)
    leaves = _leaves(torch, s, ec, sc)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda", requires_grad=True)
    e, f = m(pos, *leaves)
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    if with_energy:
        loss = loss + e
    if with_forces:
        loss = loss + ((f - torch.tensor(f_ref, device="cuda")) ** 2).sum()
    loss.backward()
    f_gpu = f.detach().cpu().numpy()
    g_forces = 2.0 * (f_gpu - f_ref) if with_forces else None
    (d_eps, d_sig, d_ecg, d_scg), dx, _, _ = _oracle_grads(s, ec, sc, s.pos, 1.0 if with_energy else 0.0,
                                                           g_forces)
    errs = {"eps_fg": _rel(leaves[0].grad.numpy(), d_eps), "sig_fg": _rel(leaves[1].grad.numpy(), d_sig),
            "eps_cg": _rel(leaves[2].grad.numpy(), d_ecg), "sig_cg": _rel(leaves[3].grad.numpy(), d_scg),
            "pos": _rel(pos.grad.cpu().numpy(), dx)}
    print(f"{s.name} N={s.n_atoms} prec={precision} E={with_energy} F={with_forces}: " +
          " ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    for k in ("eps_fg", "sig_fg", "eps_cg", "sig_cg"):
        assert errs[k] <= tol_p, (k, errs[k])
    assert errs["pos"] <= tol_x, errs["pos"]
    m.close()
    return errs


def test_fp64_energy_gradient_matches_oracle(torch):
    _compare(torch, S.neopentane(n_mol=250, seed=21), R.RELRES_PREC_FP64, 1e-9, 1e-9, with_forces=False)


def test_fp64_force_matching_gradient_matches_oracle(torch):
    _compare(torch, S.neopentane(n_mol=250, seed=21), R.RELRES_PREC_FP64, 1e-9, 1e-9)


def test_fp64_energy_plus_force_matching_propane(torch):
    _compare(torch, S.propane(), R.RELRES_PREC_FP64, 1e-9, 1e-9)


def test_fp32_force_matching_gradient_matches_oracle(torch):
    _compare(torch, S.neopentane(n_mol=500, seed=5), R.RELRES_PREC_FP32, 2e-5, 1e-4)


def test_fp32_block_copolymer_gradient_matches_oracle(torch):
    _compare(torch, S.block_copolymer(n_chain=20), R.RELRES_PREC_FP32, 2e-5, 1e-4)


def test_fp32_snapshots_of_the_20000_atom_liquid(torch):
    # the differentiable workload: seeded snapshots of the 20 000-atom liquid,
    # one context reused across snapshots (lists rebuilt as needed)
    snaps = [S.neopentane(n_mol=4000, seed=300 + k) for k in range(2)]
    s0 = snaps[0]
    ec, sc = P.cg_table_eq13(s0.eps_fg, s0.sig_fg, s0.is_hybrid, s0.group_comp, s0.mixing)
    m = _model(torch, s0, ec, sc, R.RELRES_PREC_FP32)
    leaves = _leaves(torch, s0, ec, sc)
    total = None
    for s in snaps:
        pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
        e, f = m(pos, *leaves)
        term = e + (f ** 2).sum() * 1e-3
        total = term if total is None else total + term
    total.backward()
    ref = [np.zeros(2), np.zeros(2), np.zeros((2, 2)), np.zeros((2, 2))]
    for s in snaps:
        tab = P.pair_table(s.eps_fg, s.sig_fg, s.is_hybrid, s.radii, s.mixing, eps_cg=ec, sig_cg=sc)
        f, _, _ = O.pair_forces(s.pos, s.box, s.types, tab, s.n_types, s.excl)
        (a, b, c, d), _, _, _ = _oracle_grads(s, ec, sc, s.pos, 1.0, 2e-3 * f)
        for r, x in zip(ref, (a, b, c, d)):
            r += x
    for leaf, r, name in zip(leaves, ref, ("eps_fg", "sig_fg", "eps_cg", "sig_cg")):
        err = _rel(leaf.grad.numpy(), r)
        print(f"20000-atom snapshots {name}: {err:.2e}")
        assert err <= 2e-5, (name, err)
    m.close()


def test_fp64_gradient_matches_central_differences_of_the_gpu_forward(torch):
    # independent of the oracle: Richardson-extrapolated central differences
    # of the GPU loss with respect to one FG sigma and one CG epsilon
    s = S.neopentane(n_mol=250, seed=8)
    ec, sc = P.cg_table_eq13(s.eps_fg, s.sig_fg, s.is_hybrid, s.group_comp, s.mixing)
    m = _model(torch, s, ec, sc, R.RELRES_PREC_FP64)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")

    def loss(eps, sig, ecg, scg):
        e, f = m(pos, torch.tensor(eps), torch.tensor(sig), torch.tensor(ecg), torch.tensor(scg))
        return float(e) + float((f ** 2).sum()) * 1e-3

    leaves = _leaves(torch, s, ec, sc)
    e, f = m(pos, *leaves)
    (e + (f ** 2).sum() * 1e-3).backward()
    base = [s.eps_fg.astype(float), s.sig_fg.astype(float), ec.copy(), sc.copy()]
    for k, idx in ((1, (1,)), (2, (0, 0)), (3, (0, 0))):
        h = 1e-4 * abs(base[k][idx])

        def central(step):
            vals = []
            for sgn in (1.0, -1.0):
                a = [x.copy() for x in base]
                a[k][idx] += sgn * step
                vals.append(loss(*a))
            return (vals[0] - vals[1]) / (2 * step)

        fd = (4.0 * central(h) - central(2 * h)) / 3.0
        an = float(leaves[k].grad.numpy()[idx])
        print(f"FD check param {k}{idx}: analytic {an:.10e} fd {fd:.10e}")
        assert an == pytest.approx(fd, rel=1e-6)
    m.close()


def _compare_eq13(torch, s, precision, tol_p, tol_x):
    # CG parameters that follow Eq. 13: the leaves are the FG parameters only
    from paper_2104_10231_gb300 import diff

    m = diff.RelResPair.for_system(s, precision=precision)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda", requires_grad=True)
    m.bind(pos.detach(), s.box)
    ec, sc = P.cg_table_eq13(s.eps_fg, s.sig_fg, s.is_hybrid, s.group_comp, s.mixing)
    tab_ref = P.pair_table(s.eps_fg * 1.1, s.sig_fg * 0.98, s.is_hybrid, s.radii, s.mixing,
                           eps_cg=ec * 0.9, sig_cg=sc * 1.02)
    f_ref, _, _ = O.pair_forces(s.pos, s.box, s.types, tab_ref, s.n_types, s.excl)
    eps = torch.tensor(s.eps_fg.astype(float), requires_grad=True)
    sig = torch.tensor(s.sig_fg.astype(float), requires_grad=True)
    e, f = m(pos, eps, sig)
    loss = e + ((f - torch.tensor(f_ref, device="cuda")) ** 2).sum()
    loss.backward()
    g_forces = 2.0 * (f.detach().cpu().numpy() - f_ref)
    (d_eps, d_sig, d_ecg, d_scg), dx, _, _ = _oracle_grads(s, ec, sc, s.pos, 1.0, g_forces)
    t_eps, t_sig = P.chain_cg_eq13(d_eps, d_sig, d_ecg, d_scg, s.eps_fg.astype(float), s.sig_fg.astype(float),
                                   s.is_hybrid, s.group_comp, s.mixing)
    errs = {"eps_fg": _rel(eps.grad.numpy(), t_eps), "sig_fg": _rel(sig.grad.numpy(), t_sig),
            "pos": _rel(pos.grad.cpu().numpy(), dx)}
    print(f"Eq. 13 chain {s.name} N={s.n_atoms} prec={precision}: " + " ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert errs["eps_fg"] <= tol_p and errs["sig_fg"] <= tol_p, errs
    assert errs["pos"] <= tol_x, errs
    # the CG path is part of the answer: the direct FG gradient alone is far off
    assert _rel(d_eps, t_eps) > 10 * tol_p
    m.close()


def test_fp64_gradient_through_eq13_matches_oracle(torch):
    _compare_eq13(torch, S.neopentane(n_mol=250, seed=21), R.RELRES_PREC_FP64, 1e-9, 1e-9)


def test_fp64_gradient_through_eq13_propane(torch):
    _compare_eq13(torch, S.propane(), R.RELRES_PREC_FP64, 1e-9, 1e-9)


def test_fp32_gradient_through_eq13_block_copolymer(torch):
    # two hybrid types: the A-A, A-B and B-B CG pairs all depend on every FG type
    _compare_eq13(torch, S.block_copolymer(n_chain=20), R.RELRES_PREC_FP32, 2e-5, 1e-4)


def test_fp64_eq13_gradient_matches_central_differences_of_the_gpu_forward(torch):
    # independent of the oracle: differences of the GPU loss with the CG
    # parameters re-derived by the library (Eq. 13) at every displaced FG value
    from paper_2104_10231_gb300 import diff

    s = S.neopentane(n_mol=250, seed=8)
    m = diff.RelResPair.for_system(s, precision=R.RELRES_PREC_FP64)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    m.bind(pos, s.box)

    def loss(eps, sig):
        e, f = m(pos, torch.tensor(eps), torch.tensor(sig))
        return float(e) + float((f ** 2).sum()) * 1e-3

    eps = torch.tensor(s.eps_fg.astype(float), requires_grad=True)
    sig = torch.tensor(s.sig_fg.astype(float), requires_grad=True)
    e, f = m(pos, eps, sig)
    (e + (f ** 2).sum() * 1e-3).backward()
    e0, s0 = s.eps_fg.astype(float), s.sig_fg.astype(float)
    for k, (arr, grad) in enumerate(((e0, eps.grad.numpy()), (s0, sig.grad.numpy()))):
        for t in range(len(arr)):
            h = 1e-4 * arr[t]

            def central(step):
                up, dn = arr.copy(), arr.copy()
                up[t] += step
                dn[t] -= step
                if k == 0:
                    return (loss(up, s0) - loss(dn, s0)) / (2 * step)
                return (loss(e0, up) - loss(e0, dn)) / (2 * step)

            fd = (4.0 * central(h) - central(2 * h)) / 3.0
            print(f"d/d{'eps' if k == 0 else 'sig'}[{t}]: {grad[t]:.10e} vs {fd:.10e}")
            assert abs(grad[t] - fd) <= 1e-6 * abs(fd) + 1e-9, (k, t, grad[t], fd)
    m.close()
