"""Pins of the oracle's differentiable form (parameter gradients and the
Hessian-vector product of Eq. 20) against what mathematics fixes:
finite differences of the oracle's own energy and forces (independent of the
derivative code), the exact linearity of Eq. 20 in eps, and finite differences
of the record construction of Eq. 17-19."""
import numpy as np
import pytest

from oracle import core as O
from oracle import params as P
from paper_2104_10231_gb300 import systems as S

RADII = (6.0, 7.0, 13.0, 14.0)


def _rows():
    # an ordinary pair, a hybrid pair, a hybrid pair with zero-width shells
    return [P.pair_row(0.195, 3.75, 0.0, 0.0, RADII),
            P.pair_row(0.0914, 3.95, 1.2, 4.6, RADII),
            P.pair_row(0.15, 3.8, 0.9, 4.4, (6.5, 6.5, 13.5, 13.5))]


def test_second_derivative_matches_finite_differences_in_every_region():
    h = 1e-5
    for row in _rows():
        # points inside each of the five regions (away from the boundaries)
        r = np.array([3.6, 4.5, 5.5, 6.3, 6.7, 9.0, 12.5, 13.3, 13.8, 14.5])
        r = r[np.abs(r[:, None] - np.array(row[4:8])[None, :]).min(1) > 2e-3]
        d2 = O.u_tilde_d2(row, r)
        _, dup = O.u_tilde(row, r + h)
        _, dum = O.u_tilde(row, r - h)
        fd = (dup - dum) / (2 * h)
        assert np.allclose(d2, fd, rtol=1e-6, atol=1e-9 * np.abs(fd).max() + 1e-12), (d2, fd)


def test_record_derivatives_match_finite_differences_of_the_construction():
    base = dict(eps_fg=0.12, sig_fg=3.9, eps_cg=1.1, sig_cg=4.5)
    for radii in (RADII, (6.5, 6.5, 13.5, 13.5)):
        d = P.pair_row_derivs(base["eps_fg"], base["sig_fg"], base["eps_cg"], base["sig_cg"], radii)
        for k, name in enumerate(P.PARAMS):
            h = 1e-6 * base[name]
            up = dict(base)
            dn = dict(base)
            up[name] += h
            dn[name] -= h
            fd = (P.pair_row(**up, radii=radii) - P.pair_row(**dn, radii=radii)) / (2 * h)
            scale = np.abs(fd).max()
            assert np.allclose(d[k], fd, rtol=1e-6, atol=1e-8 * scale), (name, d[k] - fd)


def _system():
    # 250 neopentane-like molecules: two types, hybrids, exclusions; small box
    return S.neopentane(n_mol=250, seed=21)


def _energy(s, eps, sig, ecg, scg):
    tab = P.pair_table(eps, sig, s.is_hybrid, s.radii, s.mixing, eps_cg=ecg, sig_cg=scg)
    f, e, w = O.pair_forces(s.pos, s.box, s.types, tab, s.n_types, s.excl)
    return e, f


def _cg(s):
    return P.cg_table_eq13(s.eps_fg, s.sig_fg, s.is_hybrid, s.group_comp, s.mixing)


def _grads(s, eps, sig, ecg, scg, g_energy, g_forces):
    tab = P.pair_table(eps, sig, s.is_hybrid, s.radii, s.mixing, eps_cg=ecg, sig_cg=scg)
    dtab = P.table_derivs(eps, sig, s.is_hybrid, s.radii, s.mixing, eps_cg=ecg, sig_cg=scg)
    g = O.pair_param_grads(s.pos, s.box, s.types, tab, dtab, s.n_types, g_energy, g_forces, s.excl)
    return P.chain_to_types(g, eps, sig, s.mixing)


def _fd_params(fun, eps, sig, ecg, scg, rel=1e-4):
    """Central differences of fun (step rel * |value|, Richardson-extrapolated
    with the 2h difference so that the O(h^2) error of the steep LJ powers
    drops out) over every per-type FG parameter and every CG entry with
    eps_cg > 0."""
    out = {}
    names = ("eps", "sig", "ecg", "scg")
    for name, arr in zip(names, (eps, sig, ecg, scg)):
        for idx in np.ndindex(arr.shape):
            if arr[idx] == 0.0:
                continue
            h = rel * abs(arr[idx])

            def central(step):
                vals = []
                for sgn in (1.0, -1.0):
                    a = [x.copy() for x in (eps, sig, ecg, scg)]
                    a[names.index(name)][idx] += sgn * step
                    vals.append(fun(*a))
                return (vals[0] - vals[1]) / (2 * step)

            out[(name, idx)] = (4.0 * central(h) - central(2 * h)) / 3.0
    return out


def _check_against_fd(an, fd, rtol):
    d_eps, d_sig, d_ecg, d_scg = an
    table = {"eps": d_eps, "sig": d_sig, "ecg": d_ecg, "scg": d_scg}
    scale = max(abs(v) for v in fd.values())
    for (name, idx), v in fd.items():
        a = table[name][idx]
        assert abs(a - v) <= rtol * abs(v) + 1e-7 * scale, (name, idx, a, v)


def test_energy_gradient_matches_finite_differences():
    s = _system()
    ecg, scg = _cg(s)
    eps, sig = s.eps_fg.astype(float), s.sig_fg.astype(float)
    an = _grads(s, eps, sig, ecg, scg, 1.0, None)
    fd = _fd_params(lambda *a: _energy(s, *a)[0], eps, sig, ecg, scg)
    assert len(fd) == 6  # eps, sig of both types; eps_cg, sig_cg of the hybrid pair
    _check_against_fd(an, fd, 2e-6)


def test_energy_is_linear_in_eps():
    # Eq. 20 scales with eps: E = sum_rows eps_fg dE/deps_fg + eps_cg dE/deps_cg
    s = _system()
    ecg, scg = _cg(s)
    eps, sig = s.eps_fg.astype(float), s.sig_fg.astype(float)
    tab = P.pair_table(eps, sig, s.is_hybrid, s.radii, s.mixing, eps_cg=ecg, sig_cg=scg)
    dtab = P.table_derivs(eps, sig, s.is_hybrid, s.radii, s.mixing, eps_cg=ecg, sig_cg=scg)
    g = O.pair_param_grads(s.pos, s.box, s.types, tab, dtab, s.n_types, 1.0, None, s.excl)
    e, _ = _energy(s, eps, sig, ecg, scg)
    lin = (tab[:, 0] * g[:, 0]).sum() + (tab[:, 2] * g[:, 2]).sum()
    assert lin == pytest.approx(e, rel=1e-11)


def test_force_matching_gradient_matches_finite_differences():
    s = _system()
    ecg, scg = _cg(s)
    eps, sig = s.eps_fg.astype(float), s.sig_fg.astype(float)
    # reference forces from perturbed parameters (a fitting target)
    _, f_ref = _energy(s, eps * 1.1, sig * 0.98, ecg * 0.9, scg * 1.02)

    def loss(*a):
        return float(((_energy(s, *a)[1] - f_ref) ** 2).sum())

    _, f = _energy(s, eps, sig, ecg, scg)
    an = _grads(s, eps, sig, ecg, scg, 0.0, 2.0 * (f - f_ref))
    fd = _fd_params(loss, eps, sig, ecg, scg)
    _check_against_fd(an, fd, 2e-6)


def test_hessian_vector_product_matches_finite_differences_of_forces():
    s = _system()
    tab = O.table_for(s)
    rng = np.random.default_rng(3)
    v = rng.normal(size=s.pos.shape)
    hv = O.pair_hvp(s.pos, s.box, s.types, tab, s.n_types, v, s.excl)
    h = 1e-5
    fp, _, _ = O.pair_forces(s.pos + h * v, s.box, s.types, tab, s.n_types, s.excl)
    fm, _, _ = O.pair_forces(s.pos - h * v, s.box, s.types, tab, s.n_types, s.excl)
    fd = -(fp - fm) / (2 * h)  # forces change by -H v
    scale = np.abs(fd).max()
    assert np.abs(hv - fd).max() <= 1e-6 * scale, np.abs(hv - fd).max() / scale
    # H is symmetric: v . H w = w . H v
    w = rng.normal(size=s.pos.shape)
    hw = O.pair_hvp(s.pos, s.box, s.types, tab, s.n_types, w, s.excl)
    assert (v * hw).sum() == pytest.approx((w * hv).sum(), rel=1e-10)


def test_planted_sign_error_in_a_derivative_record_is_caught():
    # flip the sign of the sig_cg derivative of Gamma_{c-}: the energy gradient
    # check must fail
    s = _system()
    ecg, scg = _cg(s)
    eps, sig = s.eps_fg.astype(float), s.sig_fg.astype(float)
    tab = P.pair_table(eps, sig, s.is_hybrid, s.radii, s.mixing, eps_cg=ecg, sig_cg=scg)
    dtab = P.table_derivs(eps, sig, s.is_hybrid, s.radii, s.mixing, eps_cg=ecg, sig_cg=scg)
    dtab[:, 3, P.ROW_FIELDS.index("Gam_cm")] *= -1.0
    g = O.pair_param_grads(s.pos, s.box, s.types, tab, dtab, s.n_types, 1.0, None, s.excl)
    an = P.chain_to_types(g, eps, sig, s.mixing)
    fd = _fd_params(lambda *a: _energy(s, *a)[0], eps, sig, ecg, scg)
    with pytest.raises(AssertionError):
        _check_against_fd(an, fd, 2e-6)


def test_energy_gradient_geometric_mixing():
    # the other mixing rule of the chain to per-type parameters
    s = _system().subset_copy(mixing="geometric")
    ecg, scg = _cg(s)
    eps, sig = s.eps_fg.astype(float), s.sig_fg.astype(float)
    an = _grads(s, eps, sig, ecg, scg, 1.0, None)
    fd = _fd_params(lambda *a: _energy(s, *a)[0], eps, sig, ecg, scg)
    _check_against_fd(an, fd, 2e-6)


@pytest.mark.parametrize("rule", [P.MIX_LB, P.MIX_GEOMETRIC])
def test_eq13_vector_jacobian_product_matches_finite_differences(rule):
    # d(gE eps^CG + gS sig^CG)/d(eps_t, sig_t) of every hybrid group pair of
    # three systems (one, one and two hybrid types) against Richardson
    # differences of Eq. 13 through the mixing rule
    rng = np.random.default_rng(4)
    for s in (S.neopentane(n_mol=250, seed=21), S.propane(), S.block_copolymer(n_chain=4)):
        eps, sig = s.eps_fg.astype(float), s.sig_fg.astype(float)
        nt = len(eps)
        for a in range(nt):
            for b in range(nt):
                if not (s.is_hybrid[a] and s.is_hybrid[b]):
                    continue
                ci, cj = s.group_comp[a], s.group_comp[b]
                g_e, g_s = rng.normal(), rng.normal()
                d_eps, d_sig = P.cg_pair_eq13_vjp(ci, cj, eps, sig, g_e, g_s, rule)

                def f(e, sg):
                    E, Sm = P.mix_fg(e, sg, rule)
                    ec, sc = P.cg_pair_eq13(ci, cj, E, Sm)
                    return g_e * ec + g_s * sc

                for t in range(nt):
                    for k, arr, d in ((0, eps, d_eps), (1, sig, d_sig)):
                        h = 1e-4 * arr[t]

                        def central(step):
                            up, dn = arr.copy(), arr.copy()
                            up[t] += step
                            dn[t] -= step
                            if k == 0:
                                return (f(up, sig) - f(dn, sig)) / (2 * step)
                            return (f(eps, up) - f(eps, dn)) / (2 * step)

                        fd = (4.0 * central(h) - central(2 * h)) / 3.0
                        assert abs(d[t] - fd) <= 1e-8 * abs(fd) + 1e-12, (s.name, rule, a, b, k, t, d[t], fd)


def test_energy_gradient_through_eq13_matches_finite_differences():
    # CG parameters that follow Eq. 13 from the FG ones: the chained gradient
    # (direct FG part + Eq. 13 vector-Jacobian products of the CG part)
    # against differences of the energy with the CG table recomputed at every
    # displaced FG parameter
    s = _system()
    eps, sig = s.eps_fg.astype(float), s.sig_fg.astype(float)
    ecg, scg = _cg(s)
    d_eps, d_sig, d_ecg, d_scg = _grads(s, eps, sig, ecg, scg, 1.0, None)
    t_eps, t_sig = P.chain_cg_eq13(d_eps, d_sig, d_ecg, d_scg, eps, sig, s.is_hybrid, s.group_comp, s.mixing)

    def energy(e, sg):
        ec, sc = P.cg_table_eq13(e, sg, s.is_hybrid, s.group_comp, s.mixing)
        return _energy(s, e, sg, ec, sc)[0]

    scale = max(np.abs(t_eps).max(), np.abs(t_sig).max())
    for k, arr, an in ((0, eps, t_eps), (1, sig, t_sig)):
        for t in range(len(arr)):
            h = 1e-4 * arr[t]

            def central(step):
                up, dn = arr.copy(), arr.copy()
                up[t] += step
                dn[t] -= step
                if k == 0:
                    return (energy(up, sig) - energy(dn, sig)) / (2 * step)
                return (energy(eps, up) - energy(eps, dn)) / (2 * step)

            fd = (4.0 * central(h) - central(2 * h)) / 3.0
            assert abs(an[t] - fd) <= 2e-6 * abs(fd) + 1e-7 * scale, (k, t, an[t], fd)
    # the CG path matters here: the chained gradient differs from the direct one
    assert np.abs(t_eps - d_eps).max() > 1e-3 * np.abs(t_eps).max()
