"""Pins of the oracle's parameter preparation (oracle/params.py).

Each check ties the oracle to something other than itself:

* Eq. 13 against its defining sum rule Eq. 4 (u^CG(r) = sum u^FG(r)),
  evaluated term by term at random r: catches a wrong power, a swapped
  A6/A12 or a dropped multiplicity.
* Eq. 15 against Eq. 13 under geometric mixing (two independent closed forms).
* Table 1 (Section 3.2): the printed CG column from the printed FG column.
* Eq. 17 and Eq. 18 against a numeric solve of the boundary conditions
  Eq. 7 and Eq. 8 (5x5 linear systems written from the conditions, not from
  the closed forms); documents that the printed gamma_{4+} sign fails Eq. 8.
* Eq. 19 against the continuity it exists to provide (checked on the
  potential in test_oracle_potential.py).
"""
import math
import os

import numpy as np
import pytest

from oracle import params as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_opls_ua.txt")


def _lj_plain(r, eps, sig):
    return 4.0 * eps * ((sig / r) ** 12 - (sig / r) ** 6)


def _load_table1():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            head, mid, tail = line.split("|")
            name, he, hs = head.split()
            sites = [(float(he), float(hs))]
            m = mid.split()
            for k in range(0, len(m), 3):
                sites += [(float(m[k + 1]), float(m[k + 2]))] * int(m[k])
            ce, cs = (float(x) for x in tail.split())
            rows.append((name, sites, ce, cs))
    return rows


@pytest.mark.parametrize("rule", [P.MIX_GEOMETRIC, P.MIX_LB])
def test_eq13_equals_sum_rule_eq4(rule):
    rng = np.random.default_rng(1)
    nt = 4
    eps = rng.uniform(0.05, 1.0, nt)
    sig = rng.uniform(3.0, 6.5, nt)
    comp_i = np.array([1, 2, 0, 1])
    comp_j = np.array([0, 3, 1, 1])
    E, S = P.mix_fg(eps, sig, rule)
    ecg, scg = P.cg_pair_eq13(comp_i, comp_j, E, S)
    sites_i = [t for t in range(nt) for _ in range(comp_i[t])]
    sites_j = [t for t in range(nt) for _ in range(comp_j[t])]
    for r in rng.uniform(2.5, 20.0, 50):
        direct = 0.0
        for a in sites_i:
            for b in sites_j:
                e_ab = math.sqrt(eps[a] * eps[b])
                s_ab = math.sqrt(sig[a] * sig[b]) if rule == P.MIX_GEOMETRIC else 0.5 * (sig[a] + sig[b])
                direct += _lj_plain(r, e_ab, s_ab)
        assert _lj_plain(r, ecg, scg) == pytest.approx(direct, rel=1e-12, abs=1e-300)


def test_eq15_equals_eq13_under_geometric_mixing():
    rng = np.random.default_rng(2)
    eps_a = rng.uniform(0.1, 1.5, 3)
    sig_a = rng.uniform(3.5, 4.2, 3)
    eps_b = rng.uniform(0.1, 1.5, 5)
    sig_b = rng.uniform(3.5, 4.2, 5)
    ea, sa = P.cg_site_eq15(eps_a, sig_a)
    eb, sb = P.cg_site_eq15(eps_b, sig_b)
    # Eq. 13 over the explicit site lists, geometric cross terms
    eps = np.concatenate([eps_a, eps_b])
    sig = np.concatenate([sig_a, sig_b])
    E, S = P.mix_fg(eps, sig, P.MIX_GEOMETRIC)
    comp_a = np.r_[np.ones(3, int), np.zeros(5, int)]
    comp_b = np.r_[np.zeros(3, int), np.ones(5, int)]
    e13, s13 = P.cg_pair_eq13(comp_a, comp_b, E, S)
    assert math.sqrt(ea * eb) == pytest.approx(e13, rel=1e-12)
    assert math.sqrt(sa * sb) == pytest.approx(s13, rel=1e-12)
    e13aa, s13aa = P.cg_pair_eq13(comp_a, comp_a, E, S)
    assert ea == pytest.approx(e13aa, rel=1e-12)
    assert sa == pytest.approx(s13aa, rel=1e-12)


def test_table1_cg_from_fg_eq15():
    rows = _load_table1()
    assert len(rows) == 8
    for name, sites, ce, cs in rows:
        e, s = P.cg_site_eq15([x[0] for x in sites], [x[1] for x in sites])
        # printed to 4-5 significant digits
        assert e == pytest.approx(ce, rel=5e-4), name
        assert s == pytest.approx(cs, rel=5e-4), name


def test_table1_row_by_eq13_too():
    # the same groups through Eq. 13 with geometric FG cross terms
    for name, sites, ce, cs in _load_table1():
        eps = np.array([x[0] for x in sites])
        sig = np.array([x[1] for x in sites])
        E, S = P.mix_fg(eps, sig, P.MIX_GEOMETRIC)
        comp = np.ones(len(sites), int)
        e, s = P.cg_pair_eq13(comp, comp, E, S)
        assert e == pytest.approx(ce, rel=5e-4), name
        assert s == pytest.approx(cs, rel=5e-4), name


def _solve_conditions(rows, rhs):
    return np.linalg.solve(np.array(rows, float), np.array(rhs, float))


def _poly_rows(delta):
    """Rows giving f(delta), f'(delta), f''(delta) of sum gamma_m delta^m."""
    f = [delta ** m for m in range(5)]
    d1 = [m * delta ** (m - 1) if m >= 1 else 0.0 for m in range(5)]
    d2 = [m * (m - 1) * delta ** (m - 2) if m >= 2 else 0.0 for m in range(5)]
    return f, d1, d2


@pytest.mark.parametrize("r_minus,dr,eps,sig", [(6.0, 1.0, 0.195, 3.75), (13.0, 1.0, 1.39, 3.81),
                                               (0.58, 0.04, 0.8, 0.37), (12.0, 2.0, 21.1, 3.94)])
def test_switch_off_solves_eq7(r_minus, dr, eps, sig):
    u, du, d2u = P.lj(r_minus, eps, sig)
    f0, d10, d20 = _poly_rows(0.0)
    fD, d1D, d2D = _poly_rows(dr)
    g_num = _solve_conditions([f0, d10, d20, d1D, d2D], [u, du, d2u, 0.0, 0.0])
    g = P.switch_off(u, du, d2u, dr)
    np.testing.assert_allclose(g, g_num, rtol=1e-10, atol=1e-12 * max(1.0, abs(u)))


@pytest.mark.parametrize("r_plus,dr,eps,sig", [(7.0, 1.0, 1.39, 3.81), (0.62, 0.04, 14.9, 0.39),
                                              (7.0, 0.5, 21.1, 3.94)])
def test_switch_on_solves_eq8(r_plus, dr, eps, sig):
    u, du, d2u = P.lj(r_plus, eps, sig)
    f0, d10, d20 = _poly_rows(0.0)
    fD, d1D, d2D = _poly_rows(dr)
    g_num = _solve_conditions([fD, d1D, d2D, d10, d20], [u, du, d2u, 0.0, 0.0])
    g = P.switch_on(u, du, d2u, dr)
    np.testing.assert_allclose(g, g_num, rtol=1e-10, atol=1e-12 * max(1.0, abs(u)))
    # the printed Eq. 18 gamma_{4+} (with -u''/(4 dr^2)) violates f''(dr) = u''(r+)
    g_printed = g.copy()
    g_printed[4] = -du / (2 * dr ** 3) - d2u / (4 * dr ** 2)
    curv = sum(g_printed[m] * d2D[m] for m in range(5))
    assert abs(curv - d2u) > 1e-3 * abs(d2u)


def test_derivatives_of_lj_match_finite_differences():
    for r in (3.2, 4.0, 6.5, 13.7):
        u, du, d2u = P.lj(r, 0.3, 3.9)
        h = 1e-5
        assert du == pytest.approx((P.lj(r + h, 0.3, 3.9)[0] - P.lj(r - h, 0.3, 3.9)[0]) / (2 * h), rel=1e-7)
        assert d2u == pytest.approx((P.lj(r + h, 0.3, 3.9)[1] - P.lj(r - h, 0.3, 3.9)[1]) / (2 * h), rel=1e-7)


def test_zero_width_zone():
    u, du, d2u = P.lj(7.0, 1.0, 3.8)
    assert P.poly(P.switch_off(u, du, d2u, 0.0), 0.0) == u
    assert P.poly(P.switch_on(u, du, d2u, 0.0), 0.0) == u


def test_eq19_shift_definitions():
    row = P.pair_row(0.195, 3.75, 1.4, 3.8, (6.0, 7.0, 13.0, 14.0))
    d = P.row_dict(row)
    g_cg_m = [d[f"g_cg_m{m}"] for m in range(5)]
    g_fg_m = [d[f"g_fg_m{m}"] for m in range(5)]
    assert d["Gam_cm"] == pytest.approx(P.poly(g_cg_m, 1.0), rel=1e-15)
    assert d["Gam_sp"] == pytest.approx(P.poly(g_cg_m, 1.0) + P.poly(g_fg_m, 1.0), rel=1e-15)
    assert d["Gam_sm"] == pytest.approx(d["Gam_sp"] - d["g_cg_p0"], rel=1e-15)
    row0 = P.row_dict(P.pair_row(0.195, 3.75, 1.4, 3.8, (6.0, 7.0, 13.0, 14.0), shift=False))
    assert row0["Gam_cm"] == 0.0


def test_ordinary_pairs_get_zero_cg_eq14():
    tab = P.pair_table([0.3, 0.2], [3.9, 3.7], [1, 0], (6, 7, 13, 14), mixing=P.MIX_LB,
                       group_comp=[[1, 2], [0, 0]])
    assert P.row_dict(tab[0])["eps_cg"] > 0
    for k in (1, 2, 3):
        d = P.row_dict(tab[k])
        assert d["eps_cg"] == 0.0
        assert all(d[f"g_cg_p{m}"] == 0.0 for m in range(5))
        assert d["Gam_cm"] == 0.0


def test_radii_order_validated():
    with pytest.raises(ValueError):
        P.pair_row(0.1, 3.9, 1.0, 3.9, (7.0, 6.0, 13.0, 14.0))
    with pytest.raises(ValueError):
        P.pair_row(0.1, 3.9, 1.0, 3.9, (6.0, 7.0, 15.0, 14.0))
