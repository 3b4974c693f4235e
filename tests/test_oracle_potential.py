"""Pins of the oracle's RelRes potential, Eq. 20 (oracle/relres_oracle.c).

* C0/C1/C2 continuity at r_s-, r_s+, r_c-, r_c+ (Section 2.2 asks for
  continuous energy, force and force derivative), u(r_c+) = 0, u = u' = 0
  beyond r_c+.
* u' against central differences of u inside every region (catches a
  derivative that does not belong to its energy).
* Region 1: -u' is the textbook LJ force 24 eps/r [2 (s/r)^12 - (s/r)^6]
  and u - u^FG is the constant -Gamma_{s-}.
* Region 3: -u' is the textbook LJ force with the CG parameters.
* Ordinary pairs (Eq. 14): u = 0 for r >= r_s+.
* Limits (Section 2.1): eps^CG = 0 with r_s -> r_c gives the FG reference;
  all-hybrid n = 1 groups make u^CG = u^FG so the force is plain LJ outside
  the two smoothing zones.
"""
import numpy as np
import pytest

from oracle import core as O
from oracle import params as P

RADII = (6.0, 7.0, 13.0, 14.0)


def _lj_force(r, eps, sig):
    return 24.0 * eps / r * (2.0 * (sig / r) ** 12 - (sig / r) ** 6)


def _rows():
    yield "hybrid", P.pair_row(0.0914, 3.95, 1.3914, 3.8099, RADII)
    yield "neo_hybrid", P.pair_row(0.0005, 6.4, 2.1, 5.3, RADII)
    yield "ordinary", P.pair_row(0.195, 3.75, 0.0, 0.0, RADII)
    yield "mixed_radii", P.pair_row(0.3, 3.9, 2.5, 4.1, (5.5, 6.5, 12.0, 14.0))
    yield "noshift", P.pair_row(0.0914, 3.95, 1.3914, 3.8099, RADII, shift=False)


@pytest.mark.parametrize("name,row", list(_rows()))
def test_continuity_at_every_radius(name, row):
    d = P.row_dict(row)
    for r0 in (d["rsm"], d["rsp"], d["rcm"], d["rcp"]):
        h = 1e-7
        u, du = O.u_tilde(row, [r0 - h, r0, r0 + h])
        scale = max(1e-3, abs(u).max())
        if name == "noshift" and r0 == d["rcp"]:
            # shift off: the energy jumps at r_c+ by Gamma_{c-} (reading 3)
            assert abs(u[0]) == pytest.approx(abs(P.poly([d[f"g_cg_m{m}"] for m in range(5)], 1.0)),
                                              rel=1e-4)
        else:
            assert abs(u[0] - u[2]) < 1e-6 * scale, (name, r0)
        fscale = max(1e-3, abs(du).max())
        assert abs(du[0] - du[2]) < 1e-5 * fscale, (name, r0)
        # second derivative: one-sided quadratic extrapolations of u' to r0
        # (r0 itself belongs to the region on its right: intervals are [r-, r+))
        hh = 1e-4
        _, dl = O.u_tilde(row, [r0 - 3 * hh, r0 - 2 * hh, r0 - hh])
        _, dr = O.u_tilde(row, [r0, r0 + hh, r0 + 2 * hh])
        left = (5 * dl[2] - 8 * dl[1] + 3 * dl[0]) / (2 * hh)
        right = (-3 * dr[0] + 4 * dr[1] - dr[2]) / (2 * hh)
        curv = max(1e-3, abs(left), abs(right))
        assert abs(left - right) < 1e-5 * curv, (name, r0, left, right)


@pytest.mark.parametrize("name,row", list(_rows()))
def test_zero_at_and_beyond_rc_plus(name, row):
    d = P.row_dict(row)
    u, du = O.u_tilde(row, [d["rcp"], d["rcp"] + 0.5, 50.0])
    assert np.all(u == 0.0) and np.all(du == 0.0)


@pytest.mark.parametrize("name,row", list(_rows()))
def test_derivative_matches_energy(name, row):
    d = P.row_dict(row)
    rng = np.random.default_rng(3)
    r = rng.uniform(3.3, d["rcp"] - 1e-3, 400)
    h = 1e-6
    up, _ = O.u_tilde(row, r + h)
    um, _ = O.u_tilde(row, r - h)
    _, du = O.u_tilde(row, r)
    bounds = np.array([d["rsm"], d["rsp"], d["rcm"], d["rcp"]])
    far = np.min(np.abs(r[:, None] - bounds[None, :]), axis=1) > 1e-4
    fd = (up - um) / (2 * h)
    np.testing.assert_allclose(du[far], fd[far], rtol=2e-6, atol=1e-9)


def test_region1_is_textbook_lj_force_and_shifted_energy():
    row = P.pair_row(0.0914, 3.95, 1.3914, 3.8099, RADII)
    d = P.row_dict(row)
    r = np.linspace(3.0, 5.999, 200)
    u, du = O.u_tilde(row, r)
    np.testing.assert_allclose(-du, _lj_force(r, d["eps_fg"], d["sig_fg"]), rtol=1e-12)
    lj_u = 4 * d["eps_fg"] * ((d["sig_fg"] / r) ** 12 - (d["sig_fg"] / r) ** 6)
    np.testing.assert_allclose(u - lj_u, -d["Gam_sm"], rtol=1e-9, atol=1e-12)


def test_region3_is_textbook_lj_force_with_cg_parameters():
    row = P.pair_row(0.0914, 3.95, 1.3914, 3.8099, RADII)
    d = P.row_dict(row)
    r = np.linspace(7.0, 12.999, 200)
    _, du = O.u_tilde(row, r)
    np.testing.assert_allclose(-du, _lj_force(r, d["eps_cg"], d["sig_cg"]), rtol=1e-12)


def test_ordinary_pairs_vanish_beyond_rs_plus():
    row = P.pair_row(0.195, 3.75, 0.0, 3.9, RADII)
    u, du = O.u_tilde(row, np.linspace(7.0, 20.0, 100))
    assert np.all(u == 0.0) and np.all(du == 0.0)


def test_fg_reference_limit():
    # eps^CG = 0, r_s- = 13, r_s+ = r_c- = r_c+ = 14: the FG reference system
    row = P.pair_row(0.195, 3.75, 0.0, 0.0, (13.0, 14.0, 14.0, 14.0))
    r = np.linspace(3.0, 12.99, 300)
    _, du = O.u_tilde(row, r)
    np.testing.assert_allclose(-du, _lj_force(r, 0.195, 3.75), rtol=1e-12)
    u, _ = O.u_tilde(row, np.array([14.0, 15.0]))
    assert np.all(u == 0.0)


def test_all_hybrid_n1_limit_is_lj_outside_zones():
    # a group of one site: Eq. 13 returns the FG parameters, u^CG = u^FG
    E, S = P.mix_fg([0.3], [3.9])
    ecg, scg = P.cg_pair_eq13([1], [1], E, S)
    assert ecg == pytest.approx(0.3, rel=1e-14) and scg == pytest.approx(3.9, rel=1e-14)
    row = P.pair_row(0.3, 3.9, ecg, scg, RADII)
    r = np.concatenate([np.linspace(3.0, 5.99, 50), np.linspace(7.0, 12.99, 50)])
    _, du = O.u_tilde(row, r)
    np.testing.assert_allclose(-du, _lj_force(r, 0.3, 3.9), rtol=1e-12)
    # and the energy is one continuous shifted LJ: u - u^LJ equal in regions 1 and 3
    u, _ = O.u_tilde(row, np.array([5.0, 10.0]))
    lj = 4 * 0.3 * ((3.9 / np.array([5.0, 10.0])) ** 12 - (3.9 / np.array([5.0, 10.0])) ** 6)
    d = P.row_dict(row)
    assert (u - lj)[1] == pytest.approx(-d["Gam_cm"], rel=1e-9)
