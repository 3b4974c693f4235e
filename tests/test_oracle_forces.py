"""Pins of the oracle's all-pairs RelRes sum (oracle_pair_forces).

* F = -grad E by central finite differences (catches a sign or a factor in
  the force, or a force that does not belong to the energy).
* Newton's third law: sum_i F_i = 0.
* Virial: diagonal W_aa = -dE/d(strain_aa) under an affine box scaling
  (independent of the pair loop's virial code), off-diagonal from a brute
  force pair enumeration with minimum image.
* A single pair across the periodic boundary reproduces Eq. 20 at the
  minimum-image distance; excluded pairs contribute nothing; atom order does
  not matter.
* A planted mistake (the printed gamma_{4+} sign of Eq. 18) breaks the C2
  continuity check, so that check can see such an error.
"""
import itertools

import numpy as np
import pytest

from oracle import core as O
from oracle import params as P

RADII = (6.0, 7.0, 13.0, 14.0)


def _random_system(n=90, box=30.0, seed=5):
    rng = np.random.default_rng(seed)
    pos = []
    while len(pos) < n:
        p = rng.random(3) * box
        ok = True
        for q in pos:
            d = p - q
            d -= box * np.round(d / box)
            if d @ d < 3.2 ** 2:
                ok = False
                break
        if ok:
            pos.append(p)
    pos = np.array(pos)
    types = rng.integers(0, 3, n).astype(np.int32)
    eps = [0.195, 0.0914, 0.3]
    sig = [3.75, 3.95, 3.6]
    hyb = [0, 1, 1]
    comp = [[0, 0, 0], [2, 1, 0], [1, 0, 2]]
    tab = P.pair_table(eps, sig, hyb, RADII, mixing=P.MIX_LB, group_comp=comp)
    # a few exclusions: pairs (0,1), (2,3), (2,4)
    excl_pairs = {(0, 1), (2, 3), (2, 4)}
    lists = [[] for _ in range(n)]
    for a, b in excl_pairs:
        lists[a].append(b)
        lists[b].append(a)
    off = np.zeros(n + 1, np.int32)
    idx = []
    for i in range(n):
        idx += sorted(lists[i])
        off[i + 1] = len(idx)
    return pos, np.full(3, box), types, tab, (off, np.array(idx, np.int32))


def test_forces_are_minus_gradient():
    pos, box, types, tab, excl = _random_system()
    f, e, _ = O.pair_forces(pos, box, types, tab, 3, excl)
    h = 1e-5
    for i in (0, 5, 17, 42, 89):
        for a in range(3):
            pp = pos.copy()
            pp[i, a] += h
            ep = O.pair_forces(pp, box, types, tab, 3, excl)[1]
            pp[i, a] -= 2 * h
            em = O.pair_forces(pp, box, types, tab, 3, excl)[1]
            assert f[i, a] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-8)


def test_net_force_vanishes():
    pos, box, types, tab, excl = _random_system(seed=9)
    f, _, _ = O.pair_forces(pos, box, types, tab, 3, excl)
    assert np.abs(f.sum(0)).max() < 1e-11 * np.abs(f).max()


def test_diagonal_virial_is_strain_derivative():
    pos, box, types, tab, excl = _random_system(seed=11)
    _, _, w = O.pair_forces(pos, box, types, tab, 3, excl)
    h = 1e-6
    for a in range(3):
        s = np.ones(3)
        s[a] = 1 + h
        ep = O.pair_forces(pos * s, box * s, types, tab, 3, excl)[1]
        s[a] = 1 - h
        em = O.pair_forces(pos * s, box * s, types, tab, 3, excl)[1]
        assert w[a] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-8)


def test_virial_and_energy_by_pair_enumeration():
    pos, box, types, tab, excl = _random_system(n=40, seed=13)
    f, e, w = O.pair_forces(pos, box, types, tab, 3, excl)
    off, idx = excl
    e_ref = 0.0
    w_ref = np.zeros(6)
    for i, j in itertools.combinations(range(len(pos)), 2):
        if j in idx[off[i]:off[i + 1]]:
            continue
        d = pos[i] - pos[j]
        d -= box * np.round(d / box)
        r = np.sqrt(d @ d)
        u, du = O.u_tilde(tab[types[i] * 3 + types[j]], r)
        e_ref += u[0]
        fij = -du[0] * d / r
        w_ref += [d[0] * fij[0], d[1] * fij[1], d[2] * fij[2], d[0] * fij[1], d[0] * fij[2], d[1] * fij[2]]
    assert e == pytest.approx(e_ref, rel=1e-12)
    np.testing.assert_allclose(w, w_ref, rtol=1e-10, atol=1e-10)


def test_single_pair_across_boundary():
    tab = P.pair_table([0.3], [3.9], [1], RADII, group_comp=[[1]])
    box = np.full(3, 40.0)
    for sep in (4.0, 6.5, 9.0, 13.5, 14.2):
        pos = np.array([[0.5, 20.0, 20.0], [0.5 - sep, 20.0, 20.0]])  # second atom wraps
        pos %= box
        f, e, _ = O.pair_forces(pos, box, np.zeros(2, np.int32), tab, 1)
        u, du = O.u_tilde(tab[0], sep)
        assert e == pytest.approx(u[0], rel=1e-12, abs=1e-15)
        assert f[0, 0] == pytest.approx(-du[0], rel=1e-10, abs=1e-15)


def test_row_subset_equals_full_sum():
    pos, box, types, tab, excl = _random_system(n=70, seed=23)
    f, e, _ = O.pair_forces(pos, box, types, tab, 3, excl)
    rows = np.array([0, 3, 17, 69, 42])
    fr, er = O.pair_forces_rows(pos, box, types, tab, 3, rows, excl)
    np.testing.assert_allclose(fr, f[rows], rtol=1e-13, atol=1e-13)
    _, eall = O.pair_forces_rows(pos, box, types, tab, 3, np.arange(70), excl)
    assert eall.sum() == pytest.approx(e, rel=1e-12)


def test_exclusion_removes_pair():
    tab = P.pair_table([0.3], [3.9], [1], RADII, group_comp=[[1]])
    pos = np.array([[5.0, 5.0, 5.0], [9.0, 5.0, 5.0]])
    box = np.full(3, 40.0)
    excl = (np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32))
    f, e, w = O.pair_forces(pos, box, np.zeros(2, np.int32), tab, 1, excl)
    assert e == 0.0 and np.all(f == 0.0) and np.all(w == 0.0)


def test_permutation_invariance():
    pos, box, types, tab, excl = _random_system(n=50, seed=17)
    f, e, w = O.pair_forces(pos, box, types, tab, 3, None)
    perm = np.random.default_rng(0).permutation(len(pos))
    f2, e2, w2 = O.pair_forces(pos[perm], box, types[perm], tab, 3, None)
    assert e2 == pytest.approx(e, rel=1e-12)
    np.testing.assert_allclose(f2, f[perm], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(w2, w, rtol=1e-10, atol=1e-10)


def test_planted_gamma4_sign_error_is_caught_by_c2_check():
    row = P.pair_row(0.0914, 3.95, 1.3914, 3.8099, RADII)
    d = P.row_dict(row)
    bad = row.copy()
    u, du, d2u = P.lj(d["rsp"], d["eps_cg"], d["sig_cg"])
    k = P.ROW_FIELDS.index("g_cg_p4")
    bad[k] = -du / 2.0 - d2u / 4.0  # printed sign, dr = 1
    r0, hh = d["rsp"], 1e-4

    def jump(rw):
        _, dl = O.u_tilde(rw, [r0 - 3 * hh, r0 - 2 * hh, r0 - hh])
        _, dr = O.u_tilde(rw, [r0, r0 + hh, r0 + 2 * hh])
        left = (5 * dl[2] - 8 * dl[1] + 3 * dl[0]) / (2 * hh)
        right = (-3 * dr[0] + 4 * dr[1] - dr[2]) / (2 * hh)
        return abs(left - right) / max(abs(left), abs(right))

    assert jump(row) < 1e-5
    assert jump(bad) > 1e-2
