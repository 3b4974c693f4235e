"""Pins of the oracle's bonded terms, random numbers and integrator.

* Bonded: F = -grad E by finite differences for bonds, angles and OPLS
  dihedrals; zero net force and torque; closed-form energies of chosen
  geometries (stretched bond, right angle, cis and trans dihedrals).
* splitmix64: the first outputs of the published generator for seed 0.
* CSVR: tau -> infinity leaves velocities unchanged; tau -> 0 draws the
  kinetic energy from the canonical distribution (mean K_t, variance
  2 K_t^2 / N_f), which also pins the Box-Muller normal and the
  Marsaglia-Tsang chi-squared draws it is made of.
* Velocity Verlet: bounded NVE energy error that shrinks ~4x when dt halves
  (second order), and no drift of the total momentum; 1000 steps of 1 fs on
  the propane-like configuration with neither energy drift nor momentum.
"""
import math

import numpy as np
import pytest

from oracle import core as O
from paper_2104_10231_gb300 import systems as S


def _chain(n=8, seed=3):
    rng = np.random.default_rng(seed)
    pos = np.zeros((n, 3))
    for i in range(1, n):
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        pos[i] = pos[i - 1] + rng.uniform(1.4, 1.7) * u
    pos += 20.0
    topo = S._empty_topo()
    topo["bonds"] = np.array([[i, i + 1] for i in range(n - 1)], np.int32)
    topo["bond_type"] = np.zeros(n - 1, np.int32)
    topo["bond_k"] = np.array([450.0])
    topo["bond_r0"] = np.array([1.54])
    topo["angles"] = np.array([[i, i + 1, i + 2] for i in range(n - 2)], np.int32)
    topo["angle_type"] = np.zeros(n - 2, np.int32)
    topo["angle_k"] = np.array([62.0])
    topo["angle_theta0"] = np.array([math.radians(114.0)])
    topo["dihedrals"] = np.array([[i, i + 1, i + 2, i + 3] for i in range(n - 3)], np.int32)
    topo["dihedral_type"] = np.zeros(n - 3, np.int32)
    topo["dihedral_k"] = np.array([[1.3, -0.4, 2.2, 0.7]])
    return pos, np.full(3, 40.0), topo


def _etot(pos, box, topo):
    return O.bonded(pos, box, topo)[1].sum()


def test_bonded_forces_are_minus_gradient():
    pos, box, topo = _chain()
    f, _ = O.bonded(pos, box, topo)
    h = 1e-6
    for i in range(len(pos)):
        for a in range(3):
            pp = pos.copy()
            pp[i, a] += h
            ep = _etot(pp, box, topo)
            pp[i, a] -= 2 * h
            em = _etot(pp, box, topo)
            assert f[i, a] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-6)


def test_bonded_net_force_and_torque_vanish():
    pos, box, topo = _chain(seed=7)
    f, _ = O.bonded(pos, box, topo)
    assert np.abs(f.sum(0)).max() < 1e-10
    c = pos.mean(0)
    torque = np.cross(pos - c, f).sum(0)
    assert np.abs(torque).max() < 1e-9


def test_bonded_closed_form_energies():
    box = np.full(3, 40.0)
    topo = S._empty_topo()
    topo["bonds"] = np.array([[0, 1]], np.int32)
    topo["bond_type"] = np.zeros(1, np.int32)
    topo["bond_k"] = np.array([450.0])
    topo["bond_r0"] = np.array([1.54])
    pos = np.array([[10.0, 10, 10], [11.64, 10, 10]])
    assert O.bonded(pos, box, topo)[1][0] == pytest.approx(450.0 * 0.1 ** 2, rel=1e-12)

    topo = S._empty_topo()
    topo["angles"] = np.array([[0, 1, 2]], np.int32)
    topo["angle_type"] = np.zeros(1, np.int32)
    topo["angle_k"] = np.array([62.0])
    topo["angle_theta0"] = np.array([math.radians(114.0)])
    pos = np.array([[11.5, 10, 10], [10.0, 10, 10], [10.0, 11.5, 10]])
    assert O.bonded(pos, box, topo)[1][1] == pytest.approx(62.0 * (math.pi / 2 - math.radians(114)) ** 2, rel=1e-12)

    topo = S._empty_topo()
    topo["dihedrals"] = np.array([[0, 1, 2, 3]], np.int32)
    topo["dihedral_type"] = np.zeros(1, np.int32)
    K = np.array([1.3, 0.4, 2.2, 0.7])
    topo["dihedral_k"] = K[None]
    cis = np.array([[10.0, 11.0, 10], [10.0, 10.0, 10], [11.5, 10.0, 10], [11.5, 11.0, 10]])
    trans = np.array([[10.0, 11.0, 10], [10.0, 10.0, 10], [11.5, 10.0, 10], [11.5, 9.0, 10]])
    # phi = 0: 1/2 [2 K1 + 0 + 2 K3 + 0]; phi = 180 deg: 1/2 [0 + 0 + 0 + 0]
    assert O.bonded(cis, box, topo)[1][2] == pytest.approx(K[0] + K[2], rel=1e-12)
    assert O.bonded(trans, box, topo)[1][2] == pytest.approx(0.0, abs=1e-12)
    gauche = trans.copy()
    gauche[3] = [11.5, 10.0 - math.cos(math.radians(60)) * -1.0, 10 + math.sin(math.radians(60))]
    # phi = +-60 deg
    phi = math.radians(60)
    e_expected = 0.5 * (K[0] * (1 + math.cos(phi)) + K[1] * (1 - math.cos(2 * phi))
                        + K[2] * (1 + math.cos(3 * phi)) + K[3] * (1 - math.cos(4 * phi)))
    assert O.bonded(gauche, box, topo)[1][2] == pytest.approx(e_expected, rel=1e-10)


def test_splitmix64_published_outputs():
    # splitmix64 (Steele, Lea & Flood 2014) seeded with 0: first four outputs
    expected = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [O.splitmix64(0, c) for c in range(4)] == expected


def test_csvr_limits():
    n_f = 3 * 648 - 3
    kt = 0.5 * n_f * S.KB_KCAL * 230.0
    # tau -> infinity: c = 1, nothing changes
    for step in range(5):
        assert O.csvr_alpha(0.8 * kt, kt, n_f, 1.0, 1e300, 7, step) == pytest.approx(1.0, abs=1e-12)
    # tau -> 0: K_new = K_t (R1^2 + S)/N_f, canonical: mean K_t, var 2 K_t^2 / N_f
    k0 = 1.3 * kt
    knew = np.array([k0 * O.csvr_alpha(k0, kt, n_f, 1.0, 1e-300, 11, s) ** 2 for s in range(4000)])
    assert knew.mean() == pytest.approx(kt, rel=4 * math.sqrt(2.0 / n_f / 4000))
    assert knew.var() == pytest.approx(2 * kt ** 2 / n_f, rel=0.1)


def _propane_small():
    return S.propane(n_mol=216)


def test_nve_energy_error_is_second_order():
    s = _propane_small()
    table = O.table_for(s)
    masses = s.masses

    def run(dt, n):
        p, v, th = O.md(s.pos, s.vel, s.box, masses, s.types, table, s.n_types, s.excl, s.topo,
                        n, dt, n_threads=0)
        etot = th.sum(1)
        return p, v, etot

    _, v1, e1 = run(1.0, 40)
    _, v2, e2 = run(0.5, 80)
    dev1 = np.abs(e1 - e1[0]).max()
    dev2 = np.abs(e2 - e2[0]).max()
    # the raw lattice start relaxes fast (E_pair -188 -> -467 kcal/mol in 40 fs)
    assert dev1 < 2.0  # kcal/mol, 648 atoms, KE ~ 600 kcal/mol
    ratio = dev1 / dev2
    assert 2.5 < ratio < 6.0, ratio
    p = (v1 * masses[:, None]).sum(0)
    assert np.abs(p).max() < 1e-9


def test_nve_1000_steps_on_the_propane_configuration():
    """The propane-like configuration (216 molecules, FP64) for 1000 NVE steps
    of 1 fs: after the lattice start has relaxed (100 fs), the total energy
    neither drifts nor fluctuates by more than 2e-3 of the mean kinetic
    energy, and the total momentum stays zero."""
    s = _propane_small()
    table = O.table_for(s)
    p, v, th = O.md(s.pos, s.vel, s.box, s.masses, s.types, table, s.n_types, s.excl, s.topo, 1000, 1.0,
                    n_threads=0)
    etot = th.sum(1)
    ke = th[:, 2].mean()
    tail = etot[100:]
    drift = abs(tail[-1] - tail[0]) / ke
    fluct = tail.std() / ke
    print(f"oracle NVE 1000 x 1 fs: drift {drift:.2e}, fluctuation {fluct:.2e} of <KE>")
    assert drift < 2e-3 and fluct < 2e-3, (drift, fluct)
    mom = (v * s.masses[:, None]).sum(0)
    assert np.abs(mom).max() < 1e-8
