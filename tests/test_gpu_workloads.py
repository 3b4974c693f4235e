"""GPU parity at the workload sizes and on the degenerate cases of the method.

* The 20 000-atom neopentane-like liquid (FP32) and the 20 000-atom block
  copolymer melt (FP32, dihedrals, intrachain CG pairs) against the full FP64
  oracle.
* The 1 000 000-atom neopentane-like liquid in the configuration the benchmark
  times (FP32, CSVR at 260 K, dt = 2 fs, lists rebuilt on the device): forces
  of sampled atoms against oracle rows (each row is the full O(N) sum of that
  atom), bonded forces against the oracle, and energy / virial against the
  FP64 mode of the library (which the small-size tests pin to the oracle).
* Degenerate cases: zero-width switching shells (r_- = r_+ removes a shell),
  every atom a hybrid of its own group (n = 1, so u^CG = u^FG by Eq. 13), and
  a single pair swept through all five regions of Eq. 20.
"""
import math

import numpy as np
import pytest

from oracle import core as O
from paper_2104_10231_gb300 import relres as R
from paper_2104_10231_gb300 import systems as S

pytestmark = pytest.mark.gpu

F_TOL = 1e-5
E_TOL = 1e-7


@pytest.fixture(scope="module")
def torch():
    import torch as T

    assert T.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2104_10231_gb300.build import build_library

    build_library()
    R.load()
    return T


def _dev(torch, a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _compute(torch, system, precision, pos=None, ctx=None):
    own = ctx is None
    if own:
        ctx = R.Context(R.params_for(system, precision), R.topology_for(system))
    p = _dev(torch, system.pos if pos is None else pos)
    if own:
        ctx.build_neighbors(p, system.box)
    f = torch.empty_like(p)
    e = torch.zeros(4, dtype=torch.float64, device="cuda")
    w = torch.zeros(6, dtype=torch.float64, device="cuda")
    ctx.compute(p, f, e, w)
    torch.cuda.synchronize()
    out = f.cpu().numpy(), e.cpu().numpy(), w.cpu().numpy()
    if own:
        ctx.close()
    return out


def _oracle(system, pos=None):
    pos = system.pos if pos is None else pos
    tab = O.table_for(system)
    f, e, w = O.pair_forces(pos, system.box, system.types, tab, system.n_types, system.excl)
    fb, eb = O.bonded(pos, system.box, system.topo)
    return f + fb, e, float(eb.sum()), w


def _ferr(f, ref):
    rms = math.sqrt((ref * ref).sum(1).mean())
    return float(np.abs(f - ref).max() / rms)


def _check_full(torch, system, precision, f_tol, e_tol):
    f, e, w = _compute(torch, system, precision)
    fr, er, ebr, wr = _oracle(system)
    ferr = _ferr(f, fr)
    eerr = abs(e[0] + e[1] - er) / abs(er)
    berr = abs(e[2] - ebr) / max(1.0, abs(ebr))
    werr = float(np.abs(w - wr).max() / np.abs(wr[:3]).max())
    print(f"{system.name} N={system.n_atoms}: force {ferr:.2e} energy {eerr:.2e} bonded {berr:.2e} "
          f"virial {werr:.2e}")
    assert ferr <= f_tol, ferr
    assert eerr <= e_tol, eerr
    assert berr <= e_tol, berr
    assert werr <= 10 * f_tol, werr


def test_fp32_neopentane_20000_atoms(torch):
    _check_full(torch, S.neopentane(n_mol=4000), R.RELRES_PREC_FP32, F_TOL, E_TOL)


def test_fp32_block_copolymer_20000_atoms(torch):
    s = S.block_copolymer()
    assert s.n_atoms == 20000 and len(s.topo["dihedrals"]) > 0
    _check_full(torch, s, R.RELRES_PREC_FP32, F_TOL, E_TOL)


def test_fp64_block_copolymer_2000_atoms(torch):
    _check_full(torch, S.block_copolymer(n_chain=20), R.RELRES_PREC_FP64, 1e-10, 1e-10)


def test_fp32_neopentane_1m_atoms_bench_configuration(torch):
    s = S.neopentane(n_mol=200_000)
    assert s.n_atoms == 1_000_000
    ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
    p = _dev(torch, s.pos)
    v = _dev(torch, s.vel)
    ctx.build_neighbors(p, s.box)
    th = torch.zeros((3, R.RELRES_THERMO_COLS), dtype=torch.float64, device="cuda")
    ctx.step(60, 2.0, p, v, t_target=260.0, tau_fs=100.0, seed=5, thermo_every=20, d_thermo=th)
    torch.cuda.synchronize()
    st = ctx.stats()
    assert st["n_builds"] >= 2  # the first build plus at least one device-side rebuild
    pos = p.cpu().numpy()
    f, e, w = _compute(torch, s, R.RELRES_PREC_FP32, pos=pos, ctx=ctx)
    ctx.close()
    assert np.all(np.isfinite(f))

    # sampled rows against the oracle: pair part (full rows) + bonded part
    rng = np.random.default_rng(17)
    rows = np.sort(rng.choice(s.n_atoms, size=256, replace=False)).astype(np.int32)
    tab = O.table_for(s)
    fp, _ = O.pair_forces_rows(pos, s.box, s.types, tab, s.n_types, rows, s.excl)
    fb, _ = O.bonded(pos, s.box, s.topo)
    fr = fp + fb[rows]
    rms = math.sqrt((fr * fr).sum(1).mean())
    err = float(np.abs(f[rows] - fr).max() / rms)
    print(f"1M atoms, 256 sampled rows: force {err:.2e}")
    assert err <= F_TOL, err

    # energies and virial: FP32 mode against the FP64 mode at the same positions
    f64, e64, w64 = _compute(torch, s, R.RELRES_PREC_FP64, pos=pos)
    eerr = abs((e[0] + e[1]) - (e64[0] + e64[1])) / abs(e64[0] + e64[1])
    berr = abs(e[2] - e64[2]) / abs(e64[2])
    werr = float(np.abs(w - w64).max() / np.abs(w64[:3]).max())
    ferr64 = _ferr(f, f64)
    print(f"1M atoms vs FP64 mode: energy {eerr:.2e} bonded {berr:.2e} virial {werr:.2e} force {ferr64:.2e}")
    assert eerr <= E_TOL and berr <= E_TOL
    assert werr <= 10 * F_TOL and ferr64 <= F_TOL
    # the thermo row of the last step holds the same energies
    row = th[-1].cpu().numpy()
    assert row[0] + row[1] == pytest.approx(e[0] + e[1], rel=1e-9)
    assert row[2] == pytest.approx(e[2], rel=1e-6)


def test_fp32_neopentane_200k_atoms_against_the_full_oracle(torch):
    """200 000 atoms (40 000 molecules, L = 202 A) in the benchmark's FP32
    configuration after 60 MD steps (device-side rebuilds, pruning passes,
    Morton-ordered cells, several waves of pair blocks): forces, pair energy
    E_fg + E_cg and virial against the oracle's full all-pairs FP64 sum of
    Eq. 20 at the same positions."""
    s = S.neopentane(n_mol=40_000, seed=2105)
    assert s.n_atoms == 200_000
    ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
    p = _dev(torch, s.pos)
    v = _dev(torch, s.vel)
    ctx.build_neighbors(p, s.box)
    ctx.step(60, 2.0, p, v, t_target=260.0, tau_fs=100.0, seed=6)
    torch.cuda.synchronize()
    st = ctx.stats()
    assert st["n_builds"] >= 2 and st["n_prunes"] > st["n_builds"]
    pos = p.cpu().numpy()
    f, e, w = _compute(torch, s, R.RELRES_PREC_FP32, pos=pos, ctx=ctx)
    ctx.close()
    fr, er, ebr, wr = _oracle(s, pos=pos)
    ferr = _ferr(f, fr)
    eerr = abs(e[0] + e[1] - er) / abs(er)
    berr = abs(e[2] - ebr) / max(1.0, abs(ebr))
    werr = float(np.abs(w - wr).max() / np.abs(wr[:3]).max())
    print(f"200k atoms vs full oracle: force {ferr:.2e} energy {eerr:.2e} bonded {berr:.2e} virial {werr:.2e}")
    assert ferr <= F_TOL, ferr
    assert eerr <= E_TOL, eerr
    assert berr <= E_TOL, berr
    assert werr <= 10 * F_TOL, werr


def test_zero_width_shells(torch):
    # r_s- = r_s+ and r_c- = r_c+: no smoothing shells, hard switches of Eq. 20
    s = S.neopentane(n_mol=400, seed=9).subset_copy(radii=(6.5, 6.5, 13.5, 13.5))
    _check_full(torch, s, R.RELRES_PREC_FP64, 1e-10, 1e-10)
    _check_full(torch, s, R.RELRES_PREC_FP32, F_TOL, E_TOL)


def test_every_atom_its_own_hybrid(torch):
    # n = 1: each atom is the CG site of its own group, so Eq. 13 gives
    # u^CG = u^FG and every atom is in both lists
    base = S.neopentane(n_mol=400, seed=4)
    s = base.subset_copy(name="neopentane_all_hybrid", is_hybrid=np.ones(2, np.int32),
                         group_comp=np.eye(2, dtype=np.int32))
    assert s.n_hybrid == s.n_atoms
    _check_full(torch, s, R.RELRES_PREC_FP64, 1e-10, 1e-10)
    _check_full(torch, s, R.RELRES_PREC_FP32, F_TOL, E_TOL)


def _pair_system(r):
    """Two hybrid atoms of one type (a one-atom group) at distance r."""
    pos = np.array([[20.0, 20.0, 20.0], [20.0 + r, 20.0, 20.0]])
    eo = np.zeros(3, np.int32)
    return S.System("pair", pos, np.zeros((2, 3)), np.zeros(2, np.int32), np.array([0, 1], np.int32),
                    np.full(3, 45.0), ["X"], np.array([15.035]), np.array([0.195]), np.array([3.75]),
                    np.array([1], np.int32), np.array([[1]], np.int32), (6.0, 7.0, 13.0, 14.0), "lb",
                    2.0, S._empty_topo(), eo, np.zeros(0, np.int32), 0.0, 1.0, 0)


def test_empty_and_one_atom_systems(torch):
    # no atoms: refused; one atom: no pair, zero force, energy and virial; an
    # NVE step moves it in free flight (x + v dt, v unchanged: no force), and
    # the thermostat refuses a system with fewer than two atoms
    import dataclasses

    two = _pair_system(5.0)
    one = dataclasses.replace(two, pos=two.pos[:1].copy(), vel=np.array([[0.01, -0.02, 0.005]]),
                              types=two.types[:1].copy(), mol=two.mol[:1].copy(),
                              excl_off=np.zeros(2, np.int32), excl_idx=np.zeros(0, np.int32))
    for prec in (R.RELRES_PREC_FP64, R.RELRES_PREC_FP32):
        ctx = R.Context(R.params_for(one, prec))
        with pytest.raises(R.RelresError) as ei:
            ctx.set_topology(R.make_topology(np.zeros(0, np.int32), one.mass_by_type))
        assert ei.value.status == 1  # RELRES_ERR_ARG
        ctx.set_topology(R.topology_for(one))
        p = _dev(torch, one.pos)
        v = _dev(torch, one.vel)
        ctx.build_neighbors(p, one.box)
        f = torch.empty_like(p)
        e = torch.zeros(4, dtype=torch.float64, device="cuda")
        w = torch.zeros(6, dtype=torch.float64, device="cuda")
        ctx.compute(p, f, e, w)
        assert float(f.abs().max()) == 0.0 and float(e.abs().max()) == 0.0 and float(w.abs().max()) == 0.0
        ctx.step(10, 1.0, p, v)
        x = p.cpu().numpy()
        assert np.allclose(x, one.pos + 10.0 * one.vel, rtol=0, atol=1e-9), (x, one.pos + 10.0 * one.vel)
        # unchanged up to the float-float velocity state of the FP32 path
        assert np.allclose(v.cpu().numpy(), one.vel, rtol=1e-13, atol=0)
        with pytest.raises(R.RelresError):
            ctx.step(1, 1.0, p, v, t_target=300.0)
        ctx.close()


def _eight_types(seed=31):
    """The neopentane-like liquid relabelled with the largest number of types,
    RELRES_MAX_TYPES = 8: four ordinary types for the CH3 sites and four
    hybrid types for the central sites, all with different eps and sigma, and
    a group composition per hybrid type (its own site plus four ordinary sites
    in a type-dependent mix) from which Eq. 13 gives all 16 CG pairs."""
    import dataclasses

    base = S.neopentane(n_mol=1000, seed=seed)
    rng = np.random.default_rng(seed)
    mol = base.mol
    types = np.where(base.types == 0, 4 + mol % 4, (mol + np.arange(base.n_atoms)) % 4).astype(np.int32)
    comp = np.zeros((8, 8), np.int32)
    for h in range(4):
        comp[4 + h, 4 + h] = 1
        comp[4 + h, h] += 2
        comp[4 + h, (h + 1) % 4] += 1
        comp[4 + h, (h + 2) % 4] += 1
    return dataclasses.replace(
        base, name="eight_types", types=types, type_names=[f"T{k}" for k in range(8)],
        mass_by_type=np.concatenate([np.full(4, 15.035), np.full(4, 12.011)]),
        eps_fg=rng.uniform(0.08, 0.2, 8), sig_fg=rng.uniform(3.6, 4.0, 8),
        is_hybrid=np.array([0, 0, 0, 0, 1, 1, 1, 1], np.int32), group_comp=comp)


@pytest.mark.parametrize("precision,f_tol,e_tol", [(R.RELRES_PREC_FP64, 1e-10, 1e-10),
                                                   (R.RELRES_PREC_FP32, F_TOL, E_TOL)])
def test_largest_number_of_types(torch, precision, f_tol, e_tol):
    s = _eight_types()
    assert s.n_types == R.RELRES_MAX_TYPES and len(np.unique(s.types)) == 8
    _check_full(torch, s, precision, f_tol, e_tol)


def test_single_pair_through_all_regions(torch):
    # below r_s-, in the FG shell, CG LJ, CG shell, beyond r_c+
    for r in (3.9, 5.5, 6.4, 6.999, 7.0, 9.0, 12.9, 13.5, 13.999, 14.5):
        s = _pair_system(r)
        for prec, tol in ((R.RELRES_PREC_FP64, 1e-10), (R.RELRES_PREC_FP32, 2e-6)):
            f, e, w = _compute(torch, s, prec)
            fr, er, _, wr = _oracle(s)
            scale = max(1e-3, float(np.abs(fr).max()))
            assert np.abs(f - fr).max() <= tol * scale, (r, prec, f, fr)
            assert abs(e[0] + e[1] - er) <= 1e-9 * max(1.0, abs(er)), (r, prec, e, er)
            # Newton's third law holds exactly in both modes
            assert np.abs(f[0] + f[1]).max() <= 1e-12 * scale


def _geometric_rs_radii(rs_by_type, d_s=1.0, r_c=13.5, d_c=1.0):
    """Per-type-pair radii with r_s mixed geometrically across groups
    (sqrt(r_s,a r_s,b)), shells of width d_s around r_s and d_c around r_c."""
    nt = len(rs_by_type)
    rad = np.zeros((nt, nt, 4))
    for a in range(nt):
        for b in range(nt):
            rs = math.sqrt(rs_by_type[a] * rs_by_type[b])
            rad[a, b] = (rs - d_s / 2, rs + d_s / 2, r_c - d_c / 2, r_c + d_c / 2)
    return rad


@pytest.mark.parametrize("precision,f_tol,e_tol", [(R.RELRES_PREC_FP64, 1e-10, 1e-10),
                                                   (R.RELRES_PREC_FP32, F_TOL, E_TOL)])
def test_block_copolymer_with_per_pair_radii(torch, precision, f_tol, e_tol):
    # A groups r_s = 6 A, B groups r_s = 7 A, cross pairs the geometric mean
    from oracle import params as P

    s = S.block_copolymer(n_chain=40)
    rad = _geometric_rs_radii([6.0, 7.0, 6.0, 7.0])
    mixing = R.RELRES_MIX_LB
    params = R.make_params(s.eps_fg, s.sig_fg, s.is_hybrid, s.radii, s.skin, mixing=mixing,
                           group_comp=s.group_comp, precision=precision, radii_pair=rad)
    ctx = R.Context(params, R.topology_for(s))
    p = _dev(torch, s.pos)
    ctx.build_neighbors(p, s.box)
    f = torch.empty_like(p)
    e = torch.zeros(4, dtype=torch.float64, device="cuda")
    w = torch.zeros(6, dtype=torch.float64, device="cuda")
    ctx.compute(p, f, e, w)
    torch.cuda.synchronize()
    st = ctx.stats()
    ctx.close()
    tab = P.pair_table(s.eps_fg, s.sig_fg, s.is_hybrid, s.radii, mixing=s.mixing, group_comp=s.group_comp,
                       radii_pair=rad)
    fr, er, wr = O.pair_forces(s.pos, s.box, s.types, tab, s.n_types, s.excl)
    fb, eb = O.bonded(s.pos, s.box, s.topo)
    fr = fr + fb
    ferr = _ferr(f.cpu().numpy(), fr)
    eerr = abs(float(e[0] + e[1]) - er) / abs(er)
    print(f"copolymer per-pair radii prec={precision}: force {ferr:.2e} energy {eerr:.2e} "
          f"list radius FG {st['list_radius_fg']:.2f}")
    assert st["list_radius_fg"] == pytest.approx(7.5 + s.skin)
    assert ferr <= f_tol and eerr <= e_tol


@pytest.mark.parametrize("precision,f_tol,e_tol", [(R.RELRES_PREC_FP64, 1e-10, 1e-10),
                                                   (R.RELRES_PREC_FP32, F_TOL, E_TOL)])
def test_chains_longer_than_a_force_segment(torch, precision, f_tol, e_tol):
    # 300-bead chains: no run of whole molecules fits the fused bonded + force-sum
    # kernel's 256-atom segment, so the bonded kernel + per-atom sum path runs
    s = S.block_copolymer(n_chain=12, n_bead=300, block=150, density=0.5)
    assert s.n_atoms == 3600
    _check_full(torch, s, precision, f_tol, e_tol)


def _wrapped(a, b, L):
    d = a - b
    return d - L * np.round(d / L)


@pytest.mark.parametrize("system,precision,segments", [
    ("copolymer", R.RELRES_PREC_FP32, 1),  # dihedrals inside the segmented drift kernel
    ("copolymer", R.RELRES_PREC_FP64, 1),
    ("long_chains", R.RELRES_PREC_FP32, 0),  # 300-bead chains: no segment holds a molecule
    ("long_chains", R.RELRES_PREC_FP64, 0),
])
def test_md_step_paths_track_the_oracle(torch, system, precision, segments):
    # both MD step paths (bonded terms in the segmented drift kernel, or the
    # separate bonded-term kernel + force sum + thermostat kernel) against the
    # oracle's velocity Verlet + CSVR over 20 steps
    if system == "copolymer":
        s = S.block_copolymer(n_chain=20)
    else:
        s = S.block_copolymer(n_chain=12, n_bead=300, block=150, density=0.5)
    ctx = R.Context(R.params_for(s, precision), R.topology_for(s))
    p = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    v = torch.tensor(s.vel, dtype=torch.float64, device="cuda")
    ctx.build_neighbors(p, s.box)
    th = torch.zeros((2, R.RELRES_THERMO_COLS), dtype=torch.float64, device="cuda")
    ctx.step(20, 1.0, p, v, t_target=s.temperature, tau_fs=100.0, seed=5, thermo_every=10, d_thermo=th)
    torch.cuda.synchronize()
    st = ctx.stats()
    ctx.close()
    assert st["step_segments"] == segments
    tab = O.table_for(s)
    po, vo, tho = O.md(s.pos, s.vel, s.box, s.masses, s.types, tab, s.n_types, s.excl, s.topo, 20, 1.0,
                       t_target=s.temperature, tau=100.0, seed=5)
    dx = float(np.abs(_wrapped(p.cpu().numpy(), po, s.box)).max())
    dv = float(np.abs(v.cpu().numpy() - vo).max() / np.abs(vo).max())
    ke = th.cpu().numpy()[-1, 3]
    print(f"{system} prec={precision} segments={segments}: max |dx| {dx:.2e} A, dv {dv:.2e}, "
          f"KE {ke:.6f} vs {tho[-1, 2]:.6f}")
    if precision == R.RELRES_PREC_FP64:
        assert dx < 1e-9 and dv < 1e-9
        assert ke == pytest.approx(tho[-1, 2], rel=1e-9)
    else:
        assert dx < 1e-4 and dv < 1e-4
        assert ke == pytest.approx(tho[-1, 2], rel=1e-5)


@pytest.mark.parametrize("precision,f_tol,e_tol", [(R.RELRES_PREC_FP64, 1e-10, 1e-10),
                                                   (R.RELRES_PREC_FP32, F_TOL, E_TOL)])
def test_orthorhombic_box_with_unequal_edges(torch, precision, f_tol, e_tol):
    # the neopentane liquid with its box and coordinates stretched by 1.25 along
    # y and compressed by 0.9 along z: different cell counts and fixed-point
    # scales per axis (forces, energies, virial and a short MD run)
    base = S.neopentane(n_mol=1500, seed=41)
    stretch = np.array([1.0, 1.25, 0.9])
    s = base.subset_copy(pos=np.mod(base.pos * stretch, base.box * stretch), box=base.box * stretch,
                         name="neopentane_orthorhombic")
    _check_full(torch, s, precision, f_tol, e_tol)
    ctx = R.Context(R.params_for(s, precision), R.topology_for(s))
    p = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    v = torch.tensor(s.vel, dtype=torch.float64, device="cuda")
    ctx.build_neighbors(p, s.box)
    st = ctx.stats()
    assert len(set(st["grid_fg"])) > 1  # the cell grid differs per axis
    ctx.step(20, 1.0, p, v)
    torch.cuda.synchronize()
    ctx.close()
    po, vo, _ = O.md(s.pos, s.vel, s.box, s.masses, s.types, O.table_for(s), s.n_types, s.excl, s.topo, 20, 1.0)
    dx = float(np.abs(_wrapped(p.cpu().numpy(), po, s.box)).max())
    print(f"orthorhombic prec={precision}: grid {st['grid_fg']}, max |dx| after 20 steps {dx:.2e} A")
    assert dx < (1e-9 if precision == R.RELRES_PREC_FP64 else 1e-4)
