"""GPU parity of librelres against the FP64 oracle (through the C ABI).

Error measures (the tolerances of the method's specification):
  forces: max_i |F_i - F_i^ref| / rms_i |F_i^ref|  <= 1e-5
  energy: |E - E^ref| / |E^ref|                      <= 1e-7
FP64 mode must meet far tighter bounds (1e-10); FP32 mode (FP32 pair terms
from exact fixed-point coordinate differences) the ones above.
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


def gpu_compute(torch, system, precision, shift=True, pos=None):
    ctx = R.Context(R.params_for(system, precision, shift), R.topology_for(system))
    p = _dev(torch, system.pos if pos is None else pos)
    ctx.build_neighbors(p, system.box)
    f = torch.empty_like(p)
    e = torch.zeros(4, dtype=torch.float64, device="cuda")
    w = torch.zeros(6, dtype=torch.float64, device="cuda")
    ctx.compute(p, f, e, w)
    torch.cuda.synchronize()
    out = f.cpu().numpy(), e.cpu().numpy(), w.cpu().numpy(), ctx.stats()
    ctx.close()
    return out


def oracle_compute(system, shift=True, pos=None):
    pos = system.pos if pos is None else pos
    tab = O.table_for(system, shift)
    f, e, w = O.pair_forces(pos, system.box, system.types, tab, system.n_types, system.excl)
    fb, eb = O.bonded(pos, system.box, system.topo)
    return f + fb, e, float(eb.sum()), w


def force_err(f, ref):
    rms = math.sqrt((ref * ref).sum(1).mean())
    return float(np.abs(f - ref).max() / rms)


def check(torch, system, precision, f_tol, e_tol, shift=True):
    f, e, w, st = gpu_compute(torch, system, precision, shift)
    fr, er, ebr, wr = oracle_compute(system, shift)
    ferr = force_err(f, fr)
    eerr = abs(e[0] + e[1] - er) / abs(er)
    berr = abs(e[2] - ebr) / max(1.0, abs(ebr))
    werr = float(np.abs(w - wr).max() / np.abs(wr[:3]).max())
    print(f"{system.name} prec={precision}: force {ferr:.2e} energy {eerr:.2e} "
          f"bonded {berr:.2e} virial {werr:.2e}  lists {st['mean_fg']:.1f}/{st['mean_cg']:.1f}")
    assert ferr <= f_tol, ferr
    assert eerr <= e_tol, eerr
    assert berr <= e_tol, berr
    assert werr <= 10 * f_tol, werr
    assert e[3] == pytest.approx(e[0] + e[1] + e[2], rel=1e-14, abs=1e-12)
    return ferr, eerr


def test_fp64_propane_full_config(torch):
    check(torch, S.propane(), R.RELRES_PREC_FP64, 1e-10, 1e-10)


def test_fp64_propane_no_shift(torch):
    check(torch, S.propane(), R.RELRES_PREC_FP64, 1e-10, 1e-10, shift=False)


def test_fp32_propane_full_config(torch):
    check(torch, S.propane(), R.RELRES_PREC_FP32, F_TOL, E_TOL)


def test_fp32_neopentane_2500_atoms(torch):
    check(torch, S.neopentane(n_mol=500), R.RELRES_PREC_FP32, F_TOL, E_TOL)


def test_fp64_neopentane_2500_atoms(torch):
    check(torch, S.neopentane(n_mol=500), R.RELRES_PREC_FP64, 1e-10, 1e-10)


def test_fp32_fg_only_reference(torch):
    check(torch, S.fg_only(S.neopentane(n_mol=500)), R.RELRES_PREC_FP32, F_TOL, E_TOL)


def test_fp32_ragged_sizes(torch):
    # sizes that are not multiples of the 256-thread block, several cells per axis
    for n_mol in (251, 343):
        check(torch, S.neopentane(n_mol=n_mol, seed=3), R.RELRES_PREC_FP32, F_TOL, E_TOL)


def _brute_force_list_count(system, rlist, hybrid_only):
    pos, L = system.pos, system.box
    sel = np.arange(system.n_atoms)
    if hybrid_only:
        sel = sel[system.is_hybrid[system.types] == 1]
    p = pos[sel]
    off, idx = system.excl
    total = 0
    for a in range(len(sel)):
        d = p - p[a]
        d -= L * np.round(d / L)
        r2 = (d * d).sum(1)
        hit = np.nonzero(r2 < rlist * rlist)[0]
        hit = hit[hit != a]
        ex = set(idx[off[sel[a]]:off[sel[a] + 1]].tolist())
        total += sum(1 for h in hit if sel[h] not in ex)
    return total


def test_list_sizes_match_brute_force(torch):
    s = S.neopentane(n_mol=300, seed=5)
    _, _, _, st = gpu_compute(torch, s, R.RELRES_PREC_FP32)
    nfg = _brute_force_list_count(s, st["list_radius_fg"], False)
    ncg = _brute_force_list_count(s, st["list_radius_cg"], True)
    assert round(st["mean_fg"] * s.n_atoms) == nfg
    assert round(st["mean_cg"] * s.n_hybrid) == ncg


def _gpu_md(torch, system, precision, n_steps, dt, t_target=0.0, seed=0, every=1):
    ctx = R.Context(R.params_for(system, precision), R.topology_for(system))
    p = _dev(torch, system.pos)
    v = _dev(torch, system.vel)
    ctx.build_neighbors(p, system.box)
    rows = n_steps // every if every else 0
    th = torch.zeros((max(rows, 1), R.RELRES_THERMO_COLS), dtype=torch.float64, device="cuda")
    ctx.step(n_steps, dt, p, v, t_target=t_target, tau_fs=100.0, seed=seed, thermo_every=every,
             d_thermo=th)
    torch.cuda.synchronize()
    out = p.cpu().numpy(), v.cpu().numpy(), th.cpu().numpy(), ctx.stats()
    ctx.close()
    return out


def _oracle_md(system, n_steps, dt, t_target=0.0, seed=0):
    tab = O.table_for(system)
    return O.md(system.pos, system.vel, system.box, system.masses, system.types, tab,
                system.n_types, system.excl, system.topo, n_steps, dt, t_target=t_target,
                tau=100.0, seed=seed)


def _wrapped_diff(a, b, L):
    d = a - b
    return d - L * np.round(d / L)


def test_fp64_nve_trajectory_matches_oracle(torch):
    s = S.propane()
    p, v, th, st = _gpu_md(torch, s, R.RELRES_PREC_FP64, 40, 1.0)
    po, vo, tho = _oracle_md(s, 40, 1.0)
    assert np.abs(_wrapped_diff(p, po, s.box)).max() < 1e-9
    assert np.abs(v - vo).max() < 1e-10
    np.testing.assert_allclose(th[:, 0] + th[:, 1], tho[:, 0], rtol=1e-9)
    np.testing.assert_allclose(th[:, 2], tho[:, 1], rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(th[:, 3], tho[:, 2], rtol=1e-9)
    assert np.all(p >= 0.0) and np.all(p < s.box)


def test_fp64_propane_1000_nve_steps(torch):
    # the propane-like configuration: 216 molecules, FP64, 1000 NVE steps at 1 fs
    s = S.propane()
    p, v, th, st = _gpu_md(torch, s, R.RELRES_PREC_FP64, 1000, 1.0, every=10)
    po, vo, tho = _oracle_md(s, 1000, 1.0)
    tho = tho[9::10]
    assert st["n_builds"] >= 2
    np.testing.assert_allclose(th[:, 0] + th[:, 1], tho[:, 0], rtol=1e-8)
    np.testing.assert_allclose(th[:, 3], tho[:, 2], rtol=1e-8)
    assert np.abs(_wrapped_diff(p, po, s.box)).max() < 1e-6


def test_fp64_csvr_trajectory_matches_oracle(torch):
    s = S.propane()
    p, v, th, st = _gpu_md(torch, s, R.RELRES_PREC_FP64, 30, 1.0, t_target=230.0, seed=11)
    po, vo, tho = _oracle_md(s, 30, 1.0, t_target=230.0, seed=11)
    np.testing.assert_allclose(th[:, 3], tho[:, 2], rtol=1e-8)
    assert np.abs(_wrapped_diff(p, po, s.box)).max() < 1e-8


def test_fp32_trajectory_tracks_oracle_and_rebuilds(torch):
    # long enough for several device-side list rebuilds
    s = S.propane()
    p, v, th, st = _gpu_md(torch, s, R.RELRES_PREC_FP32, 200, 1.0, every=10)
    assert st["n_builds"] >= 2
    # forces at the final positions: stepping context (lists rebuilt on the
    # device) vs a fresh build vs the oracle
    f, e, w, _ = gpu_compute(torch, s, R.RELRES_PREC_FP32, pos=p)
    fr, er, ebr, wr = oracle_compute(s, pos=p)
    assert force_err(f, fr) <= F_TOL


def test_fp32_nve_energy_drift(torch):
    s = S.propane()
    _, _, th, _ = _gpu_md(torch, s, R.RELRES_PREC_FP32, 1000, 1.0, every=10)
    etot = th[:, 0] + th[:, 1] + th[:, 2] + th[:, 3]
    ke = th[:, 3].mean()
    # the lattice start relaxes in the first ~50 fs; look at the rest
    tail = etot[10:]
    drift = abs(tail[-1] - tail[0]) / ke
    assert drift < 2e-3, drift


def test_graph_and_stream_paths_agree_bitwise(torch):
    # relres_step as CUDA graphs (conditional rebuild nodes) and as stream
    # launches (rebuild kernels gated on the device flag): same bits, same
    # rebuilds; repeated calls reuse the captured graph
    s = S.neopentane(n_mol=500, seed=12)
    outs = []
    for graphs in (True, False):
        ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
        ctx.set_graphs(graphs)
        p = _dev(torch, s.pos)
        v = _dev(torch, s.vel)
        ctx.build_neighbors(p, s.box)
        th = torch.zeros((30, R.RELRES_THERMO_COLS), dtype=torch.float64, device="cuda")
        ctx.set_timing(True)
        for _ in range(3):
            ctx.step(100, 2.0, p, v, t_target=260.0, tau_fs=100.0, seed=3, thermo_every=10, d_thermo=th)
        torch.cuda.synchronize()
        outs.append((p.cpu().numpy(), v.cpu().numpy(), th.cpu().numpy(), ctx.stats(), ctx.timings()))
        ctx.close()
    (pg, vg, tg, sg, mg), (ps, vs, ts, ss, ms) = outs
    assert sg["n_builds"] == ss["n_builds"] and sg["n_builds"] >= 3
    assert np.array_equal(pg, ps) and np.array_equal(vg, vs) and np.array_equal(tg, ts)
    # 300 steps (30 of them energy steps) plus the force evaluation at the
    # start of the first call
    assert mg["pair"][1] == ms["pair"][1] == 271
    assert mg["pair_ev"][1] == ms["pair_ev"][1] == 30
    assert mg["rebuild"][1] == 300 and mg["rebuild"][0] > 0.0
    # graph mode launches no binning or list kernel on steps without a rebuild
    assert sg["n_launches"] < ss["n_launches"]


def test_programmatic_dependent_launches_change_no_bit(torch):
    # untimed steps launch the force sum and the next drift as programmatic
    # dependents of their predecessors (each starts during the previous
    # kernel's tail and waits for it before reading its results); timed steps
    # launch every kernel the ordinary way.  Both, as graphs and as stream
    # launches, over 300 steps with rebuilds, pruning passes and energy steps:
    # the same bits.
    s = S.neopentane(n_mol=2000, seed=14)
    outs = []
    for graphs in (True, False):
        for timing in (False, True):
            ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
            ctx.set_graphs(graphs)
            p = _dev(torch, s.pos)
            v = _dev(torch, s.vel)
            ctx.build_neighbors(p, s.box)
            th = torch.zeros((30, R.RELRES_THERMO_COLS), dtype=torch.float64, device="cuda")
            ctx.set_timing(timing)
            for _ in range(3):
                ctx.step(100, 2.0, p, v, t_target=260.0, tau_fs=100.0, seed=4, thermo_every=10, d_thermo=th)
            torch.cuda.synchronize()
            st = ctx.stats()
            outs.append((p.cpu().numpy(), v.cpu().numpy(), th.cpu().numpy(), st["n_builds"], st["n_prunes"]))
            ctx.close()
    p0, v0, t0, b0, n0 = outs[0]
    assert b0 >= 3 and n0 > b0
    for p1, v1, t1, b1, n1 in outs[1:]:
        assert np.array_equal(p0, p1) and np.array_equal(v0, v1) and np.array_equal(t0, t1)
        assert (b1, n1) == (b0, n0)


def test_every_pair_launch_configuration_matches_oracle(torch):
    # threads per atom 1/2/4/8 x block sizes: each within the force tolerance
    s = S.neopentane(n_mol=500, seed=6)
    fr, er, ebr, wr = oracle_compute(s)
    ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
    p = _dev(torch, s.pos)
    ctx.build_neighbors(p, s.box)
    f = torch.empty_like(p)
    for cfg in range(7):
        ctx.set_pair_config(cfg)
        ctx.compute(p, f)
        torch.cuda.synchronize()
        err = force_err(f.cpu().numpy(), fr)
        st = ctx.stats()
        print(f"pair config {cfg} (tpa {st['pair_tpa']}, block {st['pair_block']}): force {err:.2e}")
        assert err <= F_TOL, (cfg, err)
    ctx.close()


@pytest.mark.parametrize("prune", [0.5, 0.0])
def test_fp64_several_threads_per_slot_keep_the_bits(torch, prune):
    # small FP64 systems walk each slot with eight threads in forces-only
    # launches; energy launches use one: the forces must be the same bits
    s = S.propane()
    ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP64), R.topology_for(s))
    ctx.set_prune(prune)
    p = _dev(torch, s.pos)
    ctx.build_neighbors(p, s.box)
    assert ctx.stats()["pair_tpa"] == 8 and ctx.stats()["pair_block"] == 32
    f8 = torch.empty_like(p)
    f1 = torch.empty_like(p)
    e = torch.zeros(4, dtype=torch.float64, device="cuda")
    ctx.compute(p, f8)
    ctx.compute(p, f1, e)
    torch.cuda.synchronize()
    assert np.array_equal(f8.cpu().numpy(), f1.cpu().numpy())
    fr, _, _, _ = oracle_compute(s)
    assert force_err(f8.cpu().numpy(), fr) <= 1e-10
    ctx.close()


@pytest.mark.parametrize("prune", [0.5, 0.0])
def test_autotuner_picks_a_configuration(torch, prune):
    s = S.neopentane(n_mol=5000, seed=2)  # 25 000 atoms: above the tuning threshold
    ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
    ctx.set_prune(prune)
    p = _dev(torch, s.pos)
    v = _dev(torch, s.vel)
    ctx.build_neighbors(p, s.box)
    ctx.step(5, 2.0, p, v)
    st = ctx.stats()
    # with pruning only one thread per atom (the launches that prune as they go)
    assert st["pair_tpa"] in ((1,) if prune > 0 else (1, 2, 4, 8)) and st["pair_block"] in (128, 256, 512)
    print(f"autotuned (prune {prune}): tpa {st['pair_tpa']} block {st['pair_block']}")
    ctx.close()


def test_list_overflow_inside_a_step_block_rolls_back_and_grows(torch):
    # lists sized exactly for the first build: a later device-side rebuild
    # overflows, the block is rolled back, the lists grow, the block reruns;
    # the forces at the end still match the oracle
    s = S.neopentane(n_mol=500, seed=31)
    ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
    p = _dev(torch, s.pos)
    v = _dev(torch, s.vel)
    ctx.build_neighbors(p, s.box)
    st0 = ctx.stats()
    ctx.set_list_caps(st0["max_fg"], st0["max_cg"])
    c1 = ctx.stats()
    ctx.step(600, 2.0, p, v, t_target=260.0, tau_fs=100.0, seed=4)
    torch.cuda.synchronize()
    s1 = ctx.stats()
    assert s1["n_steps"] == 600
    assert s1["cap_fg"] > c1["cap_fg"] or s1["cap_cg"] > c1["cap_cg"], (c1, s1)  # grew during the steps
    pos = p.cpu().numpy()
    f = torch.empty_like(p)
    ctx.compute(p, f)
    torch.cuda.synchronize()
    ctx.close()
    fr, _, _, _ = oracle_compute(s, pos=pos)
    assert force_err(f.cpu().numpy(), fr) <= F_TOL


def test_list_overflow_at_the_first_build_grows_the_lists(torch):
    # molecules crowded into half of a box twice as long: the capacity guessed
    # from the mean density is too small for the real one
    base = S.neopentane(n_mol=400, seed=32)
    pos = base.pos.copy()
    box = base.box.copy()
    box[0] *= 2.0
    s = base.subset_copy(pos=pos, box=box)
    f, e, w, st = gpu_compute(torch, s, R.RELRES_PREC_FP32)
    fr, er, ebr, wr = oracle_compute(s)
    assert force_err(f, fr) <= F_TOL
    assert abs(e[0] + e[1] - er) / abs(er) <= E_TOL


def test_box_too_small_is_an_error(torch):
    s = S.propane(n_mol=64, box=25.0)
    ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
    p = _dev(torch, s.pos)
    with pytest.raises(R.RelresError) as ei:
        ctx.build_neighbors(p, s.box)
    assert ei.value.status == 3
    ctx.close()


def test_nonfinite_position_is_an_error(torch):
    s = S.propane()
    ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
    p = _dev(torch, s.pos)
    ctx.build_neighbors(p, s.box)
    bad = p.clone()
    bad[5, 1] = float("nan")
    f = torch.empty_like(p)
    with pytest.raises(R.RelresError) as ei:
        ctx.compute(bad, f)
    assert ei.value.status == 5
    # the context stays usable
    ctx.compute(p, f)
    ctx.close()


def test_measured_device_rates_are_plausible(torch):
    # the probe kernels behind the design choices and the FLOP side of the roofline
    scratch = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    r = R.relres_measure_rates(scratch)
    print(r)
    assert r["sm_count"] > 0 and r["clock_mhz"] > 0
    assert 32 <= r["ffma_per_clk_sm"] <= 160
    assert 0 < r["dfma_per_clk_sm"] < r["ffma_per_clk_sm"]
    assert 0 < r["conv64_per_clk_sm"] < r["ffma_per_clk_sm"]
    assert 500 < r["copy_gbs"] < 20000
    with pytest.raises(R.RelresError):
        R.relres_measure_rates(scratch[:1024])  # too small
