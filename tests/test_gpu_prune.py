"""Dynamic pruning of the neighbour lists (relres_set_prune): the pair kernels
walk lists pruned to the interaction cutoff + delta, re-pruned whenever an atom
has moved delta/2 since the last pass.  Dropped entries contribute exactly
zero, so with one thread per list and running (FP32 or FP64) force sums the
trajectory must be the same bits as without pruning; with the default
compensated sums, which add the entries four at a time, the grouping of the
pruned list differs and the forces agree to rounding.  Forces after
displacements between the pruning and the rebuild thresholds must still match
the FP64 oracle."""
import numpy as np
import pytest

from oracle import core as O
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


def _dev(torch, a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _run(torch, s, precision, delta, n_steps, dt, graphs=True, t_target=0.0, acc=R.RELRES_ACC_FP32):
    ctx = R.Context(R.params_for(s, precision), R.topology_for(s))
    ctx.set_force_accumulation(acc)
    ctx.set_pair_config(0)
    ctx.set_graphs(graphs)
    ctx.set_prune(delta)
    p = _dev(torch, s.pos)
    v = _dev(torch, s.vel)
    ctx.build_neighbors(p, s.box)
    th = torch.zeros((n_steps // 10, R.RELRES_THERMO_COLS), dtype=torch.float64, device="cuda")
    for _ in range(2):
        ctx.step(n_steps // 2, dt, p, v, t_target=t_target, tau_fs=100.0, seed=5, thermo_every=10,
                 d_thermo=th[: n_steps // 20] if _ == 0 else th[n_steps // 20:])
    torch.cuda.synchronize()
    out = p.cpu().numpy(), v.cpu().numpy(), th.cpu().numpy(), ctx.stats()
    ctx.close()
    return out


@pytest.mark.parametrize("precision,graphs", [(R.RELRES_PREC_FP32, True), (R.RELRES_PREC_FP32, False),
                                              (R.RELRES_PREC_FP64, True)])
def test_pruned_trajectory_is_bit_identical(torch, precision, graphs):
    s = S.neopentane(n_mol=1000, seed=31) if precision == R.RELRES_PREC_FP32 else S.propane()
    dt = 2.0 if precision == R.RELRES_PREC_FP32 else 1.0
    p0, v0, t0, st0 = _run(torch, s, precision, 0.0, 400, dt, graphs, t_target=s.temperature)
    p1, v1, t1, st1 = _run(torch, s, precision, 0.5, 400, dt, graphs, t_target=s.temperature)
    print(f"{s.name}: builds {st0['n_builds']}/{st1['n_builds']}, prunes {st1['n_prunes']}, "
          f"FG {st1['mean_fg']:.1f} -> {st1['mean_fg_pruned']:.1f}, CG {st1['mean_cg']:.1f} -> "
          f"{st1['mean_cg_pruned']:.1f}")
    assert st0["n_prunes"] == 0 and st0["prune_delta"] == 0.0
    assert st1["prune_delta"] == 0.5
    assert st1["n_builds"] == st0["n_builds"] >= 3
    assert st1["n_prunes"] > 2 * st1["n_builds"]
    assert st1["mean_fg_pruned"] < 0.8 * st1["mean_fg"]
    if st1["n_hybrid"]:
        assert st1["mean_cg_pruned"] < 0.95 * st1["mean_cg"]
    assert np.array_equal(p0, p1) and np.array_equal(v0, v1)
    # thermo rows: E_FG, E_CG, E_bonded, kinetic energy, six virial components.
    # The trajectory, the kinetic and bonded energies and the virial are the
    # same bits; the pair energies of the FP32 path agree to rounding: each
    # pair's energy is evaluated once from a per-warp queue, whose grouping
    # depends on where the entries sit in the lists walked
    assert np.array_equal(t0[:, 2:], t1[:, 2:])
    if precision == R.RELRES_PREC_FP64:
        assert np.array_equal(t0, t1)
    else:
        assert np.allclose(t0[:, :2], t1[:, :2], rtol=1e-12, atol=0), np.abs(t0[:, :2] - t1[:, :2]).max()


def test_compute_after_displacements_between_the_thresholds(torch):
    # atoms moved 0.3-0.9 A: past the pruning trigger (delta/2 = 0.25 A), short
    # of the rebuild trigger (skin/2 = 1 A); the lists are pruned again, not
    # rebuilt, and the forces are the bits of the unpruned lists
    s = S.neopentane(n_mol=500, seed=17)
    rng = np.random.default_rng(4)
    shift = rng.normal(size=s.pos.shape)
    shift *= (0.3 + 0.6 * rng.random((s.n_atoms, 1))) / np.linalg.norm(shift, axis=1, keepdims=True)
    pos = np.mod(s.pos + shift, s.box)
    out = []
    for delta in (0.5, 0.0):
        ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
        ctx.set_force_accumulation(R.RELRES_ACC_FP32)  # running sums: pruning keeps the bits
        ctx.set_prune(delta)
        p = _dev(torch, s.pos)
        ctx.build_neighbors(p, s.box)
        f = torch.empty_like(p)
        ctx.compute(p, f)
        st0 = ctx.stats()
        ctx.compute(_dev(torch, pos), f)
        torch.cuda.synchronize()
        out.append((f.cpu().numpy(), st0, ctx.stats()))
        ctx.close()
    (f1, a0, a1), (f0, b0, b1) = out
    assert a1["n_builds"] == a0["n_builds"] and a1["n_prunes"] == a0["n_prunes"] + 1
    assert b1["n_builds"] == b0["n_builds"] and b1["n_prunes"] == 0
    assert np.array_equal(f1, f0)
    # and against the oracle (the displaced configuration has close contacts,
    # whose large forces set the FP32 rounding)
    tab = O.table_for(s)
    fr, _, _ = O.pair_forces(pos, s.box, s.types, tab, s.n_types, s.excl)
    fb, _ = O.bonded(pos, s.box, s.topo)
    ref = fr + fb
    rel = np.abs(f1 - ref).max(1) / np.maximum(np.linalg.norm(ref, axis=1), 1.0)
    print(f"max per-atom relative force error {rel.max():.2e}")
    assert rel.max() <= 1e-5


def test_prune_can_be_switched_on_and_off(torch):
    s = S.neopentane(n_mol=400, seed=3)
    ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
    ctx.set_force_accumulation(R.RELRES_ACC_FP32)  # running sums: pruning keeps the bits
    p = _dev(torch, s.pos)
    ctx.build_neighbors(p, s.box)
    forces = []
    for delta in (0.5, 0.0, 1.0, 0.25):
        ctx.set_prune(delta)
        f = torch.empty_like(p)
        ctx.compute(p, f)
        forces.append(f.cpu().numpy())
        assert ctx.stats()["prune_delta"] == delta
    ctx.close()
    for f in forces[1:]:
        assert np.array_equal(f, forces[0])


def test_separate_pruning_pass_with_two_threads_per_slot(torch):
    # pair launches with two threads per slot cannot prune as they go: a
    # separate pruning pass runs on the steps that need one; the lists it
    # leaves must still hold every interacting pair
    s = S.neopentane(n_mol=1000, seed=23)
    ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
    ctx.set_pair_config(3)
    ctx.set_prune(0.5)
    p = _dev(torch, s.pos)
    v = _dev(torch, s.vel)
    ctx.build_neighbors(p, s.box)
    ctx.step(300, 2.0, p, v, t_target=s.temperature, tau_fs=100.0, seed=2)
    st0 = ctx.stats()
    f = torch.empty_like(p)
    ctx.compute(p, f)
    torch.cuda.synchronize()
    st1 = ctx.stats()
    pos = p.cpu().numpy()
    ctx.close()
    assert st0["pair_tpa"] == 2 and st0["n_prunes"] > 2 * st0["n_builds"] >= 6
    assert st1["n_prunes"] == st0["n_prunes"] and st1["n_builds"] == st0["n_builds"]
    tab = O.table_for(s)
    fr, _, _ = O.pair_forces(pos, s.box, s.types, tab, s.n_types, s.excl)
    fb, _ = O.bonded(pos, s.box, s.topo)
    ref = fr + fb
    err = float(np.abs(f.cpu().numpy() - ref).max() / np.sqrt((ref * ref).sum(1).mean()))
    assert err <= 1e-5, err


def test_pruned_forces_with_compensated_sums_agree_to_rounding(torch):
    # the default accumulation groups list entries in fours, so pruned and full
    # walks round differently: the forces agree to a few FP32 ulps of the sum
    s = S.neopentane(n_mol=1000, seed=31)
    rng = np.random.default_rng(8)
    pos = np.mod(s.pos + rng.normal(scale=0.1, size=s.pos.shape), s.box)
    out = []
    for delta in (0.5, 0.0):
        ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
        assert ctx.stats()["force_acc"] == R.RELRES_ACC_COMPENSATED
        ctx.set_prune(delta)
        p = _dev(torch, pos)
        ctx.build_neighbors(p, s.box)
        f = torch.empty_like(p)
        ctx.compute(p, f)
        torch.cuda.synchronize()
        out.append(f.cpu().numpy())
        ctx.close()
    rms = np.sqrt((out[1] ** 2).sum(1).mean())
    assert np.abs(out[0] - out[1]).max() / rms < 1e-6
