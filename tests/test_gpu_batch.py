"""Batches of independent replicas (relres_batch_step): every block of steps of
all replicas runs as one CUDA graph, where replicas that allow it (same
precision and accumulation) share one drift, one pair and one force-sum launch
per step and the others run their own kernels on branches of the graph.  Every
form must give the bits of stepping each context alone with the same
arguments, and FP64 batches the oracle's velocity Verlet + CSVR."""
import numpy as np
import pytest

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


def _systems():
    # the two chemistries of the batched workload, uneven sizes and temperatures
    return [S.propane(n_mol=216, temperature=230.0, seed=1),
            S.neopentane(n_mol=500, temperature=260.0, seed=2),
            S.neopentane(n_mol=300, temperature=200.0, seed=3),
            S.propane(n_mol=400, box=31.8 * (400 / 216) ** (1 / 3), temperature=290.0, seed=4),
            S.neopentane(n_mol=5000, temperature=240.0, seed=5)]


def _contexts(torch, systems, pair_cfg):
    out = []
    for s in systems:
        ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP32), R.topology_for(s))
        if pair_cfg is not None:
            ctx.set_pair_config(pair_cfg)
        p = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
        v = torch.tensor(s.vel, dtype=torch.float64, device="cuda")
        ctx.build_neighbors(p, s.box)
        th = torch.zeros((25, R.RELRES_THERMO_COLS), dtype=torch.float64, device="cuda")
        out.append((ctx, p, v, th))
    return out


@pytest.mark.parametrize("mode", [-1, 0, 1])
def test_batch_matches_each_replica_stepped_alone(torch, mode):
    systems = _systems()
    temps = [s.temperature for s in systems]
    seeds = [11, 12, 13, 14, 15]
    # alone
    solo = _contexts(torch, systems, 0)
    for (ctx, p, v, th), t, sd in zip(solo, temps, seeds):
        for _ in range(2):
            ctx.step(125, 2.0, p, v, t_target=t, tau_fs=100.0, seed=sd, thermo_every=10, d_thermo=th)
    torch.cuda.synchronize()
    # batched (two calls: the captured graph is reused for the second)
    batch_ctx = _contexts(torch, systems, 0)
    batch = R.Batch([c for c, _, _, _ in batch_ctx])
    batch.set_mode(mode)
    for _ in range(2):
        batch.step(125, 2.0, [p for _, p, _, _ in batch_ctx], [v for _, _, v, _ in batch_ctx], temps, 100.0, seeds,
                   thermo_every=10, d_thermo=[th for _, _, _, th in batch_ctx])
    torch.cuda.synchronize()
    for k, ((c1, p1, v1, t1), (c2, p2, v2, t2)) in enumerate(zip(solo, batch_ctx)):
        s1, s2 = c1.stats(), c2.stats()
        assert s1["n_builds"] == s2["n_builds"] and s1["n_steps"] == s2["n_steps"] == 250, k
        assert np.array_equal(p1.cpu().numpy(), p2.cpu().numpy()), k
        assert np.array_equal(v1.cpu().numpy(), v2.cpu().numpy()), k
        assert np.array_equal(t1.cpu().numpy(), t2.cpu().numpy()), k
    assert max(c.stats()["n_builds"] for c, _, _, _ in batch_ctx) >= 3
    # automatic: the four replicas of at most 16 384 atoms share launches, the
    # 25 000-atom one runs on its own branch
    assert batch.n_shared() == {-1: 4, 0: 0, 1: 5}[mode]
    batch.close()
    for c, _, _, _ in solo + batch_ctx:
        c.close()


def test_batch_with_autotuned_replicas_runs_and_conserves_momentum(torch):
    systems = _systems()[1:]
    ctxs = _contexts(torch, systems, None)
    batch = R.Batch([c for c, _, _, _ in ctxs])
    batch.step(200, 2.0, [p for _, p, _, _ in ctxs], [v for _, _, v, _ in ctxs], [0.0] * len(ctxs), 100.0,
               list(range(len(ctxs))))
    torch.cuda.synchronize()
    for (c, p, v, _), s in zip(ctxs, systems):
        st = c.stats()
        assert st["n_steps"] == 200 and st["pair_tpa"] in (1, 2, 4, 8)
        m = s.mass_by_type[s.types][:, None]
        mom = (m * v.cpu().numpy()).sum(0)
        assert np.abs(mom).max() < 1e-6 * (m * np.abs(v.cpu().numpy())).sum(), mom
    batch.close()
    for c, _, _, _ in ctxs:
        c.close()


def test_fp64_batch_of_uneven_replicas_matches_oracle_md(torch):
    """Four replicas of different sizes and chemistries stepped together in
    FP64 for 30 steps with the CSVR thermostat: each replica's positions,
    velocities and thermo rows against the oracle's velocity Verlet + CSVR of
    the same replica alone (Section 3.2, MD in the canonical ensemble), to the
    tolerances of the single-context FP64 CSVR trajectory test."""
    from oracle import core as O

    systems = [S.propane(n_mol=216, temperature=230.0, seed=21),
               S.neopentane(n_mol=300, temperature=200.0, seed=22),
               S.propane(n_mol=343, box=31.8 * 7 / 6, temperature=280.0, seed=23),
               S.neopentane(n_mol=500, temperature=260.0, seed=24)]
    seeds = [31, 32, 33, 34]
    steps, dt = 30, 1.0
    ctxs = []
    for s in systems:
        ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP64), R.topology_for(s))
        p = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
        v = torch.tensor(s.vel, dtype=torch.float64, device="cuda")
        ctx.build_neighbors(p, s.box)
        th = torch.zeros((steps, R.RELRES_THERMO_COLS), dtype=torch.float64, device="cuda")
        ctxs.append((ctx, p, v, th))
    batch = R.Batch([c for c, _, _, _ in ctxs])
    batch.step(steps, dt, [p for _, p, _, _ in ctxs], [v for _, _, v, _ in ctxs],
               [s.temperature for s in systems], 100.0, seeds, thermo_every=1,
               d_thermo=[th for _, _, _, th in ctxs])
    torch.cuda.synchronize()
    assert batch.n_shared() == 4
    for k, ((ctx, p, v, th), s, sd) in enumerate(zip(ctxs, systems, seeds)):
        po, vo, tho = O.md(s.pos, s.vel, s.box, s.masses, s.types, O.table_for(s), s.n_types, s.excl, s.topo,
                           steps, dt, t_target=s.temperature, tau=100.0, seed=sd)
        pg, vg, tg = p.cpu().numpy(), v.cpu().numpy(), th.cpu().numpy()
        d = pg - po
        d -= s.box * np.round(d / s.box)
        assert np.abs(d).max() < 1e-8, k
        assert np.abs(vg - vo).max() < 1e-9, k
        np.testing.assert_allclose(tg[:, 3], tho[:, 2], rtol=1e-8, err_msg=f"replica {k} KE")
        np.testing.assert_allclose(tg[:, 0] + tg[:, 1], tho[:, 0], rtol=1e-8, err_msg=f"replica {k} pair E")
        np.testing.assert_allclose(tg[:, 2], tho[:, 1], rtol=1e-7, atol=1e-9, err_msg=f"replica {k} bonded E")
        assert ctx.stats()["n_steps"] == steps
    batch.close()
    for c, _, _, _ in ctxs:
        c.close()


def test_mixed_precision_batch_takes_graph_branches_and_matches_solo(torch):
    """Replicas whose kernels cannot share a launch (one FP64, one FP32) run
    on graph branches, with the bits of stepping each alone."""
    systems = [S.propane(n_mol=216, temperature=230.0, seed=41), S.neopentane(n_mol=400, temperature=250.0, seed=42)]
    precs = [R.RELRES_PREC_FP64, R.RELRES_PREC_FP32]

    def make():
        out = []
        for s, pr in zip(systems, precs):
            ctx = R.Context(R.params_for(s, pr), R.topology_for(s))
            ctx.set_pair_config(0)
            p = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
            v = torch.tensor(s.vel, dtype=torch.float64, device="cuda")
            ctx.build_neighbors(p, s.box)
            out.append((ctx, p, v))
        return out

    temps = [s.temperature for s in systems]
    solo = make()
    for (c, p, v), t, sd in zip(solo, temps, (3, 4)):
        c.step(60, 1.0, p, v, t_target=t, tau_fs=100.0, seed=sd)
    both = make()
    batch = R.Batch([c for c, _, _ in both])
    batch.step(60, 1.0, [p for _, p, _ in both], [v for _, _, v in both], temps, 100.0, [3, 4])
    torch.cuda.synchronize()
    assert batch.n_shared() == 0
    # shared launches cannot mix precisions
    batch.set_mode(1)
    with pytest.raises(R.RelresError):
        batch.step(10, 1.0, [p for _, p, _ in both], [v for _, _, v in both], temps, 100.0, [3, 4])
    for (c1, p1, v1), (c2, p2, v2) in zip(solo, both):
        assert np.array_equal(p1.cpu().numpy(), p2.cpu().numpy())
        assert np.array_equal(v1.cpu().numpy(), v2.cpu().numpy())
    batch.close()
    for c, _, _ in solo + both:
        c.close()
