"""Segments of whole molecules that share the term records of a prototype.

The drift kernel evaluates the bonded terms of each segment of whole molecules
in one block.  A segment whose term records and incident-term lists are those
of an earlier segment shifted by an atom offset reads the earlier segment's
records (its prototype) instead of its own.  These tests step a liquid of
identical molecules (every full segment shares one prototype) and the same
liquid with the two atoms of one bond of randomly chosen molecules written in
the other order (every segment its own prototype; a bond's force does not
depend on the order of its atoms: the fixed-point difference and every
product only change sign), and require the same trajectory bit for bit.
"""
import copy

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


def _flip_some_bonds(system, seed=11):
    s = copy.copy(system)
    topo = dict(system.topo)
    bonds = np.array(topo["bonds"], dtype=np.int64).reshape(-1, 2).copy()
    rng = np.random.default_rng(seed)
    flip = rng.random(len(bonds)) < 0.25
    bonds[flip] = bonds[flip][:, ::-1]
    topo["bonds"] = bonds
    s.topo = topo
    return s


def _run(torch, system, precision, n_steps, t_target):
    ctx = R.Context(R.params_for(system, precision), R.topology_for(system))
    p = torch.tensor(system.pos, dtype=torch.float64, device="cuda")
    v = torch.tensor(system.vel, dtype=torch.float64, device="cuda")
    ctx.build_neighbors(p, system.box)
    ctx.step(n_steps, 2.0 if precision == R.RELRES_PREC_FP32 else 1.0, p, v, t_target=t_target, seed=3)
    torch.cuda.synchronize()
    st = ctx.stats()
    ctx.close()
    return p.cpu().numpy(), v.cpu().numpy(), st


@pytest.mark.parametrize("name,precision,t_target", [
    ("neopentane", R.RELRES_PREC_FP32, 260.0),
    ("propane", R.RELRES_PREC_FP64, 0.0),
])
def test_prototype_segments_give_the_same_trajectory(torch, name, precision, t_target):
    base = S.neopentane(n_mol=4000, seed=9) if name == "neopentane" else S.propane()
    p0, v0, st0 = _run(torch, base, precision, 60, t_target)
    p1, v1, st1 = _run(torch, _flip_some_bonds(base), precision, 60, t_target)
    print(f"{name}: {st0['n_segments']} segments, {st0['n_segment_protos']} prototypes "
          f"(flipped bonds: {st1['n_segment_protos']})")
    assert st0["step_segments"] == 1 and st1["step_segments"] == 1
    assert st0["n_segments"] == st1["n_segments"] > 1
    # identical molecules: the full segments share one prototype, a shorter last one has its own
    assert st0["n_segment_protos"] <= 2
    assert st1["n_segment_protos"] == st1["n_segments"]
    assert np.array_equal(p0, p1)
    assert np.array_equal(v0, v1)
