"""Call boundaries of relres_step.

A call given back the position and velocity arrays the previous call
returned continues from that call's end state on the device: the forces are
reused and, in FP32 mode with the same time step, so are the velocity state
and the thermostat factors of the last step.  So a trajectory split into
calls of any length is the same bits as one call (FP32, CSVR).  A call whose
arrays were changed in between reads them: new velocities replace the
velocity state, new positions are read and their forces evaluated.  Both are
compared with a context that starts from the changed arrays; its lists are
built afresh, so FP32 forces can differ by an ulp (the compensated sums meet
the entries in another order), hence the FP32 tolerance (a change that was
not read would be off by 1e-3 A/fs or 0.4 A).
"""
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


def _periodic_max_diff(a, b, box):
    d = np.abs(a - b)
    return np.minimum(d, box - d).max()  # either side of the periodic boundary


def _ctx(torch, s, pos, vel, precision=R.RELRES_PREC_FP32):
    ctx = R.Context(R.params_for(s, precision), R.topology_for(s))
    p = torch.tensor(np.ascontiguousarray(pos), dtype=torch.float64, device="cuda")
    v = torch.tensor(np.ascontiguousarray(vel), dtype=torch.float64, device="cuda")
    ctx.build_neighbors(p, s.box)
    return ctx, p, v


@pytest.mark.parametrize("graphs", [True, False])
def test_trajectory_split_into_calls_is_one_call(torch, graphs):
    s = S.neopentane(n_mol=500, seed=23)
    runs = []
    for split in ([150], [100, 50], [1] * 30 + [120], [7] * 21 + [3]):
        assert sum(split) == 150
        ctx, p, v = _ctx(torch, s, s.pos, s.vel)
        ctx.set_graphs(graphs)
        for n in split:
            ctx.step(n, 2.0, p, v, t_target=s.temperature, tau_fs=100.0, seed=9)
        torch.cuda.synchronize()
        st = ctx.stats()
        runs.append((p.cpu().numpy(), v.cpu().numpy(), st["n_builds"], st["n_steps"]))
        ctx.close()
    p0, v0, b0, n0 = runs[0]
    assert n0 == 150 and b0 >= 2
    for p1, v1, b1, n1 in runs[1:]:
        assert n1 == 150 and b1 == b0
        assert np.array_equal(p0, p1) and np.array_equal(v0, v1)


@pytest.mark.parametrize("precision", [R.RELRES_PREC_FP32, R.RELRES_PREC_FP64])
def test_changed_arrays_are_read(torch, precision):
    s = S.neopentane(n_mol=500, seed=29)
    tol = 1e-6 if precision == R.RELRES_PREC_FP32 else 1e-9
    ctx, p, v = _ctx(torch, s, s.pos, s.vel, precision)
    ctx.step(40, 2.0, p, v, t_target=s.temperature, tau_fs=100.0, seed=3)
    torch.cuda.synchronize()
    # new velocities, same positions
    v.mul_(0.5)
    p_a, v_a = p.clone(), v.clone()
    ctx.step(10, 2.0, p, v, t_target=0.0, seed=4)
    ref, rp, rv = _ctx(torch, s, p_a.cpu().numpy(), v_a.cpu().numpy(), precision)
    ref.step(10, 2.0, rp, rv, t_target=0.0, seed=4)
    torch.cuda.synchronize()
    np.testing.assert_allclose(v.cpu().numpy(), rv.cpu().numpy(), rtol=0, atol=tol)
    assert _periodic_max_diff(p.cpu().numpy(), rp.cpu().numpy(), s.box) <= tol
    ref.close()
    # new positions (every atom moved by the same 0.4 A: the same forces), same velocities
    shift = torch.tensor([0.4, 0.0, 0.0], dtype=torch.float64, device="cuda")
    box = torch.tensor(s.box, dtype=torch.float64, device="cuda")
    p.copy_(torch.remainder(p + shift, box))
    p_b, v_b = p.clone(), v.clone()
    ctx.step(10, 2.0, p, v, t_target=0.0, seed=5)
    ref, rp, rv = _ctx(torch, s, p_b.cpu().numpy(), v_b.cpu().numpy(), precision)
    ref.step(10, 2.0, rp, rv, t_target=0.0, seed=5)
    torch.cuda.synchronize()
    np.testing.assert_allclose(v.cpu().numpy(), rv.cpu().numpy(), rtol=0, atol=tol)
    assert _periodic_max_diff(p.cpu().numpy(), rp.cpu().numpy(), s.box) <= tol
    ref.close()
    ctx.close()
