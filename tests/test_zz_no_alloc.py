"""relres_pair_forces_static: the entry point that allocates no device memory.

It exists for callers that cannot let a library allocate device memory (a host
program that owns the GPU memory budget through its own allocator, or a loop
where cudaMalloc's device synchronisation is not allowed).  Its scratch lives
in one static device array shared by every call.  This test calls it through
the C ABI twice in a row (at two different configurations, so that any stale
scratch contents from the first call would show) and compares each result with
relres_compute, the context-based entry point, within the FP64 tolerances of
the other GPU parity tests.  It also checks that an oversize request is
rejected before any GPU work.  The file is named to be collected last.
"""
import math

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


def _reference(torch, s, pos):
    """Pair forces, energy and virial through relres_compute (FP64 context,
    no bonded terms in the topology)."""
    topo = R.make_topology(s.types, s.mass_by_type, s.excl, None)
    ctx = R.Context(R.params_for(s, R.RELRES_PREC_FP64), topo)
    p = torch.tensor(pos, dtype=torch.float64, device="cuda")
    ctx.build_neighbors(p, s.box)
    f = torch.empty_like(p)
    e = torch.zeros(4, dtype=torch.float64, device="cuda")
    w = torch.zeros(6, dtype=torch.float64, device="cuda")
    ctx.compute(p, f, e, w)
    torch.cuda.synchronize()
    out = f.cpu().numpy(), float(e[0] + e[1]), w.cpu().numpy()
    ctx.close()
    return out


def _static(torch, s, pos, params):
    dev = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    d_pos = dev(pos, torch.float64)
    d_type = dev(s.types, torch.int32)
    d_eo = dev(s.excl_off, torch.int32)
    d_ei = dev(s.excl_idx, torch.int32)
    f = torch.full_like(d_pos, float("nan"))
    e = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    w = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    R.relres_pair_forces_static(params, s.n_atoms, d_type, d_pos, s.box, f, e, w, d_eo, d_ei,
                                stream=stream if stream else None)
    torch.cuda.synchronize()
    return f.cpu().numpy(), float(e[0]), w.cpu().numpy()


def test_static_entry_matches_compute_on_two_calls(torch):
    s = S.propane()  # 648 atoms, L = 31.8 A: all ranges below L/2
    params = R.params_for(s, R.RELRES_PREC_FP64)
    rng = np.random.default_rng(4)
    configs = [s.pos, (s.pos + rng.normal(scale=0.05, size=s.pos.shape)) % s.box]
    for pos in configs:
        f_ref, e_ref, w_ref = _reference(torch, s, pos)
        f, e, w = _static(torch, s, pos, params)
        rms = math.sqrt((f_ref * f_ref).sum(1).mean())
        assert np.abs(f - f_ref).max() / rms <= 1e-10
        assert abs(e - e_ref) / abs(e_ref) <= 1e-10
        assert np.abs(w - w_ref).max() / np.abs(w_ref[:3]).max() <= 1e-10


def test_static_entry_rejects_oversize(torch):
    s = S.propane()
    params = R.params_for(s, R.RELRES_PREC_FP64)
    d = torch.zeros(3, dtype=torch.float64, device="cuda")
    t = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(R.RelresError) as ei:
        R.relres_pair_forces_static(params, R.RELRES_STATIC_MAX_ATOMS + 1, t, d, s.box, d)
    assert ei.value.status == 1
