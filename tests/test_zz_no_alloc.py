"""relres_pair_forces_static: the entry point that allocates no device memory.

It exists for callers that cannot let a library allocate device memory (a host
program that owns the GPU memory budget through its own allocator, or a loop
where cudaMalloc's device synchronisation is not allowed).  Its scratch lives
in one static device array shared by every call, so consecutive calls must not
see each other's leftovers.  These tests call it through the C ABI and compare
every result with the FP64 oracle's all-pairs sum of Eq. 20 (Section 2.5),
within the FP64 tolerances of the other GPU parity tests:

- two calls in a row that differ in everything the array holds: a
  16 000-atom liquid with Eq. 19 in full (63 of the 64 partial-sum rows), then
  the 648-atom propane-like liquid with Gamma_{c-} = 0 ("shift no", 3 rows), so
  a stale type-pair table or stale partial sums of the first call would show;
- an atom type out of range, which must give NaN (and no table read with it),
  followed by a valid call that is unaffected;
- an oversize request, rejected before any GPU work.

The file is named to be collected last.
"""
import math

import numpy as np
import pytest

from paper_2104_10231_gb300 import relres as R
from paper_2104_10231_gb300 import systems as S

pytestmark = pytest.mark.gpu

TOL = 1e-10  # FP64 all-pairs sums against the FP64 oracle: rounding order only


@pytest.fixture(scope="module")
def torch():
    import torch as T

    assert T.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2104_10231_gb300.build import build_library

    build_library()
    R.load()
    return T


def _oracle(s, pos, shift):
    from oracle import core as O

    return O.pair_forces(pos, s.box, s.types, O.table_for(s, shift=shift), s.n_types, s.excl)


def _static(torch, s, pos, params, types=None):
    dev = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    d_pos = dev(pos, torch.float64)
    d_type = dev(s.types if types is None else types, torch.int32)
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


def _check(got, ref):
    f, e, w = got
    f_ref, e_ref, w_ref = ref
    rms = math.sqrt((f_ref * f_ref).sum(1).mean())
    assert np.abs(f - f_ref).max() / rms <= TOL
    assert abs(e - e_ref) / abs(e_ref) <= TOL
    assert np.abs(w - w_ref).max() / np.abs(w_ref[:3]).max() <= TOL


def test_static_entry_matches_oracle_on_two_different_calls(torch):
    big = S.neopentane(n_mol=3200, seed=77)  # 16 000 atoms, L = 87 A: near RELRES_STATIC_MAX_ATOMS
    assert 15000 < big.n_atoms <= R.RELRES_STATIC_MAX_ATOMS
    small = S.propane()  # 648 atoms, L = 31.8 A
    calls = [(big, big.pos, True), (small, small.pos, False)]
    for s, pos, shift in calls:
        got = _static(torch, s, pos, R.params_for(s, R.RELRES_PREC_FP64, shift=shift))
        _check(got, _oracle(s, pos, shift))


def test_static_entry_flags_out_of_range_types(torch):
    s = S.propane()
    params = R.params_for(s, R.RELRES_PREC_FP64)
    bad = np.array(s.types, dtype=np.int32)
    bad[5] = s.n_types + 3
    bad[17] = -1
    f, e, w = _static(torch, s, s.pos, params, types=bad)
    assert math.isnan(e) and np.isnan(w).all()
    assert np.isnan(f[5]).all() and np.isnan(f[17]).all()
    # the flag does not outlive the call
    _check(_static(torch, s, s.pos, params), _oracle(s, s.pos, True))


def test_static_entry_rejects_oversize(torch):
    s = S.propane()
    params = R.params_for(s, R.RELRES_PREC_FP64)
    d = torch.zeros(3, dtype=torch.float64, device="cuda")
    t = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(R.RelresError) as ei:
        R.relres_pair_forces_static(params, R.RELRES_STATIC_MAX_ATOMS + 1, t, d, s.box, d)
    assert ei.value.status == 1
