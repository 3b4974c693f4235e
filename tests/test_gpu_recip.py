"""The reciprocals the pair kernels use instead of correctly rounded division
and square root, held to their error bounds against exact values (host FP64 /
long double): FP32 1/x (hardware estimate plus one Newton-Raphson step) within
one ulp of the correctly rounded result, FP64 1/x and 1/sqrt(x) (FP32 estimate
plus one FP64 Newton-Raphson step) within 2e-13 relative."""
import numpy as np
import pytest

from paper_2104_10231_gb300 import relres as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T

    assert T.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2104_10231_gb300.build import build_library

    build_library()
    R.load()
    return T


def _inputs():
    rng = np.random.default_rng(17)
    # squared distances of the pair kernels (1e-2 .. 1e3 A^2) and a wide sweep
    x = np.concatenate([10.0 ** rng.uniform(-2.0, 3.0, 200_000), 10.0 ** rng.uniform(-30.0, 30.0, 50_000),
                        np.array([1.0, 2.0, 3.0, 7.0, 36.0, 49.0, 196.0, 0.5, 0.25, 1e-3])])
    # FP32 inputs exactly (the FP32 path sees float(x)); FP64 inputs as drawn
    return x


def test_recip_error_bounds(torch):
    x = _inputs()
    d_x = torch.tensor(x, dtype=torch.float64, device="cuda")
    o32 = torch.empty(len(x), dtype=torch.float32, device="cuda")
    o64 = torch.empty(2 * len(x), dtype=torch.float64, device="cuda")
    R.relres_eval_recip(d_x, o32, o64)
    o32 = o32.cpu().numpy()
    o64 = o64.cpu().numpy()
    # FP32: against the correctly rounded reciprocal of float(x); results in
    # the normal range only (smaller ones are flushed to 0 by design)
    xf = x.astype(np.float32)
    ref32 = (1.0 / xf.astype(np.float64)).astype(np.float32)
    normal = (np.abs(ref32) >= np.finfo(np.float32).tiny) & np.isfinite(ref32)
    ulp = np.spacing(ref32[normal])
    err_ulp = np.abs(o32[normal].astype(np.float64) - ref32[normal].astype(np.float64)) / ulp
    print(f"FP32 1/x: max {err_ulp.max():.2f} ulp, {np.mean(err_ulp > 0):.4f} of results off by one")
    assert err_ulp.max() <= 1.0
    assert np.all(o32[~normal & np.isfinite(ref32) & (xf > 1)] == 0.0)
    # FP64: exact values in long double where the platform has them, else FP64
    xl = x.astype(np.longdouble)
    r64 = (1 / xl).astype(np.float64)
    rs64 = (1 / np.sqrt(xl)).astype(np.float64)
    in32 = (x > 1e-37) & (x < 1e37)  # the FP32 estimate exists
    rel = np.abs(o64[: len(x)][in32] - r64[in32]) / r64[in32]
    rel_s = np.abs(o64[len(x):][in32] - rs64[in32]) / rs64[in32]
    print(f"FP64 1/x: max rel {rel.max():.2e}; 1/sqrt(x): max rel {rel_s.max():.2e}")
    assert rel.max() < 2e-13
    assert rel_s.max() < 2e-13


def test_recip_rejects_bad_arguments(torch):
    with pytest.raises(R.RelresError):
        R.load()
        R._check(R.load().relres_eval_recip(None, None, None, 4, None))
    assert R.load().relres_eval_recip(None, None, None, 0, None) == R.RELRES_OK
