"""The FP32 reciprocal of the collision's velocities against the exact quotient.

The FP32 kernels divide the momenta by rho through one reciprocal: the hardware's
approximate reciprocal r0 (at most one unit in the last place off) refined by one
Newton-Raphson step for 1/x, r = r0 + r0 (1 - x r0).  One step from a one-ulp start
leaves an error of the order of the start's square plus the final rounding, so every
result must lie within one ulp of 1/x (computed in FP64, exact to far below an FP32
ulp), and nearly all must be the correctly rounded quotient.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rcp(x):
    import torch
    from paper_1504_07034_gb300 import abi
    lib = abi.load()
    xd = torch.from_numpy(x).cuda()
    rd = torch.empty_like(xd)
    abi.check(lib.lbrs_selftest_rcp_f32(xd.data_ptr(), rd.data_ptr(), xd.numel(), None))
    torch.cuda.synchronize()
    return rd.cpu().numpy()


def _inputs():
    rng = np.random.default_rng(7)
    x = [np.exp(rng.uniform(np.log(1e-6), np.log(1e6), 1 << 20)),      # densities over 12 decades
         rng.uniform(0.1, 10.0, 1 << 20)]                               # the workloads' range
    p2 = np.float32(2.0) ** np.arange(-60, 61, dtype=np.float32)
    x.append(p2)                                                        # exact reciprocals
    x.append(np.nextafter(p2, np.float32(np.inf)))                      # just above a power of two
    x.append(np.nextafter(p2, np.float32(0)))                           # just below
    x.append(np.float32(1.0) + np.arange(1, 4097, dtype=np.float32) * np.finfo(np.float32).eps)
    return np.concatenate([np.asarray(v, dtype=np.float32) for v in x])


def test_reciprocal_within_one_ulp_of_the_quotient():
    x = _inputs()
    r = _rcp(x)
    exact = 1.0 / x.astype(np.float64)
    nearest = exact.astype(np.float32)
    ulp = np.spacing(np.abs(nearest)).astype(np.float64)
    err = np.abs(r.astype(np.float64) - exact) / ulp
    assert np.all(np.isfinite(r))
    assert err.max() <= 1.0, (x[err.argmax()], err.max())
    assert np.mean(r == nearest) >= 0.99
    p2 = (x == np.float32(2.0) ** np.round(np.log2(x)))
    assert np.array_equal(r[p2], nearest[p2])                           # powers of two: exact


def test_reciprocal_rejects_bad_arguments():
    from paper_1504_07034_gb300 import abi
    lib = abi.load()
    assert lib.lbrs_selftest_rcp_f32(None, None, -1, None) == abi.LBRS_EINVAL
    assert lib.lbrs_selftest_rcp_f32(None, None, 4, None) == abi.LBRS_EINVAL
    assert lib.lbrs_selftest_rcp_f32(None, None, 0, None) == 0
