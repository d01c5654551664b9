"""Table-driven exp/log of the kernels against the double-double oracle and
against CUDA's exp/log (ulp distances)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_08729_gb300 import _binding as B

pytestmark = pytest.mark.gpu


def _eval(which, a, dev):
    t = torch.tensor(a, dtype=torch.float64, device=dev)
    out = torch.empty_like(t)
    B.check(B.lib().logbessel_math_eval(which, t.data_ptr(), out.data_ptr(), t.numel(),
                                        torch.cuda.current_stream(dev).cuda_stream))
    return out.cpu().numpy()


def _ulps(a, b):
    ia = a.view(np.int64).astype(object)
    ib = b.view(np.int64).astype(object)
    return np.array([abs(int(x) - int(y)) for x, y in zip(ia, ib)])


def _ref(fn, a):
    out = np.empty_like(a)
    for i, v in enumerate(a):
        h, l = fn(float(v))
        out[i] = h + l
    return out


def test_exp(cuda):
    rng = np.random.default_rng(1)
    a = np.concatenate([rng.uniform(-707, 707, 4000), rng.uniform(-1, 1, 2000), rng.uniform(-1e-3, 1e-3, 500),
                        [0.0, -0.0, 1e-300, -745.0, 709.7, 800.0, -800.0, np.inf, -np.inf, np.nan]])
    got = _eval(0, a, cuda)
    lib = _eval(2, a, cuda)
    fin = np.abs(a) < 700
    ref = _ref(oracle.dd_exp, a[fin])
    u = _ulps(got[fin], ref)
    assert u.max() <= 1, u.max()
    assert _ulps(got[fin], lib[fin]).max() <= 2
    # outside |y| < 708 the libm function is used: identical results
    fb = ~(np.abs(a) < 708)
    np.testing.assert_array_equal(got[fb], lib[fb])


def test_exp_term(cuda):
    """The exp of the quadrature terms (no low table part): within 2 ulp; y < -708 flushes to 0."""
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.uniform(-707, 707, 4000), rng.uniform(-40, 0, 2000), rng.uniform(-1e-3, 1e-3, 500),
                        [0.0, -0.0, 1e-300]])
    got = _eval(6, a, cuda)
    ref = _ref(oracle.dd_exp, a)
    assert _ulps(got, ref).max() <= 2
    np.testing.assert_array_equal(_eval(6, np.array([-708.5, -745.0, -1e300]), cuda), 0.0)


def test_log(cuda):
    rng = np.random.default_rng(2)
    a = np.concatenate([np.exp(rng.uniform(-700, 700, 4000)), rng.uniform(0.5, 2.0, 3000),
                        1.0 + rng.uniform(-1e-6, 1e-6, 500), [1.0, 2.0, 0.5, np.sqrt(2.0), 1.4142135, 1.4142136]])
    got = _eval(1, a, cuda)
    lib = _eval(3, a, cuda)
    ref = _ref(oracle.dd_log, a)
    u = _ulps(got, ref)
    big = np.abs(ref) > 1e-300
    assert u[big].max() <= 1, u[big].max()
    assert _ulps(got, lib).max() <= 2
    assert np.max(np.abs(got - ref)) <= 2.3e-16 * np.maximum(1.0, np.abs(ref)).max()


def test_log_fallbacks(cuda):
    a = np.array([0.0, -1.0, 5e-324, 1e-310, np.inf, np.nan])
    got = _eval(1, a, cuda)
    lib = _eval(3, a, cuda)
    np.testing.assert_array_equal(got, lib)


def test_integer_pipe_exp_log_bit_exact(cuda):
    """The integer-pipe exp and log on the GPU give the same bits as their host
    build (which the CPU suite holds to 0.51 ulp of the oracle)."""
    from intmath_host import ix_exp, ix_log
    rng = np.random.default_rng(21)
    y = np.concatenate([rng.uniform(-708, 708, 50000), rng.uniform(-1, 1, 20000), -np.exp(rng.uniform(-60, 6, 20000)),
                        [0.0, -0.0, 1e-300, -708.5, 708.5, 700.0]])
    np.testing.assert_array_equal(_eval(7, y, cuda), ix_exp(y))
    z = np.concatenate([np.exp(rng.uniform(-708, 709, 50000)), rng.uniform(0.5, 2.0, 20000),
                        1.0 + rng.uniform(-1e-9, 1e-9, 5000), [1.0, 2.0, 0.5, np.e, 1e-300, 1e300]])
    np.testing.assert_array_equal(_eval(8, z, cuda), ix_log(z))


def test_integer_pipe_rcp_rsqrt_bit_exact(cuda):
    """The integer-pipe reciprocal and 1/sqrt on the GPU give the same bits as
    their host build (held to 0.51 / 0.52 ulp on the CPU)."""
    from intmath_host import ix_rcp, ix_rsqrt
    rng = np.random.default_rng(22)
    z = np.concatenate([np.exp(rng.uniform(-708, 708, 50000)), rng.uniform(1.0, 2.0, 20000),
                        1.0 + rng.uniform(0, 1e-9, 5000), 2.0 ** np.arange(-1022, 1023, 7),
                        [1.0, 2.0, 0.5, 3.0, 1e-300, 1e300, 2.0 ** 1023, 0.0, np.inf]])
    np.testing.assert_array_equal(_eval(9, z, cuda), ix_rcp(z))
    np.testing.assert_array_equal(_eval(10, z, cuda), ix_rsqrt(z))


def test_fixed_point_node_functions_bit_equal_to_host(cuda):
    """The Q53 log and the Q58 exponential of a Q53 shift (the K integral's
    node functions) give the same bits on the GPU as in the host build that
    tests/test_intmath.py checks against exact references."""
    from intmath_host import ix_exp_q58_fx, ix_log_q53
    rng = np.random.default_rng(12)
    z = np.concatenate([np.exp(rng.uniform(-700, 700, 3000)), rng.uniform(1e-3, 200.0, 3000),
                        1.0 + np.arange(512) / 512.0, [0.0, -1.0, 5e-324, np.inf, np.nan]])
    got = _eval(11, z, cuda).view(np.int64)
    assert np.array_equal(got, ix_log_q53(z))
    d = np.concatenate([-rng.integers(0, 42 * 2 ** 53, 5000, dtype=np.int64), np.array([0, -1, -(2 ** 62)], dtype=np.int64)])
    got = _eval(12, d.view(np.float64), cuda).view(np.uint64)
    assert np.array_equal(got, ix_exp_q58_fx(d))
