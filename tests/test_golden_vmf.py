"""The vMF concentration estimates printed in Sec. 6.3 (Table "vMF
results"), reproduced from the printed kappa0 alone.

kappa0 = R (p - R^2) / (1 - R^2) fixes the mean resultant length R of the
data set; from R, two Newton updates F(kappa) (Eq. "kappa estimates", with
A_p(kappa) = I_{p/2}(kappa) / I_{p/2-1}(kappa)) must land on the printed
kappa1 and kappa2, and the root of A_p(kappa) = R (the maximum of the
log-likelihood) on the printed gradient estimate.  The oracle supplies
A_p on the CPU; the CUDA path (d/dkappa log C_p) supplies it for the Newton
fit on the GPU.  Tolerances are the printed rounding: half a unit of the
last printed decimal of the compared value, plus the spread that half a
unit of the printed kappa0 causes through R.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "vmf_kappa_estimates.txt")


def _rows():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            p, gf, ge, k0, k1, k2, dec = line.split()
            rows.append((int(p), float(gf), float(ge), float(k0), float(k1), float(k2), int(dec)))
    return rows


def r_from_kappa0(p, k0):
    """Root in (0, 1) of R^3 - k0 R^2 - p R + k0 = 0."""
    roots = np.roots([1.0, -k0, -float(p), k0])
    r = [z.real for z in roots if abs(z.imag) < 1e-12 and 0.0 < z.real < 1.0]
    assert len(r) == 1
    return r[0]


def a_p(p, kappa):
    kappa = np.atleast_1d(np.asarray(kappa, dtype=np.float64))
    return np.exp(oracle.log_i(np.full_like(kappa, p / 2.0), kappa)
                  - oracle.log_i(np.full_like(kappa, p / 2.0 - 1.0), kappa))


def newton_update(p, kappa, R):
    a = a_p(p, kappa)[0]
    return kappa - (a - R) / (1.0 - a * a - (p - 1.0) / kappa * a)


def mle(p, R):
    """Root of A_p(kappa) = R by bisection (A_p increases in kappa)."""
    lo, hi = 1e-3 * p, 1e3 * p
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if a_p(p, mid)[0] < R:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _estimates(p, k0):
    R = r_from_kappa0(p, k0)
    k1 = newton_update(p, k0, R)
    k2 = newton_update(p, k1, R)
    return R, k1, k2, mle(p, R)


@pytest.mark.parametrize("row", _rows(), ids=lambda r: "p%d" % r[0])
def test_newton_updates_and_mle(row):
    p, _, grad_est, k0, k1_paper, k2_paper, dec = row
    half = 0.5 * 10.0 ** (-dec)
    _, k1, k2, km = _estimates(p, k0)
    # spread of the derived values when kappa0 moves by half a printed unit
    lo = _estimates(p, k0 - half)
    hi = _estimates(p, k0 + half)
    for got, paper, i in ((k1, k1_paper, 1), (k2, k2_paper, 2), (km, grad_est, 3)):
        spread = 0.5 * abs(hi[i] - lo[i])
        assert abs(got - paper) <= half + spread + 1e-9 * paper, (p, i, got, paper)


def test_updates_move_off_kappa0():
    """For p = 2048 the printed kappa0 and kappa2 differ by 29 printed units:
    a Newton step that did nothing (or went the wrong way) fails above."""
    p, _, _, k0, _, k2_paper, dec = _rows()[0]
    _, _, k2, _ = _estimates(p, k0)
    assert abs(k0 - k2_paper) > 20 * 10.0 ** (-dec)
    assert abs(k2 - k2_paper) < abs(k0 - k2_paper) / 10


@pytest.mark.gpu
@pytest.mark.parametrize("row", _rows(), ids=lambda r: "p%d" % r[0])
def test_gpu_newton_fit_matches_printed_estimates(cuda, row):
    """The CUDA path's Newton fit (A_p from d/dkappa log C_p) from the same R:
    its first two iterates are kappa1, kappa2, its limit the gradient estimate."""
    from paper_2409_08729_gb300 import vmf
    p, _, grad_est, k0, k1_paper, k2_paper, dec = row
    half = 0.5 * 10.0 ** (-dec)
    R = r_from_kappa0(p, k0)
    fit = vmf.fit_kappa(p, R, device=cuda)
    lo = _estimates(p, k0 - half)
    hi = _estimates(p, k0 + half)
    for got, paper, i in ((fit["kappa1"], k1_paper, 1), (fit["kappa2"], k2_paper, 2), (fit["kappa"], grad_est, 3)):
        assert abs(got - paper) <= half + 0.5 * abs(hi[i] - lo[i]) + 1e-9 * paper, (p, i, got, paper)
    assert abs(fit["kappa"] - mle(p, R)) <= 1e-11 * fit["kappa"]
