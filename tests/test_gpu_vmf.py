"""vMF log-normaliser and Newton fit of the concentration (paper Sec. 6.3)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_08729_gb300 import vmf
from paper_2409_08729_gb300.workloads import vmf_mean_resultant

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d", [3.0, 2048.0, 8192.0, 32768.0])
def test_log_c_against_oracle(cuda, d):
    kappa = np.exp(np.linspace(np.log(1e-3), np.log(10 * d), 500))
    got = vmf.log_c(d, torch.tensor(kappa, device=cuda)).cpu().numpy()
    ref = oracle.vmf_log_c(np.full_like(kappa, d), kappa)
    scale = np.maximum(np.abs(ref), np.maximum(1.0, d / 2 * np.abs(np.log(kappa))))
    assert np.max(np.abs(got - ref) / scale) <= 4e-15


def test_log_c_zero_limit(cuda):
    got = vmf.log_c(3.0, torch.tensor([0.0], dtype=torch.float64, device=cuda)).item()
    assert abs(got - (-np.log(4 * np.pi))) < 1e-15      # C_3(0) = 1/(4 pi)


@pytest.mark.parametrize("d", [2048, 8192, 32768])
def test_score_central_difference(cuda, d):
    """d/dk log C_d from the adjoint kernel vs a central difference of log C_d."""
    kappa = torch.tensor([d / 10.0, float(d), 10.0 * d], dtype=torch.float64, device=cuda)
    g = vmf.log_c(d, kappa, deriv=True)
    h = 1e-5 * kappa
    fd = (vmf.log_c(d, kappa + h) - vmf.log_c(d, kappa - h)) / (2 * h)
    assert torch.all((g - fd).abs() <= 1e-7 * g.abs() + 1e-9)


@pytest.mark.parametrize("d", [2048, 8192, 32768])
@pytest.mark.parametrize("ratio", [0.1, 1.0, 10.0])
def test_newton_fit(cuda, d, ratio):
    kappa_true = ratio * d
    R, _ = vmf_mean_resultant(d, kappa_true, 50000, seed=d + int(ratio * 10), device=cuda)
    fit = vmf.fit_kappa(d, R, device=cuda)
    k = fit["kappa"]
    # the solution satisfies A_d(k) = R to rounding
    A = vmf.mean_ratio(d, torch.tensor([k], dtype=torch.float64, device=cuda)).item()
    assert abs(A - R) <= 1e-13 * R
    # Sra's second iterate agrees with the converged fit (paper Sec. 6.3: ~1e-11)
    assert abs(fit["kappa2"] - k) <= 1e-9 * k
    # and the estimate is near the truth (sampling error ~ kappa / sqrt(n d))
    assert abs(k - kappa_true) <= 0.05 * kappa_true + 2.0
