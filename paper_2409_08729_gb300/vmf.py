"""von Mises-Fisher concentration fitting on the GPU library (paper Sec. 6.3).

log C_d(k) = (d/2 - 1) log k - (d/2) log 2pi - log I_{d/2-1}(k) and its
derivative come from logbessel_vmf_log_c; the score of the log-likelihood
logLik(k) = log C_d(k) + k R (R = mean resultant length, mu at its estimate
xbar / R, Eq. "mean direction estimate") is R - A_d(k) with
A_d(k) = I_{d/2}(k) / I_{d/2-1}(k) = -d/dk log C_d(k), evaluated by the
hand-written adjoint kernel.  Newton's method on A_d(k) = R uses
A_d'(k) = 1 - A_d^2 - (d-1) A_d / k; started from Sra's estimate
k_0 = R (d - R^2) / (1 - R^2), its first two iterates are Sra's k_1 and k_2
(Eq. "kappa estimates").
"""
import math

import torch

from . import _binding as B


def log_c(d, kappa, deriv=False):
    """log C_d(kappa) (deriv=False) or d/dkappa log C_d (deriv=True) for a CUDA tensor kappa."""
    if not isinstance(kappa, torch.Tensor) or kappa.device.type != "cuda":
        raise ValueError("kappa must be a CUDA tensor")
    k = kappa.to(torch.float64).contiguous()
    out = torch.empty_like(k)
    with torch.cuda.device(k.device):
        B.check(B.lib().logbessel_vmf_log_c(B.LB_F64, float(d), k.data_ptr(), out.data_ptr(), k.numel(),
                                            1 if deriv else 0, torch.cuda.current_stream(k.device).cuda_stream))
    return out


def mean_ratio(d, kappa):
    """A_d(kappa) = I_{d/2}(kappa) / I_{d/2-1}(kappa)."""
    return -log_c(d, kappa, deriv=True)


def sra_kappa0(d, R):
    return R * (d - R * R) / (1.0 - R * R)


def fit_kappa(d, R, device="cuda", tol=1e-15, max_iter=50):
    """Maximum-likelihood concentration for mean resultant length R in dimension d.

    Returns dict(kappa, iterations, kappa0, kappa1, kappa2, history)."""
    k = torch.tensor([sra_kappa0(d, R)], dtype=torch.float64, device=device)
    hist = [float(k)]
    prev = math.inf
    for it in range(max_iter):
        A = mean_ratio(d, k)
        dA = 1.0 - A * A - (d - 1.0) * A / k
        step = (A - R) / dA
        s = abs(float(step))
        # Newton's steps shrink quadratically until A_d's rounding; a step no
        # smaller than the one before means that floor is reached (iterates
        # 2 and on: kappa_1 and kappa_2 are always formed)
        if it >= 2 and s >= prev:
            break
        k = k - step
        hist.append(float(k))
        if s <= tol * abs(float(k)):
            break
        prev = s
    return {"kappa": hist[-1], "iterations": len(hist) - 1, "kappa0": hist[0],
            "kappa1": hist[1] if len(hist) > 1 else math.nan,
            "kappa2": hist[2] if len(hist) > 2 else math.nan, "history": hist}


def log_likelihood(d, kappa, R):
    """Mean log-likelihood log C_d(kappa) + kappa R at the estimated mean direction."""
    return log_c(d, kappa) + kappa * R
