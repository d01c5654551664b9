"""Algorithmic work of the evaluation kernels, for the roofline: a fixed table.

Work is the number of FP64 arithmetic operations the method performs, one
per add, subtract, multiply, fused multiply-add or compare: each is one
issue of the FP64 pipe, whose peak is 2 operations per SM per clock
(152 SMs x 2 x 2.07 GHz = 629.3 G op/s on GB300).  Calls to transcendental
and other library functions (log, exp, reciprocal, 1/sqrt, lgamma) are
counted by name and NOT priced: how a call is evaluated (here mostly on the
integer pipes) is the implementation's business, so the FP64 operations of
the method are a lower bound on the FP64-pipe work of any implementation,
and frac = (table operations) / (time x peak) is the share of the FP64
pipe's capacity that did the method's own arithmetic.

Per pair, in tight mode, with n the pair's own term count (not the warp's):

  region          general pair                  one order for the whole call
  mu_K (n terms)  3n + 7     rcp, log           n + 6     rcp, log
  U_K             K(K+1)/2 + K + 14             3K + 12
                  rcp, rsqrt, 3 log             rsqrt, 3 log
  series (n)      4n + 7     rcp, 2 log, lgamma 2n + 5    2 log
  K integral      8 per g node, 6 per h node,   7 per g node, 6 per h node,
                  11 per pair                   10 per pair
                  exp: 2 per g node + 1 per h node (1 + 1 for one order),
                  log: 1 per node + 3 per pair, rcp, lgamma (per pair)

mu_K: per term a_k = (mu - (2k-1)^2)/k (one fma with constants), times
+-1/(8x), Horner step (fma); per pair mu = 4v^2, 8x, S^2 and two scalings,
the final fma.  With one order the coefficients a_k (s/8)^k are the call's:
one fma per term.
U_K: x' = x/v, 1 + x'^2, r = r^2 t, t^2, +-t/v, the Debye polynomial P_k of
degree k in t^2 by Horner (k fmas, k = 1..K), Horner over k in q (K fmas),
eta (3), w = S^2 t / v (3), scaling, halving, final fma.  With one order the
sum is one polynomial of degree 3K in t (3K fmas).
Series (the linear fraction of the reading of Eq. "log Iv" with a_0 as
shift): per term d_k = k(k+v) (fma), A <- d B + y A (mul, fma), B <- d B;
per pair y = x^2/4, A/B, v+1, x/2, two combining operations.  With one
order the ratios 1/(k(k+v)) are the call's: per term y r_k and one fma.
K integral (Eq. "log Kv integral", Gauss nodes): a g node forms s = u^beta
(beta log u, exp), 2x + s, log, c + log beta, fma, - s; an h node s + 2x,
log, y + ., fma; every node then takes part in the log-sum-exp of Eq. "log
sum trick" (compare for the maximum, L - m, exp, add).  Per pair: v - 1/2,
2x, beta (2v + 1 and a scaling, a reciprocal), v + 1/2 for lgamma, the
prefactor (fma and two subtractions), the final logarithm and two additions.
With one order u^beta and lgamma(v + 1/2) are the call's.
"""
import numpy as np

PEAK_FP64_OPS = 152 * 2 * 2.07e9       # FP64-pipe operations per second: SMs x DFMA/clk x max clock
PEAK_FP32_OPS = 152 * 128 * 2.07e9     # FP32-pipe operations per second: SMs x FP32 lanes x max clock

REGION_NAMES = {0: "mu20", 1: "u13", 2: "fallback", 4: "mu3", 5: "u4", 6: "u6", 7: "u9"}
REGION_K = {0: 20, 1: 13, 4: 3, 5: 4, 6: 6, 7: 9}      # expansion terms of each region


def mu_terms(v, x, K=20, eps=1.4e-17):
    """Terms the mu_K expression needs for each pair: the first k after which
    a term falls below eps (2^-56: the FP64 kernels' single-precision
    estimate; the FP32 form counts to 2^-24)."""
    v = np.asarray(v, dtype=np.float32)
    x = np.asarray(x, dtype=np.float32)
    mu = np.float32(4.0) * v * v
    inv8x = np.float32(1.0) / (np.float32(8.0) * x)
    t = np.ones_like(x)
    n = np.full(x.shape, K, dtype=np.int64)
    done = np.zeros(x.shape, dtype=bool)
    for k in range(1, K + 1):
        t = np.where(done, t, t * (mu - np.float32((2 * k - 1) ** 2)) * inv8x / np.float32(k))
        hit = ~done & (np.abs(t) < eps)
        n = np.where(hit, k, n)
        done |= hit
    return n


def series_terms(v, x, eps=1.4e-17):
    """Terms the power series sums for each pair (the kernels' single-precision
    estimate: past the peak index, until a term is below eps of the sum;
    2^-56 in FP64, 1.5e-8 in the FP32 form)."""
    v = np.asarray(v, dtype=np.float32)
    x = np.asarray(x, dtype=np.float32)
    y = np.float32(0.25) * x * x
    kpk = np.float32(0.5) * (np.sqrt(x * x + v * v) - v)
    term = np.ones_like(x)
    T = np.zeros_like(x)
    n = np.ones(x.shape, dtype=np.int64)
    done = np.zeros(x.shape, dtype=bool)
    for k in range(1, 91):
        active = ~done
        if not active.any():
            break
        term = np.where(active, term * y / (np.float32(k) * (np.float32(k) + v)), term)
        T = np.where(active, T + term, T)
        n = np.where(active, k, n)
        done |= active & (np.float32(k) > kpk) & (term <= np.float32(eps) * (1 + T))
    return n


def kint_nodes(v, x, one_slot=True, low_slot=True):
    """g and h nodes of the tight K-integral rule of each pair (values; |v|
    given).  The split g rule (v < 0.4, x < 1e-3) has 64 + 32 + 32 nodes,
    plus 32 more below x ~ 4e-21; 1.2 < v <= 5 takes 24 g + 40 h nodes;
    2 <= v <= 16.5 the one-slot rules, 22 + 10 (v < 7) or 12 + 20, and
    0.9 <= v < 2 with x >= 0.8 the one-slot rule of 24 + 8 nodes (FP64 only:
    low_slot False for the FP32 form)."""
    v = np.asarray(v, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    split = np.where(np.log(128 * np.maximum(x, 1e-320)) + 40 < -4, 160, 128)
    ng = np.where((v >= 0.9) | (x >= 0.25), 32, np.where((v >= 0.4) | (x >= 1e-3), 64, split))
    nh = np.where(v <= 1.2, 32, np.where(v <= 5.0, 48, 32))
    packed = (v > 1.2) & (v <= 5.0)
    ng, nh = np.where(packed, 24, ng), np.where(packed, 40, nh)
    one = (v >= 2.0) & (v <= 16.5) & one_slot
    ng = np.where(one, np.where(v < 7.0, 22, 12), ng)
    nh = np.where(one, np.where(v < 7.0, 10, 20), nh)
    low = (v >= 0.9) & (v < 2.0) & (x >= 0.8) & one_slot & low_slot
    ng, nh = np.where(low, 24, ng), np.where(low, 8, nh)
    return ng, nh


def region_ops(region, v, x, shared=False, fp32=False):
    """Operations per pair of the per-thread expressions (tile kernel): FP64,
    or FP32 for the FP32-mixed form (term counts to single precision; its
    calls pass no order constants, so shared does not apply)."""
    shape = np.shape(x)
    shared = shared and not fp32
    if region in (0, 4):
        n = mu_terms(v, x, REGION_K[region], eps=6e-8 if fp32 else 1.4e-17)
        return (n + 6) if (shared and region == 0) else (3 * n + 7)
    if region in REGION_K:
        K = REGION_K[region]
        return np.full(shape, 3 * K + 12 if shared else K * (K + 1) // 2 + K + 14, dtype=np.int64)
    n = series_terms(v, x, eps=1.5e-8 if fp32 else 1.4e-17)
    return (2 * n + 5) if shared else (4 * n + 7)


def kint_ops(v, x, shared=False, fp32=False):
    """Operations per pair of the K integral (Gauss rules; the FP32 form takes
    the same rules, in single precision)."""
    ng, nh = kint_nodes(v, x, low_slot=not fp32)
    return ng * (7 if shared else 8) + nh * 6 + (10 if shared else 11)


def region_calls(region, shared=False):
    """Library calls per pair (named, not priced) of each expression."""
    if region in (0, 4):
        return {"rcp": 1, "log": 1}
    if region in REGION_K:
        return {"rsqrt": 1, "log": 3} if shared else {"rcp": 1, "rsqrt": 1, "log": 3}
    return {"log": 2} if shared else {"rcp": 1, "log": 2, "lgamma": 1}


def kint_calls(ng, nh, shared=False):
    calls = {"exp": (1 if shared else 2) * ng + nh, "log": ng + nh + 3}
    if not shared:
        calls.update(rcp=1, lgamma=1)
    return calls
