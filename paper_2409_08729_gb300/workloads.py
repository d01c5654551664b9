"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

Only input generation lives here: no part of the evaluation method.  The
shapes follow the paper's workloads (uniform samples over (v, x) regions,
paper Sec. 5.1-5.2, and the Fig. 1 sweep of v = 2^0..2^10 with x ~ U[1, 100]).
"""
import numpy as np

SWEEP_ORDERS = tuple(float(2 ** k) for k in range(11))     # v = 2^0 .. 2^10


def sweep_pairs(n_per_v=10000, seed=0):
    """Fig. 1 shape: every order v in SWEEP_ORDERS with n_per_v arguments x ~ U[1, 100].

    Returns float64 arrays (v, x) of length 11 * n_per_v, grouped by order."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(1.0, 100.0, size=(len(SWEEP_ORDERS), n_per_v))
    v = np.repeat(np.asarray(SWEEP_ORDERS)[:, None], n_per_v, axis=1)
    return v.ravel(), x.ravel()


def sweep_device(n_per_v, seed, device):
    """Same sweep generated on the GPU with torch's Philox generator.

    Returns (x_all, v_mixed): x_all is [11 * n_per_v] grouped by order (block
    k belongs to SWEEP_ORDERS[k]); v_mixed assigns an order drawn uniformly
    from SWEEP_ORDERS to every argument, in random order, for the mixed-order
    launch."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    n = n_per_v * len(SWEEP_ORDERS)
    x_all = torch.empty(n, dtype=torch.float64, device=device)
    x_all.uniform_(1.0, 100.0, generator=g)
    orders = torch.tensor(SWEEP_ORDERS, dtype=torch.float64, device=device)
    idx = torch.randint(0, len(SWEEP_ORDERS), (n,), generator=g, device=device)
    return x_all, orders[idx]


def robust_pairs(n, seed=0, vmax=1e5, xmin=1e-6, xmax=1e5):
    """Robustness sweep: v log-uniform on [1e-6, vmax] with 1% exactly 0 and 1%
    exactly 1/2; x log-uniform on [xmin, xmax]."""
    rng = np.random.default_rng(seed)
    v = np.exp(rng.uniform(np.log(1e-6), np.log(vmax), n))
    x = np.exp(rng.uniform(np.log(xmin), np.log(xmax), n))
    k = rng.permutation(n)
    v[k[: n // 100]] = 0.0
    v[k[n // 100: n // 50]] = 0.5
    return v, x


def robust_device(n, seed, device, vmax=1e5, xmin=1e-6, xmax=1e5):
    """robust_pairs generated on the GPU (torch Philox): v log-uniform on
    [1e-6, vmax] with 1% exactly 0 and 1% exactly 1/2, x log-uniform on
    [xmin, xmax].  Returns float64 device tensors (v, x)."""
    import math
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    v = torch.empty(n, dtype=torch.float64, device=device)
    x = torch.empty(n, dtype=torch.float64, device=device)
    v.uniform_(math.log(1e-6), math.log(vmax), generator=g).exp_()
    x.uniform_(math.log(xmin), math.log(xmax), generator=g).exp_()
    u = torch.rand(n, dtype=torch.float64, device=device, generator=g)
    v[u < 0.01] = 0.0
    v[(u >= 0.01) & (u < 0.02)] = 0.5
    return v, x


def paper_regions(n, seed=0, which="small", kind="i"):
    """Paper Sec. 5.1 test regions: Small [0,150]^2; Large [150,1e4]^2 for I and
    [150,4000]^2 for K; uniform samples."""
    rng = np.random.default_rng(seed)
    if which == "small":
        lo, hi = 0.0, 150.0
    else:
        lo, hi = 150.0, (1e4 if kind == "i" else 4000.0)
    return rng.uniform(lo, hi, n), rng.uniform(lo, hi, n)


# Thresholds of the region table (paper Table "input ranges") and of the tight
# dispatch; used to place test points on both sides of every boundary.
PAPER_EDGES_X = (19.6931, 30.0, 35.9074, 59.6925, 84.4153, 274.2377, 1400.0)
PAPER_EDGES_V = (0.3, 0.46, 0.6, 0.7, 3.05, 3.1, 12.6964, 15.3919, 20.1534, 56.9971, 163.6993)
TIGHT_EDGES_X = (25.0, 30.0, 59.6925)
TIGHT_EDGES_V = (0.7, 13.6, 16.0)
# corners (x, v) of the wider mu_20 and U_13 ranges of log K and log I values
K_VALUE_CORNERS = ((18.5, 9.5), (20.0, 12.5), (22.0, 13.6), (19.0, 10.0), (14.0, 14.0))
I_VALUE_CORNERS = ((19.0, 4.5), (21.0, 7.5), (23.0, 9.5), (19.5, 10.0), (17.5, 12.0), (14.5, 14.0))


def boundary_pairs(seed=0, per_edge=24):
    """Pairs within +-1e-6 relative and +-1% of every region threshold."""
    rng = np.random.default_rng(seed)
    vs, xs = [], []
    for e in PAPER_EDGES_X + TIGHT_EDGES_X:
        for rel in (-1e-2, -1e-6, 0.0, 1e-6, 1e-2):
            xs.append(np.full(per_edge, e * (1 + rel)))
            vs.append(np.exp(rng.uniform(np.log(1e-3), np.log(200.0), per_edge)))
    for e in PAPER_EDGES_V + TIGHT_EDGES_V:
        for rel in (-1e-2, -1e-6, 0.0, 1e-6, 1e-2):
            vs.append(np.full(per_edge, e * (1 + rel)))
            xs.append(np.exp(rng.uniform(np.log(1e-3), np.log(2000.0), per_edge)))
    # the edges of the wider value ranges: x near each corner's x with v up to
    # just past its v, and v near its v with x up to 30
    for xe, ve in K_VALUE_CORNERS + I_VALUE_CORNERS:
        for rel in (-1e-2, -1e-6, 0.0, 1e-6, 1e-2):
            xs.append(np.full(per_edge, xe * (1 + rel)))
            vs.append(rng.uniform(0.0, ve * 1.02, per_edge))
            vs.append(np.full(per_edge, ve * (1 + rel)))
            xs.append(rng.uniform(xe * 0.98, 30.0, per_edge))
    # the curved mu_20 boundaries: paper (log v = 0.5113 log x + 0.7939) and tight (v^2 = 3.24 x)
    x = np.exp(rng.uniform(np.log(60.0), np.log(1e5), 200))
    for rel in (-1e-2, -1e-6, 1e-6, 1e-2):
        vs.append(np.exp(0.5113 * np.log(x) + 0.7939) * (1 + rel)); xs.append(x)
        vs.append(np.sqrt(3.24 * x) * (1 + rel)); xs.append(x)
    return np.concatenate(vs), np.concatenate(xs)


def edge_pairs():
    """Domain edges: zeros, infinities, NaN, negative order/argument, tiny and huge values."""
    inf, nan = np.inf, np.nan
    vals_v = [0.0, 0.5, 1.0, 2.5, 1e-300, 1e5, inf, nan, -1.0, -0.5]
    vals_x = [0.0, 1e-300, 1e-6, 1.0, 25.0, 30.0, 1e5, 1e300, inf, nan, -1.0]
    V, X = np.meshgrid(np.array(vals_v), np.array(vals_x))
    return V.ravel(), X.ravel()


def vmf_mean_resultant(d, kappa, n, seed=0, device="cuda", chunk=2048):
    """Mean resultant length R = |mean of n unit vectors| drawn from the von
    Mises-Fisher distribution on S^(d-1) with mean direction e_1.

    Synthetic stand-in for the l2-normalised image features of paper Sec. 6.3.
    The component w = mu^T x follows Wood's rejection sampler (Wood 1994,
    "Simulation of the von Mises Fisher distribution"); the tangent part is
    sqrt(1 - w^2) times a uniform direction orthogonal to e_1, drawn as a
    normalised Gaussian vector.  Only the running sums are kept, so d = 32768
    needs no n x d array.  Returns (R, mean of w)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    dm1 = float(d - 1)
    k = float(kappa)
    b = dm1 / (2.0 * k + np.sqrt(4.0 * k * k + dm1 * dm1))
    x0 = (1.0 - b) / (1.0 + b)
    c = k * x0 + dm1 * np.log(1.0 - x0 * x0)
    beta = torch.distributions.Beta(torch.tensor(dm1 / 2, dtype=torch.float64, device=device),
                                    torch.tensor(dm1 / 2, dtype=torch.float64, device=device))
    ws = []
    need = n
    torch.manual_seed(seed)   # Beta sampling draws from the default generator
    while need > 0:
        m = max(2 * need, 1024)
        z = beta.sample((m,))
        w = (1.0 - (1.0 + b) * z) / (1.0 - (1.0 - b) * z)
        u = torch.rand(m, dtype=torch.float64, device=device, generator=g)
        ok = k * w + dm1 * torch.log1p(-x0 * w) - c >= torch.log(u)
        w = w[ok][:need]
        ws.append(w)
        need -= w.numel()
    w = torch.cat(ws)
    tang = torch.zeros(d - 1, dtype=torch.float64, device=device)
    for s0 in range(0, n, chunk):
        wc = w[s0:s0 + chunk]
        xi = torch.randn(wc.numel(), d - 1, dtype=torch.float64, device=device, generator=g)
        xi = xi / xi.norm(dim=1, keepdim=True)
        tang += (torch.sqrt(torch.clamp(1.0 - wc * wc, min=0.0))[:, None] * xi).sum(dim=0)
    mean_w = w.mean()
    xbar_norm2 = mean_w * mean_w + (tang / n).pow(2).sum()
    return float(torch.sqrt(xbar_norm2)), float(mean_w)
