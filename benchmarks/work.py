"""Algorithmic work of a benchmark step from the fixed operation table
(optable.py): every call's pairs are classified on the GPU and counted per
region; the mean operations per pair of each region come from a random
sample of its pairs (term and node counts depend on the pair).  The result
is reported region by region, so the roofline figures can be recomputed by
hand as sum(pairs x mean operations) / (kernel time x peak)."""
import numpy as np
import torch

import paper_2409_08729_gb300 as lb

from . import optable as OT


def call_work(kind, v, x, fp32=False, sample=1 << 19, seed=0):
    """Work of one call: {"tiles": {region: [pairs, mean_ops]}, "kint": {...}}.
    v is a device tensor of one order (the call shares it) or one per pair."""
    shared = v.numel() == 1
    regs = lb.classify(kind, v, x).view(-1)
    n = regs.numel()
    counts = torch.bincount(regs.long(), minlength=8).cpu().numpy()
    g = torch.Generator(device=x.device)
    g.manual_seed(seed)
    pos = torch.randint(0, n, (min(sample, n),), generator=g, device=x.device)
    rs = regs[pos].cpu().numpy()
    xs = x.view(-1)[pos].double().cpu().numpy()
    vs = (v.view(-1)[pos] if not shared else v.view(-1).expand(n)[pos]).double().abs().cpu().numpy()
    out = {"tiles": {}, "kint": {}}
    for r, name in OT.REGION_NAMES.items():
        c = int(counts[r])
        if c == 0:
            continue
        sel = rs == r
        if not sel.any():                          # too rare to be sampled: count the pairs, price one
            sel = np.zeros_like(rs, dtype=bool)
        if kind == "k" and r == 2:
            ops = OT.kint_ops(vs[sel], xs[sel], shared, fp32) if sel.any() else np.array([0.0])
            out["kint"]["integral"] = [c, float(np.mean(ops))]
        else:
            ops = OT.region_ops(r, vs[sel], xs[sel], shared, fp32) if sel.any() else np.array([0.0])
            out["tiles"][name] = [c, float(np.mean(ops))]
    return out


def merge(total, part):
    """Accumulate call_work results: pairs add, mean operations weighted."""
    for kern, regs in part.items():
        dst = total.setdefault(kern, {})
        for name, (c, m) in regs.items():
            c0, m0 = dst.get(name, [0, 0.0])
            dst[name] = [c0 + c, (c0 * m0 + c * m) / (c0 + c)]
    return total


def ops_of(work, kern):
    return sum(c * m for c, m in work.get(kern, {}).values())
