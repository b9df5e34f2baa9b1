"""Whole-output comparison of two device arrays, for the full-size parity
tests (imported by them; collects no tests)."""


def max_abs_diff(a, b, chunk=1 << 28):
    """max |a - b| in FP64 over entries where neither is NaN, and whether
    the NaN patterns differ; a and b are flat device tensors of equal
    length, scanned in chunks so that the temporaries stay small."""
    import torch
    worst, differs = 0.0, False
    for c0 in range(0, a.numel(), chunk):
        x = a[c0:c0 + chunk].double()
        y = b[c0:c0 + chunk].double()
        nx, ny = torch.isnan(x), torch.isnan(y)
        differs |= bool((nx != ny).any().item())
        d = torch.where(nx | ny, torch.zeros_like(x), (x - y).abs())
        worst = max(worst, float(d.max().item()))
    return worst, differs
