"""Algorithmic operation count of one oracle step per cell.  TEST INFRASTRUCTURE ONLY.

Runs oracle.mhd.step under a torch function mode that counts, for every elementwise
arithmetic operation, one operation per output element, split by kind.  The oracle does
each stage once per cell on whole arrays (one flux per face, one EMF per edge), so the
count divided by the number of cells it ran on is the scheme's operation count per
cell-update.  Selections (torch.where), shifts (torch.roll), copies and indexing are
data movement and are not counted.  Run:  python -m oracle.flops
"""
from __future__ import annotations

import collections

import torch
from torch.overrides import TorchFunctionMode

KINDS = {
    "add": "add", "__add__": "add", "__radd__": "add", "__iadd__": "add",
    "sub": "add", "__sub__": "add", "__rsub__": "add", "__isub__": "add",
    "neg": "add", "__neg__": "add",
    "mul": "mul", "__mul__": "mul", "__rmul__": "mul", "__imul__": "mul",
    "div": "div", "__truediv__": "div", "__rtruediv__": "div", "true_divide": "div",
    "sqrt": "sqrt",
    "abs": "cmp", "__abs__": "cmp",
    "ge": "cmp", "__ge__": "cmp", "le": "cmp", "__le__": "cmp", "gt": "cmp", "__gt__": "cmp",
    "lt": "cmp", "__lt__": "cmp", "maximum": "cmp", "minimum": "cmp", "sign": "cmp",
    "__pow__": "mul", "pow": "mul",
}


class CountOps(TorchFunctionMode):
    def __init__(self):
        super().__init__()
        self.n = collections.Counter()

    def __torch_function__(self, func, types, args=(), kwargs=None):
        out = func(*args, **(kwargs or {}))
        name = getattr(func, "__name__", "")
        kind = KINDS.get(name)
        if kind is not None and isinstance(out, torch.Tensor):
            self.n[kind] += out.numel()
        return out


def count_step(n=32, gamma=5.0 / 3.0):
    """Operations per padded cell of one 3D step on an n^3 patch (guard 3), by kind."""
    from oracle import mhd
    g = 3
    N = n + 2 * g
    torch.manual_seed(0)
    U = torch.empty(1, 8, N, N, N, dtype=torch.float64)
    U[:, 0] = 1.0 + 0.1 * torch.rand(N, N, N)
    U[:, 1:4] = 0.1 * torch.randn(3, N, N, N)
    U[:, 5:8] = 0.1 * torch.randn(3, N, N, N)
    U[:, 4] = 3.0
    with CountOps() as c:
        mhd.step(U, 1e-3, [True, True, True], [1.0 / 64] * 3, gamma)
    cells = N ** 3
    per = {k: v / cells for k, v in c.n.items()}
    per["total"] = sum(per.values())
    return per


if __name__ == "__main__":
    r = count_step()
    print({k: round(v, 1) for k, v in sorted(r.items())})
