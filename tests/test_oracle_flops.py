"""The operation counter behind the roofline's algorithmic flops per cell (oracle/flops.py):
one operation per output element of each elementwise arithmetic call, by kind, and data
movement (selections, shifts, indexing) not counted; and the count of one oracle step is
the figure the benchmark divides by."""
import torch

from oracle import flops as F


def test_counter_on_known_expressions():
    a, b, c = (torch.rand(7, 5, dtype=torch.float64) for _ in range(3))
    with F.CountOps() as k:
        d = a * b + c
        e = torch.sqrt(d) / (b + 1.0)
        f = torch.where(e > 0.5, e, a)          # one compare; the selection is data movement
        g = torch.roll(f, 1, 0)[1:, :]          # data movement only
        h = torch.maximum(g, -g)                # one negation (add) and one max (compare)
    n = a.numel()
    assert k.n["mul"] == n
    assert k.n["add"] == 2 * n + (n - 5)
    assert k.n["sqrt"] == n and k.n["div"] == n
    assert k.n["cmp"] == n + (n - 5)
    assert h.shape == (6, 5)


def test_step_count_is_the_benchmark_figure():
    import bench
    per = F.count_step()
    flops = per["total"] - per.get("cmp", 0.0)
    assert abs(flops - bench.FLOPS_PER_CELL) <= 0.5, per
