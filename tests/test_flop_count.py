"""FP64 flops of one 2D sweep per interior node, counted on the PyTorch
restatement of the step (oracle/torch_ref.py, pinned to the C oracle), for the
roofline of the FP64 bench leg.

Every arithmetic op the restatement dispatches (add, sub, mul, div, sqrt,
1 - x) counts one flop per output element; sign changes, comparisons,
selections, abs and data movement count none.  An op whose operand is a whole
field of zeros (the zero components of the gravity source vector) is not part
of the method and is skipped.  Counts on nx x nz grids are differenced over
two widths and two heights, which cancels the plate rows and leaves the cost
of one interior node.  The formulas evaluate three differences per TVD
interface, of which two repeat a neighbouring interface's (2 x 4 = 8
subtractions): the distinct count drops them.  bench.py reports the FP64
leg's ALU fraction with the distinct counts.
"""
import pytest
import torch
from torch.utils._python_dispatch import TorchDispatchMode

import bench
from oracle.torch_ref import Model

FLOP_OPS = {"add", "sub", "mul", "div", "sqrt", "rsub"}
BINARY = {"add", "sub", "mul", "div", "rsub"}


class _Count(TorchDispatchMode):
    def __init__(self):
        super().__init__()
        self.by_op = {}

    def __torch_dispatch__(self, func, types, args=(), kwargs=None):
        out = func(*args, **(kwargs or {}))
        name = func.__name__.split(".")[0].rstrip("_")
        if name in FLOP_OPS:
            live = torch.ones(out.shape, dtype=torch.bool)
            if name in BINARY:
                for a in args[:2]:
                    a = torch.as_tensor(a)
                    z = (a == 0).flatten(1).all(1)[:, None, None] if a.dim() == 3 else (a == 0).all()
                    live &= ~torch.broadcast_to(z, out.shape)
            self.by_op[name] = self.by_op.get(name, 0) + int(live.sum())
        return out


def _count(nx, nz, direction):
    g = torch.Generator().manual_seed(1)
    m = Model(nx, nz)
    X = (torch.rand(4, nz, nx, dtype=torch.float64, generator=g) * 0.01 +
         torch.tensor([1.0, 0.01, 0.01, 15.0], dtype=torch.float64)[:, None, None])
    mu, kth = m.coefs(1e8)
    with _Count() as c:
        (m.sweep_z if direction == "z" else m.sweep_x)(X, 1e-4, mu, kth)
    return c.by_op


def flops_per_interior_node(direction):
    a, b, c, d = (_count(nx, nz, direction) for nx, nz in ((128, 66), (64, 66), (128, 34), (64, 34)))
    ops = set(a) | set(b) | set(c) | set(d)
    per = {k: (a.get(k, 0) - b.get(k, 0) - c.get(k, 0) + d.get(k, 0)) / (64 * 32) for k in ops}
    return per


@pytest.mark.parametrize("direction", ["z", "x"])
def test_bench_flop_counts_match_the_restatement(direction):
    per = flops_per_interior_node(direction)
    assert all(v == int(v) for v in per.values()), per  # data-independent
    total = int(sum(per.values()))
    assert per["div"] == 23 and per["sqrt"] == 1
    assert total == bench.FP64_FLOPS_FORMULA[direction]
    assert bench.FP64_FLOPS[direction] == total - 8
