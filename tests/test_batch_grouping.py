"""paper_1308_4605_gb300.batch.StackedBatch on CPU: problems are grouped by
grid (cells, boundary codes, spacing, theta) into one stacked handle each, in
the order of first appearance, and the solutions and records come back in
the problems' order.  The C calls are replaced by fakes (no GPU)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if not os.path.exists(os.path.join(ROOT, "paper_1308_4605_gb300", "libstokes_gb300.so")):
    pytest.skip("library not built", allow_module_level=True)
torch = pytest.importorskip("torch")
sys.path.insert(0, ROOT)
from paper_1308_4605_gb300 import batch  # noqa: E402


class _FakeSolver:
    made = []

    def __init__(self, dim, n, bc, h, count=None):
        self.dim, self.n, self.bc, self.h, self.count = dim, tuple(n), tuple(bc), h, count
        self.handle = object()
        self.coef = None
        _FakeSolver.made.append(self)

    def face_shape(self, a):
        nx, ny = self.n
        walls = self.bc[2 * a] != 0
        ext = [nx, ny]
        if walls:
            ext[a] += 1
        return (self.count, ext[1], ext[0])

    def cell_shape(self):
        return (self.count, self.n[1], self.n[0])

    def set_coefficients(self, rho, mu, theta):
        self.coef = (rho.clone(), mu.clone(), theta)

    def zeros(self, device="cpu"):
        return [torch.zeros(self.face_shape(a), dtype=torch.float64) for a in range(2)], \
            torch.zeros(self.cell_shape(), dtype=torch.float64)

    def instance_info(self, k):
        return {"instance": k, "solver": _FakeSolver.made.index(self)}

    def close(self):
        pass


@pytest.fixture
def fakes(monkeypatch):
    _FakeSolver.made = []
    calls = []

    def solve_batched(hs, p, bu, bp, xu, xp):
        calls.append(len(hs))
        for g in range(len(hs)):          # x = b, so the routing can be checked
            for a in range(2):
                xu[g][a].copy_(bu[g][a])
            xp[g].copy_(bp[g])
        return []

    monkeypatch.setattr(batch.S, "StokesSolver", _FakeSolver)
    monkeypatch.setattr(batch.S, "stk_solve_batched", solve_batched)
    return calls


def _problem(n, bc, h=1.0, theta=1.0, tag=0.0):
    nx, ny = n
    return {"n": n, "bc": bc, "h": h, "theta": theta,
            "rho": torch.full((1, ny, nx), 1.0 + tag, dtype=torch.float64),
            "mu": torch.full((1, ny, nx), 2.0 + tag, dtype=torch.float64)}


def test_grouping_and_order(fakes):
    P, W = (0,) * 4, (1,) * 4
    probs = [_problem((8, 8), P, tag=0), _problem((16, 8), P, tag=1), _problem((8, 8), P, tag=2),
             _problem((8, 8), W, tag=3), _problem((8, 8), P, theta=0.5, tag=4), _problem((16, 8), P, tag=5)]
    sb = batch.StackedBatch(probs)
    assert [idx for idx, _ in sb.groups] == [[0, 2], [1, 5], [3], [4]]
    counts = [sv.count for sv in _FakeSolver.made]
    assert counts == [2, 2, 1, 1]
    # each group's coefficients stacked in order
    rho0 = _FakeSolver.made[0].coef[0]
    assert rho0.shape == (2, 8, 8) and float(rho0[0, 0, 0]) == 1.0 and float(rho0[1, 0, 0]) == 3.0
    assert _FakeSolver.made[3].coef[2] == 0.5
    bus, bps = [], []
    for i, p in enumerate(probs):
        nx, ny = p["n"]
        walls = p["bc"][0] != 0
        bus.append([torch.full((ny, nx + (1 if walls else 0)), 10.0 * i, dtype=torch.float64),
                    torch.full((ny + (1 if walls else 0), nx), 10.0 * i + 1, dtype=torch.float64)])
        bps.append(torch.full((ny, nx), 10.0 * i + 2, dtype=torch.float64))
    xu, xp, infos = sb.solve(bus, bps, precond=2)
    assert fakes == [4]                   # one batched call for all groups
    for i in range(len(probs)):
        assert float(xu[i][0].reshape(-1)[0]) == 10.0 * i
        assert float(xu[i][1].reshape(-1)[0]) == 10.0 * i + 1
        assert float(xp[i].reshape(-1)[0]) == 10.0 * i + 2
    assert infos[2] == {"instance": 1, "solver": 0} and infos[5] == {"instance": 1, "solver": 1}
