"""Host logic of the warm-start pipeline (no GPU): the acceptance rule with
its cold fallback, the naive baselines and the parameter initialisation,
with the batched solver replaced by a stand-in."""

import numpy as np

from paper_2311_12180_gb300 import pdlp as P
from paper_2311_12180_gb300 import warmstart as W


class _LP:
    def __init__(self, i):
        self.i, self.n, self.m = i, 3, 2


class _FakeBatch:
    """Warm solves of odd-numbered LPs hit the iteration limit; cold solves
    always succeed in 100 iterations, warm ones in 40."""

    calls = []

    def __init__(self, lps):
        self.lps = lps

    def solve(self, tol, max_iter, x0=None, y0=None):
        _FakeBatch.calls.append((len(self.lps), x0 is not None, max_iter))
        k = len(self.lps)
        xs = [np.full(3, lp.i, float) for lp in self.lps]
        ys = [np.zeros(2) for _ in self.lps]
        if x0 is None:
            return xs, ys, np.zeros(k, np.int32), np.full(k, 100)
        st = np.array([P.ITER_LIMIT if lp.i % 2 else P.OPTIMAL for lp in self.lps], np.int32)
        return xs, ys, st, np.where(st == P.OPTIMAL, 40, max_iter)

    def close(self):
        pass


def test_fallback_resolves_failed_warm_starts_cold(monkeypatch):
    monkeypatch.setattr(P, "BatchSolver", _FakeBatch)
    _FakeBatch.calls = []
    r = W.solve_with_fallback(_LP, 5, 1e-6, lambda i: (np.zeros(3), np.zeros(2)), max_iter=500, chunk=2)
    assert r["fallbacks"] == 2
    assert np.all(r["status"] == P.OPTIMAL)
    assert list(r["iters"]) == [40, 600, 40, 600, 40]  # failed warm (500) + cold (100)
    # the cold re-solve covers exactly the two failed LPs, in one chunk
    assert (2, False, 500) in _FakeBatch.calls


def test_solve_many_chunks_and_hands_out_every_solution(monkeypatch):
    monkeypatch.setattr(P, "BatchSolver", _FakeBatch)
    got = {}
    st, it, _, _ = W.solve_many(_LP, 7, 1e-4, chunk=3, on_solution=lambda i, x, y: got.__setitem__(i, x[0]))
    assert sorted(got) == list(range(7)) and all(got[i] == i for i in got)
    assert np.all(st == P.OPTIMAL) and np.all(it == 100)


def test_baselines_and_init():
    T = np.array([[1.0, 2.0, 3.0], [3.0, 4.0, 5.0]])
    mx, my = W.mean_start(T, 2)
    assert np.array_equal(mx, [2.0, 3.0]) and np.array_equal(my, [4.0])
    idx = W.nearest_index(np.array([[0.0, 0.0], [10.0, 0.0]]), np.array([[9.0, 1.0], [-1.0, 0.5]]))
    assert list(idx) == [1, 0]
    p = W.init_params(4, 8, 3, seed=0)
    assert p.dtype == np.float32 and p.size == 4 * 8 + 8 + 8 * 8 + 8 + 8 * 3 + 3
    assert np.all(p[32:40] == 0) and np.abs(p[:32]).max() <= np.sqrt(6 / 4)
    assert np.array_equal(p, W.init_params(4, 8, 3, seed=0))


def test_leave_one_out_neighbour_and_residual_inputs():
    import numpy as np

    from paper_2311_12180_gb300 import warmstart as W

    rng = np.random.default_rng(4)
    X = rng.standard_normal((300, 5))
    nn = W.nearest_index(X, X, exclude_self=True, chunk=64)
    d = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d, np.inf)
    assert np.array_equal(nn, d.argmin(1))
    assert np.all(nn != np.arange(300))
    assert np.array_equal(W.nearest_index(X, X[:7]), np.arange(7))  # itself when not excluded
    R = W.residual_inputs(X[:3], X[nn[:3]])
    assert R.shape == (3, 10) and np.allclose(R[:, 5:], X[nn[:3]] - X[:3], atol=1e-6)
