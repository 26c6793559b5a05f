"""Learned warm starts for a parametric LP family (BF16 MLP on the GPU).

A family maps a latent parameter theta to an LP of fixed dimensions.  The
training targets are the solver's own solutions (x, y) of sampled members,
computed by the batched GPU solver; the network (pdlp.Mlp) is trained by the
library's kernels; its prediction for a new theta is passed to the solver as
the start point, which the first PDHG step projects onto X x Y.  A warm
start is accepted only if PDHG from it reaches the requested KKT tolerance
within the iteration limit; otherwise the instance is solved again from the
cold (zero) start, which is also the yardstick every warm start is compared
with.
"""

from __future__ import annotations

import time

import numpy as np

from . import pdlp as P


def init_params(in_dim: int, hidden: int, out_dim: int, seed: int) -> np.ndarray:
    """He-uniform weights, zero biases (flat layout of pdlp_mlp_set_params)."""
    rng = np.random.default_rng([0x11A1, seed])
    parts = []
    for fan_in, fan_out in ((in_dim, hidden), (hidden, hidden), (hidden, out_dim)):
        lim = np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, fan_in * fan_out))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def solve_many(make_lp, count, tol, max_iter=1_000_000, chunk=2048, start=None, on_solution=None):
    """Solves LPs make_lp(0..count-1) with the batched solver, `chunk` LPs per
    launch.  start(i) -> (x0, y0) gives warm starts (None: cold).  Each
    solution is handed to on_solution(i, x, y).  Returns (status, iters,
    solve_seconds, create_seconds); solve_seconds covers the batched solves
    only (the graph is captured by an untimed 1-iteration solve first)."""
    st = np.empty(count, dtype=np.int32)
    it = np.empty(count, dtype=np.int64)
    solve_s = create_s = 0.0
    for c0 in range(0, count, chunk):
        ids = range(c0, min(count, c0 + chunk))
        lps = [make_lp(i) for i in ids]
        t = time.perf_counter()
        b = P.BatchSolver(lps)
        create_s += time.perf_counter() - t
        try:
            x0 = y0 = None
            if start is not None:
                pairs = [start(i) for i in ids]
                x0 = np.concatenate([np.asarray(p[0], dtype=np.float64) for p in pairs])
                y0 = np.concatenate([np.asarray(p[1], dtype=np.float64) for p in pairs])
            b.solve(tol=tol, max_iter=1, x0=x0, y0=y0)
            t = time.perf_counter()
            xs, ys, s, k = b.solve(tol=tol, max_iter=max_iter, x0=x0, y0=y0)
            solve_s += time.perf_counter() - t
        finally:
            b.close()
        st[c0:c0 + len(ids)] = s
        it[c0:c0 + len(ids)] = k
        if on_solution is not None:
            for j, i in enumerate(ids):
                on_solution(i, xs[j], ys[j])
    return st, it, solve_s, create_s


def solve_with_fallback(make_lp, count, tol, start, max_iter=1_000_000, chunk=2048):
    """The acceptance rule: warm solves, then cold re-solves of every LP whose
    warm solve did not reach `tol`.  Returns a dict of statuses, iterations
    (warm + cold for the fallbacks) and seconds."""
    st, it, solve_s, create_s = solve_many(make_lp, count, tol, max_iter, chunk, start)
    bad = np.flatnonzero(st != P.OPTIMAL)
    total = it.copy()
    if bad.size:
        st2, it2, s2, c2 = solve_many(lambda j: make_lp(int(bad[j])), bad.size, tol, max_iter, chunk)
        total[bad] += it2
        st = st.copy()
        st[bad] = st2
        solve_s += s2
        create_s += c2
    return {"status": st, "iters": total, "warm_iters": it, "fallbacks": int(bad.size), "solve_s": solve_s,
            "create_s": create_s}


def train(X, T, hidden=256, schedule=((2000, 1e-3),), batch=256, seed=0, max_batch=None):
    """Trains the MLP X -> T (rows are samples) with Adam, mini-batches drawn
    without replacement within each step; `schedule` lists (steps, lr)
    segments.  Returns (net, losses)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    batch = min(batch, X.shape[0])
    net = P.Mlp(X.shape[1], hidden, T.shape[1], max_batch=max_batch or max(batch, 256))
    net.set_params(init_params(X.shape[1], hidden, T.shape[1], seed))
    net.set_data(X, T)
    rng = np.random.default_rng([0x7A1B, seed])
    losses = []
    for steps, lr in schedule:
        idx = np.stack([rng.choice(X.shape[0], size=batch, replace=False) for _ in range(steps)])
        losses.append(net.train(idx, lr=lr))
    return net, np.concatenate(losses)


def mean_start(T, n):
    """Naive warm start: the mean training solution, for every instance."""
    mu = np.asarray(T, dtype=np.float64).mean(axis=0)
    return mu[:n], mu[n:]


def nearest_index(train_X, X, exclude_self: bool = False, chunk: int = 2048):
    """Index of the nearest training parameter for each row of X (with
    exclude_self, X is the training set itself and each row's own index is
    skipped: the leave-one-out neighbour)."""
    A = np.asarray(train_X, dtype=np.float64)
    B = np.asarray(X, dtype=np.float64)
    a2 = (A * A).sum(1)
    out = np.empty(B.shape[0], dtype=np.int64)
    for c0 in range(0, B.shape[0], chunk):
        Bc = B[c0:c0 + chunk]
        d = (Bc * Bc).sum(1)[:, None] - 2 * Bc @ A.T + a2[None, :]
        if exclude_self:
            d[np.arange(Bc.shape[0]), np.arange(c0, c0 + Bc.shape[0])] = np.inf
        out[c0:c0 + chunk] = np.argmin(d, axis=1)
    return out


def residual_inputs(theta, theta_nn):
    """Inputs of the neighbour-residual model: the parameter and its offset
    from the neighbour whose solution the prediction corrects."""
    theta = np.asarray(theta, dtype=np.float32)
    return np.concatenate([theta, np.asarray(theta_nn, dtype=np.float32) - theta], axis=1)
