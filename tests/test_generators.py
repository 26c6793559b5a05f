"""Input generators (no solver arithmetic): single members of a batch are
rebuilt exactly, so a batch member can be studied without its batch."""

import numpy as np

import lpgen


def test_batch_lp_equals_the_member_of_its_batch():
    batch = lpgen.batch_lps(12, seed=3, m_lo=20, m_hi=400)
    for i in (0, 5, 11):
        one = lpgen.batch_lp(i, seed=3, m_lo=20, m_hi=400)
        ref = batch[i]
        assert (one.m, one.n, one.n_eq) == (ref.m, ref.n, ref.n_eq)
        for f in ("row_ptr", "col_idx", "val", "c", "q", "l", "u", "x_star", "y_star"):
            assert np.array_equal(getattr(one, f), getattr(ref, f)), f


def test_permuted_lp_is_the_same_lp():
    import oracle

    lp = lpgen.tiny_lp(3)
    p = lpgen.permuted(lp, 1)
    assert p.nnz == lp.nnz and np.all(np.diff(p.row_ptr) >= 0)
    assert sorted(p.val.tolist()) == sorted(lp.val.tolist())
    t = oracle.kkt_terms(p, p.x_star, p.y_star)  # the planted pair, permuted, is still optimal
    assert t["rp"] < 1e-12 and t["rd"] < 1e-12 and abs(t["pobj"] - lp.obj_star) < 1e-10 * (1 + abs(lp.obj_star))
    # equality rows stay first
    assert p.n_eq == lp.n_eq and np.array_equal(np.sort(p.q[: p.n_eq]), np.sort(lp.q[: lp.n_eq]))


def test_batch_subset_builds_the_same_members():
    """A rank of a sharded batch builds only its LPs: each equals the member of
    the whole batch, and the expected work follows the realised nonzeros."""
    full = lpgen.batch_lps(10, seed=3)
    sub = lpgen.batch_subset([2, 5, 9], 10, seed=3)
    for i, lp in zip([2, 5, 9], sub):
        assert np.array_equal(lp.row_ptr, full[i].row_ptr) and np.array_equal(lp.col_idx, full[i].col_idx)
        assert np.array_equal(lp.val, full[i].val) and np.array_equal(lp.c, full[i].c)
    w = lpgen.batch_work(10, seed=3)
    assert np.corrcoef(w, [lp.nnz for lp in full])[0, 1] > 0.99
