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
