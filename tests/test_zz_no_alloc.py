"""The allocation-free scaling entry point, called through the C ABI on
device buffers, against the scaling pdlp_create computes with its own
allocations (pdlp_get_scaling, bitwise) and against the FP64 oracle.

Kept in its own file, collected after every other test file, so that a run
stopping at the first failure has already run the rest of the suite."""

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle
from paper_2311_12180_gb300 import pdlp as P

pytestmark = pytest.mark.gpu


def _device_case(lp, torch):
    K = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    KT = K.T.tocsr()  # rows of K', entries in increasing row-of-K order
    KT.sort_indices()
    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    return dict(
        K_ptr=t(K.indptr.astype(np.int32), torch.int32), K_idx=t(K.indices.astype(np.int32), torch.int32),
        K_val=t(K.data, torch.float64), KT_ptr=t(KT.indptr.astype(np.int32), torch.int32),
        KT_idx=t(KT.indices.astype(np.int32), torch.int32), KT_val=t(KT.data, torch.float64),
        D1=torch.empty(max(lp.m, 1), dtype=torch.float64, device=dev),
        D2=torch.empty(lp.n, dtype=torch.float64, device=dev), KT=KT)


def _call(lp, d, torch):
    stream = torch.cuda.current_stream().cuda_stream
    P.pdlp_scale_device_noalloc(lp.m, lp.n, d["K_ptr"].data_ptr(), d["K_idx"].data_ptr(), d["K_val"].data_ptr(),
                                d["KT_ptr"].data_ptr(), d["KT_idx"].data_ptr(), d["KT_val"].data_ptr(), 10, 1.0,
                                d["D1"].data_ptr(), d["D2"].data_ptr(), stream)
    torch.cuda.synchronize()
    return (d["D1"][: lp.m].cpu().numpy(), d["D2"].cpu().numpy(), d["K_val"].cpu().numpy(),
            d["KT_val"].cpu().numpy())


@pytest.mark.parametrize("case", ["tiny", "powerlaw"])
def test_noalloc_scaling_matches_solver_scaling(case):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    lp = lpgen.tiny_lp(3) if case == "tiny" else lpgen.large_lp(5, m=3000, n=6000, nnz=60000)
    with P.Solver(lp) as s:
        D1e, D2e, ve = s.scaling()
    outs = []
    for _ in range(2):  # two calls in a row, each on fresh unscaled copies
        d = _device_case(lp, torch)
        outs.append(_call(lp, d, torch))
    sv, oD1, oD2 = oracle.precondition(lp, ruiz_iters=10, pc_alpha=1.0)
    for D1, D2, v, vt in outs:
        # the same divisions in the same order as pdlp_create's scaling: bitwise
        assert np.array_equal(D1, D1e) and np.array_equal(D2, D2e) and np.array_equal(v, ve)
        # and the FP64 oracle's Sec. 2.2 scaling up to the order of the
        # Pock-Chambolle sums
        np.testing.assert_allclose(D1, oD1, rtol=1e-13)
        np.testing.assert_allclose(D2, oD2, rtol=1e-13)
        np.testing.assert_allclose(v, sv, rtol=1e-13)
        # K' scaled with the same divisions stays the exact transpose of K
        Ks = sp.csr_matrix((v, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n)).T.tocsr()
        Ks.sort_indices()
        assert np.array_equal(Ks.data, vt)
    assert all(np.array_equal(a, b) for a, b in zip(outs[0], outs[1]))


def test_noalloc_rejects_sizes_beyond_its_limit():
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    with pytest.raises(P.PdlpError) as e:
        P.pdlp_scale_device_noalloc(262145, 10, p, p, p, p, p, p, 10, 1.0, p, p, None)
    assert e.value.code == P.ERR_INVALID and "262144" in str(e.value)
