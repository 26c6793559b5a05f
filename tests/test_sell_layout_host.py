"""Host-side create code, no GPU.  The sliced-ELL layout (csrc/pdlp_sell.h): the row
renumbering, slices, long rows and work schedule that the step and check
kernels walk, checked against the properties the kernels rely on (a
permutation that keeps the equality rows first, rows by length inside each
group, slices of 32 consecutive rows inside a group, long rows whole, every
row in exactly one work item, disjoint storage that fills the total, items
by cost).  The threaded stable CSR transpose (csrc/pdlp_host.h) against
scipy.  Each header is compiled into a small host program with nvcc."""

import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SELL_LONG = 48


@pytest.fixture(scope="module")
def layout_exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("sell") / "sell_layout_host")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-x", "cu", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "paper_2311_12180_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "sell_layout_host.cpp"), "-o", exe], check=True)
    return exe


def _layout(exe, lengths, split):
    lengths = np.asarray(lengths, dtype=np.int64)
    ptr = np.concatenate([[0], np.cumsum(lengths)])
    text = "%d %d\n%s\n" % (lengths.size, split, " ".join(map(str, ptr)))
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    total, nlong, nslices, nitems = map(int, out[0].split())
    rows = lengths.size
    vec = lambda s: np.array(s.split(), dtype=np.int64) if rows else np.zeros(0, np.int64)
    perm, base, lane = vec(out[1]), vec(out[2]), vec(out[3])
    items = np.array([list(map(int, l.split())) for l in out[4:4 + nitems]], dtype=np.int64).reshape(-1, 4)
    return dict(total=total, nlong=nlong, nslices=nslices, perm=perm, base=base, lane=lane, items=items)


def _check(L, lengths, split):
    lengths = np.asarray(lengths, dtype=np.int64)
    rows = lengths.size
    perm, base, lane, items = L["perm"], L["base"], L["lane"], L["items"]
    # a permutation that keeps the two groups in place
    assert np.array_equal(np.sort(perm), np.arange(rows))
    assert np.all((perm < split) == (np.arange(rows) < split))
    ln = lengths[perm]  # internal row -> its length
    for g0, g1 in ((0, split), (split, rows)):
        seg, src = ln[g0:g1], perm[g0:g1]
        assert np.all(np.diff(seg) <= 0)  # longest first
        ties = np.diff(seg) == 0
        assert np.all(np.diff(src)[ties] > 0)  # stable among equal lengths
    assert np.array_equal(lane == 0, ln > SELL_LONG)
    group = (np.arange(rows) >= split).astype(int)
    covered = np.zeros(rows, dtype=int)
    regions = []
    nlong = nslices = 0
    for r, nr, length, off in items:
        assert off % 32 == 0
        if nr == -1:  # a long row, stored whole
            assert lane[r] == 0 and length == ln[r] and base[r] == off
            size = (length + 31) // 32 * 32
            covered[r] += 1
            nlong += 1
            cost = (length + 31) // 32 + 2
        else:  # a slice of nr consecutive rows of one group, entry k of row l at off + 32 k + l
            assert 1 <= nr <= 32 and r + nr <= rows
            rs = np.arange(r, r + nr)
            assert np.all(group[rs] == group[r]) and np.all(lane[rs] == 1)
            assert np.array_equal(base[rs], off + np.arange(nr))
            assert length == ln[r] >= ln[rs].max()
            g_end = split if r < split else rows
            first_slice = r - (split if r >= split else 0) - int(np.sum((ln > SELL_LONG) & (group == group[r])))
            assert first_slice % 32 == 0 and (nr == 32 or r + nr == g_end)
            size = 32 * length
            covered[rs] += 1
            nslices += 1
            cost = length + 2
        regions.append((off, off + size, cost))
    assert np.all(covered == 1)
    assert (nlong, nslices) == (L["nlong"], L["nslices"])
    spans = sorted((a, b) for a, b, _ in regions if b > a)
    assert all(spans[i][1] == spans[i + 1][0] for i in range(len(spans) - 1))
    assert sum(b - a for a, b in spans) == L["total"] and (not spans or (spans[0][0] == 0 and spans[-1][1] == L["total"]))
    costs = [c for _, _, c in regions]
    assert all(costs[i] >= costs[i + 1] for i in range(len(costs) - 1))


def _zipf_lengths(rng, rows, cap=400):
    return np.minimum(rng.zipf(1.6, size=rows), cap) - rng.integers(0, 2, size=rows)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_power_law_rows(layout_exe, seed):
    rng = np.random.default_rng(seed)
    rows = 1500 + 37 * seed
    lengths = _zipf_lengths(rng, rows)
    split = int(0.4 * rows)
    L = _layout(layout_exe, lengths, split)
    assert L["nlong"] == int(np.sum(lengths > SELL_LONG)) > 0
    _check(L, lengths, split)


@pytest.mark.parametrize("case", ["empty", "all_long", "all_zero", "no_equalities", "all_equalities",
                                  "ties_33", "exactly_32", "boundary_48_49"])
def test_edge_cases(layout_exe, case):
    lengths, split = {
        "empty": ([], 0),
        "all_long": ([49, 200, 64, 1000, 50], 2),
        "all_zero": ([0] * 70, 35),
        "no_equalities": (list(range(100)), 0),
        "all_equalities": (list(range(100, 0, -1)), 100),
        "ties_33": ([5] * 33, 10),
        "exactly_32": ([7] * 32 + [3] * 32, 32),
        "boundary_48_49": ([48, 49, 48, 49, 1], 2),
    }[case]
    L = _layout(layout_exe, lengths, split)
    _check(L, lengths, split)
    if case == "empty":
        assert L["total"] == 0 and len(L["items"]) == 0
    if case == "all_zero":
        assert L["total"] == 0 and L["nslices"] == 4  # 35 -> 32 + 3, 35 -> 32 + 3
    if case == "exactly_32":
        assert L["nslices"] == 2 and L["total"] == 32 * 7 + 32 * 3
    if case == "boundary_48_49":
        assert L["nlong"] == 2


@pytest.fixture(scope="module")
def transpose_exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("tr") / "csr_transpose_host")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-x", "cu", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "paper_2311_12180_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "csr_transpose_host.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("m,n,nnz", [(0, 5, 0), (7, 0, 0), (50, 40, 300), (3000, 5000, 200000)])
def test_threaded_host_transpose_is_the_stable_transpose(transpose_exe, m, n, nnz):
    """csr_transpose (several threads from 65536 nonzeros on) equals the
    stable transpose: K' rows hold K's entries in increasing row order, the
    values moved bit for bit (scipy's CSR -> CSC conversion as the judge);
    empty rows and columns included."""
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(m + n)
    if nnz:
        rows = np.sort(rng.integers(0, m, size=nnz))
        cols = rng.integers(0, n, size=nnz)
        keep = np.unique(rows.astype(np.int64) * n + cols, return_index=True)[1]
        rows, cols = rows[keep], cols[keep]
    else:
        rows = cols = np.zeros(0, dtype=np.int64)
    vals = rng.standard_normal(rows.size) * np.exp(rng.uniform(-30, 30, rows.size))
    ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=ptr[1:])
    bits = vals.view(np.uint64)
    text = "%d %d %d\n%s\n%s\n%s\n" % (m, n, rows.size, " ".join(map(str, ptr)), " ".join(map(str, cols)),
                                     " ".join("%x" % b for b in bits))
    out = subprocess.run([transpose_exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    tp = np.array(out[0].split(), dtype=np.int64)
    ti = np.array(out[1].split(), dtype=np.int64)
    tv = np.array([int(h, 16) for h in out[2].split()], dtype=np.uint64).view(np.float64)
    K = sp.csr_matrix((vals, cols, ptr), shape=(m, n))
    C = K.tocsc()
    C.sort_indices()
    assert np.array_equal(tp, C.indptr) and np.array_equal(ti, C.indices)
    assert np.array_equal(tv.view(np.uint64), np.asarray(C.data).view(np.uint64))
