"""The SELL-32 copies and the block layouts of the IC(0) sweeps, built on the
host (layouts.h), on the CPU: bit-exact index work, checked entry by entry.

The factor patterns are the library's: IC(0) keeps the pattern of the strict
lower part of the reordered A_h (Sec. 6.4), the levels are the longest-path
levels of that DAG, and the internal numbering sorts rows by level (a
topological order, so the factor stays lower triangular).  A and the
orderings come from the oracle; the levels are recomputed here from their
definition.  Several SM counts exercise both grid-sizing branches (one wave,
and a multiple of the SM count) and the per-block caps.
"""
import ctypes as C
import os

import numpy as np
import pytest
import scipy.sparse as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ROWS, ENTRIES, SLOTS = 256, 2048, 2048  # block caps of layouts.h


@pytest.fixture(scope="module")
def lt(host_lib):
    return host_lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


_patterns = {}


def factor_patterns(oracle_mod, dim, N, p, ordering):
    """(L ptr, L col, U ptr, U col, lev_ptr) in the internal numbering."""
    key = (dim, N, p, ordering)
    if key not in _patterns:
        _patterns[key] = _factor_patterns(oracle_mod, dim, N, p, ordering)
    return _patterns[key]


def _factor_patterns(oracle_mod, dim, N, p, ordering):
    P = oracle_mod.Problem(dim, N, p, ordering=ordering)
    perm, _, _ = P.ordering_arrays()
    A = P.scipy("A").tocsr()[perm][:, perm].tocsr()
    Lp = sp.tril(A, k=-1).tocsr()
    n = A.shape[0]
    lev = np.zeros(n, np.int64)
    for r in range(n):  # longest path from a source of the DAG of L
        c = Lp.indices[Lp.indptr[r]:Lp.indptr[r + 1]]
        lev[r] = lev[c].max() + 1 if len(c) else 0
    order = np.argsort(lev, kind="stable")
    Ai = A[order][:, order].tocsr()
    L = sp.tril(Ai, k=-1).tocsr()
    U = sp.triu(Ai, k=1).tocsr()
    L.sort_indices()
    U.sort_indices()
    counts = np.bincount(lev, minlength=lev.max() + 1)
    lev_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return (L.indptr.astype(np.int32), L.indices.astype(np.int32), U.indptr.astype(np.int32),
            U.indices.astype(np.int32), lev_ptr)


def packed(lt, ptr, col, lev_ptr, n_sm, split):
    n, nlev = len(ptr) - 1, len(lev_ptr) - 1
    sizes = np.zeros(3, np.int64)
    lt.lt_packed(_p(ptr), _p(col), C.c_int32(n), _p(lev_ptr), C.c_int32(nlev), C.c_int32(n_sm),
                 C.c_int32(split), _p(sizes))
    ok, nb, ns = (int(v) for v in sizes)
    if not ok:
        return None
    desc = np.zeros(4 * nb, np.int32)
    pcol = np.zeros(max(ns, 1), np.int32)
    psrc = np.zeros(max(ns, 1), np.int32)
    lev_b = np.zeros(nlev, np.int32)
    lev_nb = np.zeros(nlev, np.int32)
    lev_mean = np.zeros(nlev, np.float32)
    caps = np.zeros(2, np.int32)
    lt.lt_packed_fetch(_p(desc), _p(pcol), _p(psrc), _p(lev_b), _p(lev_nb), _p(lev_mean), _p(caps))
    return dict(desc=desc.reshape(-1, 4), col=pcol[:ns], src=psrc[:ns], lev_b=lev_b, lev_nb=lev_nb,
                lev_mean=lev_mean, cap=int(caps[0]), rcap=int(caps[1]))


def staged(lt, ptr, lev_ptr, n_sm):
    n, nlev = len(ptr) - 1, len(lev_ptr) - 1
    sizes = np.zeros(3, np.int64)
    lt.lt_staged(_p(ptr), C.c_int32(n), _p(lev_ptr), C.c_int32(nlev), C.c_int32(n_sm), _p(sizes))
    ok, nb = int(sizes[0]), int(sizes[1])
    if not ok:
        return None
    desc = np.zeros(4 * nb, np.int32)
    lev_b = np.zeros(nlev, np.int32)
    lev_nb = np.zeros(nlev, np.int32)
    caps = np.zeros(2, np.int32)
    lt.lt_staged_fetch(_p(desc), _p(lev_b), _p(lev_nb), _p(caps))
    return dict(desc=desc.reshape(-1, 4), lev_b=lev_b, lev_nb=lev_nb, ecap=int(caps[0]), rcap=int(caps[1]))


def check_level_blocks(lev_ptr, lev_b, lev_nb, first_rows, n_rows, n_sm):
    """Blocks of level l are lev_b[l] .. + lev_nb[l] - 1 and cover its rows in order."""
    nlev = len(lev_ptr) - 1
    assert lev_b[0] == 0 and np.array_equal(lev_b[1:], np.cumsum(lev_nb)[:-1])
    assert lev_b[-1] + lev_nb[-1] == len(first_rows)
    for l in range(nlev):
        b0, b1 = lev_b[l], lev_b[l] + lev_nb[l]
        starts, sizes = first_rows[b0:b1], n_rows[b0:b1]
        assert starts[0] == lev_ptr[l]
        assert np.array_equal(starts[1:], starts[:-1] + sizes[:-1])
        assert starts[-1] + sizes[-1] == lev_ptr[l + 1]
        R = lev_ptr[l + 1] - lev_ptr[l]
        if R > 0:
            assert np.all(sizes > 0)
            # a level never gets fewer blocks than min(rows, SM count)
            assert lev_nb[l] >= min(R, n_sm) or lev_nb[l] * ROWS >= R


def check_packed(lay, ptr, col, lev_ptr, n_sm, split):
    n, nnz, nlev = len(ptr) - 1, int(ptr[-1]), len(lev_ptr) - 1
    level = np.repeat(np.arange(nlev), np.diff(lev_ptr))
    D = lay["desc"]
    rb, nr, off, w = D[:, 0], D[:, 1], D[:, 2], D[:, 3]
    lo, lr = w & 0xFFFF, w >> 16
    if split == 0:
        assert np.all(lr == 0)
    # caps and the dense packing of the blocks
    assert np.all(nr <= ROWS) and np.all(nr * (lo + lr) <= SLOTS)
    assert lay["cap"] == int((nr * (lo + lr)).max()) and lay["rcap"] == int(nr.max())
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(nr * (lo + lr))[:-1]]))
    assert len(lay["col"]) == int((nr * (lo + lr)).sum())
    check_level_blocks(lev_ptr, lay["lev_b"], lay["lev_nb"], rb, nr, n_sm)
    # every entry exactly once, padding marked, columns copied
    src, pcol = lay["src"], lay["col"]
    real = src >= 0
    assert np.array_equal(np.sort(src[real]), np.arange(nnz))
    assert np.all(pcol[~real] == -1)
    assert np.array_equal(pcol[real], col[src[real]])
    # each entry at its row's slot, split by the level of its column, in CSR order
    expect = np.full(len(src), -1, np.int64)
    first_count = np.zeros(nlev, np.int64)
    for b in range(len(D)):
        for i in range(nr[b]):
            r = rb[b] + i
            e = np.arange(ptr[r], ptr[r + 1])
            second = (level[col[e]] == level[r] - split) if split else np.zeros(len(e), bool)
            e1, e2 = e[~second], e[second]
            assert len(e1) <= lo[b] and len(e2) <= lr[b]
            expect[off[b] + np.arange(len(e1)) * nr[b] + i] = e1
            expect[off[b] + nr[b] * lo[b] + np.arange(len(e2)) * nr[b] + i] = e2
            first_count[level[r]] += len(e1)
    assert np.array_equal(expect, src)
    rows = np.diff(lev_ptr)
    mean = np.where(rows > 0, first_count / np.maximum(rows, 1), 0.0)
    np.testing.assert_allclose(lay["lev_mean"], mean, rtol=1e-6)
    return lo, lr


CASES = [(2, 60, 3, "multicolour"), (3, 6, 3, "multicolour"), (2, 24, 4, "rcm"), (2, 10, 3, "natural")]


@pytest.mark.parametrize("dim,N,p,ordering", CASES)
@pytest.mark.parametrize("n_sm", [1, 3, 152])
def test_packed_and_split_layouts(oracle_mod, lt, dim, N, p, ordering, n_sm):
    Lptr, Lcol, Uptr, Ucol, lev_ptr = factor_patterns(oracle_mod, dim, N, p, ordering)
    for ptr, col, split in ((Lptr, Lcol, 0), (Uptr, Ucol, 0), (Lptr, Lcol, 1), (Uptr, Ucol, -1)):
        lay = packed(lt, ptr, col, lev_ptr, n_sm, split)
        assert lay is not None
        lo, lr = check_packed(lay, ptr, col, lev_ptr, n_sm, split)
        if split and ordering == "multicolour":
            assert lr.max() > 0 and lo.max() > 0  # both segments are used


@pytest.mark.parametrize("dim,N,p,ordering", CASES)
@pytest.mark.parametrize("n_sm", [1, 3, 152])
def test_staged_layout(oracle_mod, lt, dim, N, p, ordering, n_sm):
    Lptr, _, Uptr, _, lev_ptr = factor_patterns(oracle_mod, dim, N, p, ordering)
    for ptr in (Lptr, Uptr):
        lay = staged(lt, ptr, lev_ptr, n_sm)
        D = lay["desc"]
        r0, r1, e0, e1 = D[:, 0], D[:, 1], D[:, 2], D[:, 3]
        assert np.array_equal(e0, ptr[r0]) and np.array_equal(e1, ptr[r1])
        assert np.all(r1 - r0 <= ROWS) and np.all(e1 - e0 <= ENTRIES)
        assert lay["ecap"] == int((e1 - e0).max()) and lay["rcap"] == int((r1 - r0).max())
        check_level_blocks(lev_ptr, lay["lev_b"], lay["lev_nb"], r0, r1 - r0, n_sm)


def test_a_level_of_many_rows_is_cut_at_the_caps(lt):
    """One level of 5000 rows of 40 entries on 2 SMs: at least the
    ceil(entries / cap) blocks the caps force (the target share per block is
    set from that count rounded up to a multiple of the SM count, and the
    greedy cut may add one), every block within the row and slot caps."""
    n0, n1, k = 40, 5000, 40
    ptr = np.concatenate([np.zeros(n0 + 1, np.int64), k * np.arange(1, n1 + 1)]).astype(np.int32)
    col = np.tile(np.arange(k, dtype=np.int32), n1)
    lev_ptr = np.array([0, n0, n0 + n1], np.int32)
    lay = packed(lt, ptr, col, lev_ptr, 2, 0)
    check_packed(lay, ptr, col, lev_ptr, 2, 0)
    assert -(-n1 * k // SLOTS) <= lay["lev_nb"][1] <= -(-n1 * k // SLOTS) + 2
    st = staged(lt, ptr, lev_ptr, 2)
    assert st["lev_nb"][1] >= (n1 * k) // ENTRIES


@pytest.mark.parametrize("extra,ok", [(0, True), (1, False)])
def test_rows_longer_than_a_block_make_the_layouts_unavailable(lt, extra, ok):
    """A row of 2048 entries fits one block; 2049 does not, and then no block
    layout is built (the library falls back to the CSR and SELL sweeps)."""
    m = SLOTS + extra
    ptr = np.concatenate([np.zeros(m + 1, np.int64), [m]]).astype(np.int32)
    col = np.arange(m, dtype=np.int32)
    lev_ptr = np.array([0, m, m + 1], np.int32)
    for split in (0, 1):
        lay = packed(lt, ptr, col, lev_ptr, 152, split)
        assert (lay is not None) == ok
        if ok:
            check_packed(lay, ptr, col, lev_ptr, 152, split)
    assert (staged(lt, ptr, lev_ptr, 152) is not None) == ok


def sell(lt, ptr, col, lev_ptr):
    n, nlev = len(ptr) - 1, len(lev_ptr) - 1
    sizes = np.zeros(3, np.int64)
    lt.lt_sell(_p(ptr), _p(col), C.c_int32(n), _p(lev_ptr), C.c_int32(nlev), _p(sizes))
    ok, ns, slots = (int(v) for v in sizes)
    assert ok
    row0 = np.zeros(ns + 1, np.int32)
    off = np.zeros(ns + 1, np.int32)
    rowlen = np.zeros(max(n, 1), np.int32)
    scol = np.zeros(max(slots, 1), np.int32)
    ssrc = np.zeros(max(slots, 1), np.int32)
    lev_slice = np.zeros(nlev + 1, np.int32)
    lt.lt_sell_fetch(_p(row0), _p(off), _p(rowlen), _p(scol), _p(ssrc), _p(lev_slice))
    return row0, off, rowlen[:n], scol[:slots], ssrc[:slots], lev_slice


@pytest.mark.parametrize("dim,N,p,ordering", CASES)
def test_sell_copies(oracle_mod, lt, dim, N, p, ordering):
    """Slices of at most 32 rows inside one level, each padded to its longest
    row; entry k of the row in lane i at off[s] + 32 k + i, every entry once,
    padding marked -1 in the slot map."""
    Lptr, Lcol, Uptr, Ucol, lev_ptr = factor_patterns(oracle_mod, dim, N, p, ordering)
    for ptr, col in ((Lptr, Lcol), (Uptr, Ucol)):
        row0, off, rowlen, scol, ssrc, lev_slice = sell(lt, ptr, col, lev_ptr)
        n, ns = len(ptr) - 1, len(row0) - 1
        assert np.array_equal(rowlen, np.diff(ptr))
        assert row0[0] == 0 and row0[-1] == n and np.all(np.diff(row0) >= 1) and np.all(np.diff(row0) <= 32)
        for l in range(len(lev_ptr) - 1):  # the slices of a level tile exactly its rows
            assert row0[lev_slice[l]] == lev_ptr[l] and row0[lev_slice[l + 1]] == lev_ptr[l + 1]
        expect = np.full(len(ssrc), -1, np.int64)
        for s in range(ns):
            rows = np.arange(row0[s], row0[s + 1])
            assert off[s + 1] - off[s] == 32 * rowlen[rows].max(initial=0)
            for i, r in enumerate(rows):
                expect[off[s] + 32 * np.arange(rowlen[r]) + i] = np.arange(ptr[r], ptr[r + 1])
        assert np.array_equal(expect, ssrc)
        real = ssrc >= 0
        assert np.array_equal(scol[real], col[ssrc[real]])


def test_a_diagonal_only_factor_gives_empty_copies(lt):
    """A factor with no strict entries (one level of 70 rows, every row empty):
    the SELL copy has no slots and the packed copy no slots, and both still
    tile the level, so the upload sends no entry and reads nothing past the
    empty host vectors."""
    n = 70
    ptr = np.zeros(n + 1, np.int32)
    col = np.zeros(1, np.int32)  # a valid pointer for an empty vector
    lev_ptr = np.array([0, n], np.int32)
    row0, off, rowlen, scol, ssrc, lev_slice = sell(lt, ptr, col[:0], lev_ptr)
    assert len(scol) == 0 and len(ssrc) == 0 and np.all(rowlen == 0)
    assert row0[lev_slice[0]] == 0 and row0[lev_slice[1]] == n
    assert np.all(off == 0)
    for split in (0, 1):
        lay = packed(lt, ptr, col[:0], lev_ptr, 152, split)
        assert lay is not None and len(lay["col"]) == 0 and len(lay["src"]) == 0
        check_packed(lay, ptr, col[:0], lev_ptr, 152, split)
