"""The library's host-side spaces, orderings, level sets and sparsity
patterns (csrc/pattern.cpp, compiled by g++ without CUDA) against the
oracle, bit for bit: the same ordering permutation and level sets, and the
same nonzero structure of A_h, B and Q once the internal numbering is mapped
back to the natural one.  The derived structures the kernels read are
checked from their definitions: L and U = L^T as the strict triangles of
the internal A, the maps that fill U from L and B^T from B, the diagonal
positions, and the internal numbering as the stable sort of ordering
positions by level."""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse as sp

ORDERINGS = {"natural": 0, "rcm": 1, "multicolour": 2}
NAMES = ["perm", "level", "rlevel", "lev_ptr", "int_to_pos", "order", "iorder", "A_ptr", "A_col", "A_diag",
         "L_ptr", "L_col", "U_ptr", "U_col", "U_map", "B_ptr", "B_col", "Bt_ptr", "Bt_col", "Bt_map",
         "Q_ptr", "Q_col"]


def host_pattern(lib, dim, N, p, ordering):
    sizes = np.zeros(11, np.int64)
    msg = C.create_string_buffer(256)
    rc = lib.lt_pattern(C.c_int32(dim), C.c_int32(N), C.c_int32(p), C.c_int32(ORDERINGS.get(ordering, ordering)),
                        sizes.ctypes.data_as(C.c_void_p), msg, C.c_int32(256))
    if rc:
        raise ValueError(msg.value.decode())
    lib.lt_pattern_array.restype = C.c_int64
    out = dict(zip(["n_u", "n_p", "nlev", "nrlev", "ncolours", "nnzA", "nnzL", "nnzB", "nnzQ", "nL", "nU"],
                   (int(v) for v in sizes)))
    for w, name in enumerate(NAMES):
        n = lib.lt_pattern_array(C.c_int32(w), None)
        a = np.zeros(max(n, 1), np.int32)
        lib.lt_pattern_array(C.c_int32(w), a.ctypes.data_as(C.c_void_p))
        out[name] = a[:n]
    return out


def structure(M):
    M = sp.csr_matrix(M)
    M.sort_indices()
    return M.indptr.copy(), M.indices.copy()


def ones(ptr, col, shape):
    return sp.csr_matrix((np.ones(len(col)), col, ptr), shape=shape)


CASES = [(2, 5, 2), (2, 8, 3), (2, 6, 4), (2, 4, 6), (3, 3, 3), (3, 2, 2), (3, 4, 4)]


@pytest.mark.parametrize("ordering", ["natural", "rcm", "multicolour"])
@pytest.mark.parametrize("dim,N,p", CASES)
def test_pattern_matches_oracle(oracle_mod, host_lib, dim, N, p, ordering):
    H = host_pattern(host_lib, dim, N, p, ordering)
    P = oracle_mod.Problem(dim, N, p, ordering=ordering)
    n, n_p = H["n_u"], H["n_p"]
    assert (n, n_p) == (P.n_u, P.n_p)
    # the ordering and both level sets, bit for bit
    perm, lev, rlev = P.ordering_arrays()
    assert np.array_equal(H["perm"], perm)
    assert np.array_equal(H["level"], lev) and np.array_equal(H["rlevel"], rlev)
    assert H["nlev"] == lev.max() + 1 and H["nrlev"] == rlev.max() + 1
    if ordering == "multicolour":
        assert H["ncolours"] == dim * (p + 1) * p ** (dim - 1)
    # internal numbering: ordering positions sorted by level, stable
    assert np.array_equal(H["int_to_pos"], np.argsort(lev, kind="stable"))
    assert np.array_equal(H["lev_ptr"], np.concatenate([[0], np.cumsum(np.bincount(lev))]))
    order = H["order"]
    assert np.array_equal(order, perm[H["int_to_pos"]])
    assert np.array_equal(H["iorder"][order], np.arange(n))
    # A, B, Q: the oracle's structure after mapping internal -> natural
    Pm = sp.csr_matrix((np.ones(n), (np.arange(n), order)), shape=(n, n))  # row r picks natural order[r]
    A_int = ones(H["A_ptr"], H["A_col"], (n, n))
    A_nat = (Pm.T @ A_int @ Pm).tocsr()
    assert H["nnzA"] == A_int.nnz
    for got, want in ((A_nat, P.scipy("A")),
                      ((ones(H["B_ptr"], H["B_col"], (n_p, n)) @ Pm).tocsr(), P.scipy("B")),
                      (ones(H["Q_ptr"], H["Q_col"], (n_p, n_p)), P.scipy("Q"))):
        g, w = structure(got), structure(want)
        assert np.array_equal(g[0], w[0]) and np.array_equal(g[1], w[1])
    assert H["nnzB"] == len(H["B_col"]) and H["nnzQ"] == len(H["Q_col"])
    # columns ascending in every row; the diagonal position of every A row
    for ptr, col in ((H["A_ptr"], H["A_col"]), (H["B_ptr"], H["B_col"]), (H["Q_ptr"], H["Q_col"])):
        row = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
        assert np.all((np.diff(col) > 0) | (np.diff(row) != 0))
    assert np.array_equal(H["A_col"][H["A_diag"]], np.arange(n))
    # L and U: the strict triangles of the internal A (the factor's pattern)
    Lw, Uw = structure(sp.tril(A_int, k=-1)), structure(sp.triu(A_int, k=1))
    assert np.array_equal(H["L_ptr"], Lw[0]) and np.array_equal(H["L_col"], Lw[1])
    assert np.array_equal(H["U_ptr"], Uw[0]) and np.array_equal(H["U_col"], Uw[1])
    assert H["nnzL"] == len(H["L_col"]) + n
    # U_map: U(r, j) is filled from L(j, r)
    urow = np.repeat(np.arange(n), np.diff(H["U_ptr"]))
    lrow = np.repeat(np.arange(n), np.diff(H["L_ptr"]))
    assert np.array_equal(H["L_col"][H["U_map"]], urow)
    assert np.array_equal(lrow[H["U_map"]], H["U_col"])
    # B^T (internal velocity rows, ascending pressure columns) and its map into B
    Btw = structure(ones(H["B_ptr"], H["B_col"], (n_p, n)).T)
    assert np.array_equal(H["Bt_ptr"], Btw[0]) and np.array_equal(H["Bt_col"], Btw[1])
    btrow = np.repeat(np.arange(n), np.diff(H["Bt_ptr"]))
    brow = np.repeat(np.arange(n_p), np.diff(H["B_ptr"]))
    assert np.array_equal(H["B_col"][H["Bt_map"]], btrow)
    assert np.array_equal(brow[H["Bt_map"]], H["Bt_col"])


@pytest.mark.parametrize("args,msg", [((4, 4, 3, 0), "dim"), ((2, 4, 7, 0), "p must"), ((2, 4, 1, 0), "p must"),
                                      ((2, 0, 3, 0), "N out of range"), ((2, 4, 3, 3), "ordering")])
def test_invalid_problems_are_rejected(host_lib, args, msg):
    with pytest.raises(ValueError, match=msg):
        host_pattern(host_lib, *args)
