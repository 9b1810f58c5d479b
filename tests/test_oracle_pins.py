"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- a closed form, exact rational arithmetic, a library routine
(scipy, networkx, torch autograd) or brute force -- so that a dropped term, a
wrong sign, a wrong index or a transposed operand in ``oracle/`` fails here.

CPU only (no GPU marker)."""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _csr(rp, ci, v=None):
    n = len(rp) - 1
    if v is None:
        v = np.ones(len(ci))
    return sp.csr_matrix((v, ci, rp), shape=(n, n))


def _split_lu(rp, ci, lu):
    """Dense L (unit) and U from the combined factor stored in A's pattern."""
    n = len(rp) - 1
    D = _csr(rp, ci, lu).toarray()
    L = np.tril(D, -1) + np.eye(n)
    U = np.triu(D)
    return L, U


# ---------------------------------------------------------------- validation
def test_validate_diag_positions_match_search():
    rp, ci, _ = W.random_csr(40, 4.0, seed=3)
    st, diag, _ = O.validate(rp, ci)
    assert st == O.OK
    for i in range(40):
        row = ci[rp[i]:rp[i + 1]]
        assert diag[i] == rp[i] + int(np.searchsorted(row, i))
        assert ci[diag[i]] == i


@pytest.mark.parametrize("case", ["unsorted", "duplicate", "out_of_range", "negative", "no_diag",
                                  "bad_rowptr"])
def test_validate_rejects(case):
    rp = np.array([0, 2, 4, 6], dtype=np.int32)
    ci = np.array([0, 1, 0, 1, 1, 2], dtype=np.int32)
    want_row, want = 2, O.ERR_PATTERN
    if case == "unsorted":
        ci = np.array([0, 1, 0, 1, 2, 1], dtype=np.int32)
    elif case == "duplicate":
        ci = np.array([0, 1, 0, 1, 2, 2], dtype=np.int32)
    elif case == "out_of_range":
        ci = np.array([0, 1, 0, 1, 2, 3], dtype=np.int32)
    elif case == "negative":
        ci = np.array([0, 1, -1, 1, 1, 2], dtype=np.int32)
        want_row = 1
    elif case == "no_diag":
        ci = np.array([0, 1, 0, 2, 1, 2], dtype=np.int32)
        want_row, want = 1, O.ERR_NO_DIAG
    elif case == "bad_rowptr":
        rp = np.array([0, 2, 1, 6], dtype=np.int32)
        want_row = 1
    st, _, bad = O.validate(rp, ci)
    assert st == want and bad == want_row


# -------------------------------------------------------------------- levels
def _nx_generations(rp, ci, upper):
    nx = pytest.importorskip("networkx")
    n = len(rp) - 1
    G = nx.DiGraph()
    G.add_nodes_from(range(n))
    for i in range(n):
        for j in ci[rp[i]:rp[i + 1]]:
            if (j > i) if upper else (j < i):
                G.add_edge(int(j), i)
    lev = np.zeros(n, dtype=np.int32)
    for l, gen in enumerate(nx.topological_generations(G)):
        lev[list(gen)] = l
    return lev


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("upper", [False, True])
def test_levels_equal_networkx_generations(seed, upper):
    rp, ci, _ = W.random_csr(60, 3.0 + seed, seed=seed)
    want = _nx_generations(rp, ci, upper)
    for route in ("longest_path", "peel"):
        lev, nlev = O.levels(rp, ci, upper=upper, route=route)
        assert np.array_equal(lev, want)
        assert nlev == want.max() + 1


@pytest.mark.parametrize("name,m,coef,dim,gen", [
    ("lap5", 9, (1, 1), 2, lambda m: W.lap5(m)),
    ("lap7", 6, (1, 1, 1), 3, lambda m: W.lap7(m)),
    ("cd27", 5, (1, 2, 4), 3, lambda m: W.cd27(m)[:3]),
    ("aniso5", 11, (1, 1), 2, lambda m: W.aniso5(m)),
])
def test_levels_stencil_closed_forms(name, m, coef, dim, gen):
    rp, ci, _ = gen(m)
    g = np.indices((m,) * dim).reshape(dim, -1)        # slowest axis first
    g = g[::-1]                                          # -> x, y, (z); x varies fastest
    want = sum(c * g[i] for i, c in enumerate(coef)).astype(np.int32)
    lev, nlev = O.levels(rp, ci)
    assert np.array_equal(lev, want)
    # backward (U) levels mirror the grid
    back = sum(c * (m - 1 - g[i]) for i, c in enumerate(coef)).astype(np.int32)
    ulev, _ = O.levels(rp, ci, upper=True)
    assert np.array_equal(ulev, back)


def test_level_counts_golden():
    gens = {"lap5": lambda m: W.lap5(m), "lap7": lambda m: W.lap7(m),
            "cd27": lambda m: W.cd27(m)[:3], "aniso5": lambda m: W.aniso5(m)}
    for name, m, nlev, wmax, wmed in _read_golden("stencil_levels.txt"):
        m, nlev, wmax, wmed = int(m), int(nlev), int(wmax), int(wmed)
        rp, ci, _ = gens[name](m)
        lev, got = O.levels(rp, ci)
        w = np.bincount(lev)
        assert got == nlev and w.max() == wmax and int(np.median(w)) == wmed


def test_bucket_levels_is_stable_sort():
    rp, ci, _ = W.random_csr(80, 4.0, seed=11)
    lev, nlev = O.levels(rp, ci)
    ptr, rows = O.bucket_levels(lev, nlev)
    assert np.array_equal(rows, np.lexsort((np.arange(80), lev)))
    assert np.array_equal(ptr, np.concatenate([[0], np.cumsum(np.bincount(lev))]))


# --------------------------------------------------------- transpose/permute
def test_transpose_matches_scipy_csc():
    rp, ci, _ = W.random_csr(70, 5.0, seed=4)
    colptr, rowidx, c2c = O.transpose(rp, ci)
    A = _csr(rp, ci, np.arange(len(ci), dtype=np.float64)).tocsc()
    A.sort_indices()
    assert np.array_equal(colptr, A.indptr) and np.array_equal(rowidx, A.indices)
    assert np.array_equal(c2c, A.data.astype(np.int32))


def test_transposed_levels_are_levels_of_transpose():
    rp, ci, _ = W.random_csr(50, 4.0, seed=5)
    At = _csr(rp, ci).T.tocsr()
    At.sort_indices()
    lev_ut, *_ = O.transposed_level_sets(rp, ci, "Ut")
    assert np.array_equal(lev_ut, _nx_generations(At.indptr, At.indices, upper=False))
    lev_lt, *_ = O.transposed_level_sets(rp, ci, "Lt")
    assert np.array_equal(lev_lt, _nx_generations(At.indptr, At.indices, upper=True))


def test_permute_matches_scipy():
    rp, ci, _ = W.random_csr(45, 4.0, seed=6)
    perm = np.random.default_rng(0).permutation(45).astype(np.int32)
    iperm, brp, bci, vmap = O.permute(rp, ci, perm)
    A = _csr(rp, ci, np.arange(len(ci), dtype=np.float64))
    B = A[perm][:, perm].tocsr()
    B.sort_indices()
    assert np.array_equal(iperm[perm], np.arange(45))
    assert np.array_equal(brp, B.indptr) and np.array_equal(bci, B.indices)
    assert np.array_equal(vmap, B.data.astype(np.int32))


# --------------------------------------------------------------------- ILU(0)
def _ilu0_fraction(rp, ci, v):
    """Exact-rational ILU(0) by right-looking (KIJ) Gaussian elimination with
    every update outside the pattern dropped -- a different loop order from
    the oracle's up-looking form; in exact arithmetic they coincide."""
    n = len(rp) - 1
    S = [[False] * n for _ in range(n)]
    A = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            S[i][ci[p]] = True
            A[i][ci[p]] = Fraction(float(v[p]))
    for k in range(n):
        for i in range(k + 1, n):
            if not S[i][k]:
                continue
            A[i][k] = A[i][k] / A[k][k]
            for j in range(k + 1, n):
                if S[i][j] and S[k][j]:
                    A[i][j] -= A[i][k] * A[k][j]
    return [A[i][ci[p]] for i in range(n) for p in range(rp[i], rp[i + 1])]


@pytest.mark.parametrize("seed", range(8))
def test_ilu0_matches_exact_rational_brute_force(seed):
    n = 9 + seed
    rp, ci, v = W.random_csr(n, 3.0 + seed % 3, seed=100 + seed, dominant=(seed % 2 == 0))
    lu, st, _ = O.ilu0(rp, ci, v)
    assert st == O.OK
    exact = _ilu0_fraction(rp, ci, v)
    for got, want in zip(lu, exact):
        assert abs(got - float(want)) <= 1e-12 * max(1.0, abs(float(want)))


@pytest.mark.parametrize("seed", range(4))
def test_ilu0_defining_property_on_pattern(seed):
    rp, ci, v = W.random_csr(120, 5.0, seed=200 + seed)
    lu, st, _ = O.ilu0(rp, ci, v)
    assert st == O.OK
    L, U = _split_lu(rp, ci, lu)
    LU = L @ U
    A = _csr(rp, ci, v).toarray()
    mask = _csr(rp, ci).toarray() > 0
    assert np.allclose(LU[mask], A[mask], rtol=1e-12, atol=1e-12)


def _milu0_fraction(rp, ci, v):
    """Exact-rational modified ILU(0) by right-looking (KIJ) elimination: an
    update outside the pattern lands on the diagonal of its row instead of
    being dropped."""
    n = len(rp) - 1
    S = [[False] * n for _ in range(n)]
    A = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            S[i][ci[p]] = True
            A[i][ci[p]] = Fraction(float(v[p]))
    for k in range(n):
        for i in range(k + 1, n):
            if not S[i][k]:
                continue
            A[i][k] = A[i][k] / A[k][k]
            for j in range(k + 1, n):
                if S[k][j]:
                    if S[i][j]:
                        A[i][j] -= A[i][k] * A[k][j]
                    else:
                        A[i][i] -= A[i][k] * A[k][j]
    return A, [A[i][ci[p]] for i in range(n) for p in range(rp[i], rp[i + 1])]


@pytest.mark.parametrize("seed", range(6))
def test_milu0_matches_exact_rational_and_keeps_row_sums(seed):
    n = 10 + seed
    rp, ci, v = W.random_csr(n, 3.0 + seed % 3, seed=300 + seed, dominant=True)
    lu, st, _ = O.ilu0(rp, ci, v, milu=True)
    assert st == O.OK
    A, exact = _milu0_fraction(rp, ci, v)
    for got, want in zip(lu, exact):
        assert abs(got - float(want)) <= 1e-12 * max(1.0, abs(float(want)))
    # the exact factors keep every row sum of A: (L U) e == A e, exactly
    Ae = [sum(Fraction(float(v[p])) for p in range(rp[i], rp[i + 1])) for i in range(n)]
    usum = [sum(A[k][j] for j in range(k, n)) for k in range(n)]      # row sums of U
    for i in range(n):
        # row i of L U times e = (U e)_i + sum over k < i of l_ik (U e)_k
        lue = usum[i] + sum(A[i][k] * usum[k] for k in range(i))
        assert lue == Ae[i]


@pytest.mark.parametrize("seed", range(3))
def test_milu0_defining_property(seed):
    # off-diagonal pattern entries of L U equal A's; row sums of L U equal A's
    rp, ci, v = W.random_csr(150, 5.0, seed=400 + seed)
    lu, st, _ = O.ilu0(rp, ci, v, milu=True)
    assert st == O.OK
    L, U = _split_lu(rp, ci, lu)
    LU = L @ U
    A = _csr(rp, ci, v).toarray()
    mask = _csr(rp, ci).toarray() > 0
    np.fill_diagonal(mask, False)
    assert np.allclose(LU[mask], A[mask], rtol=1e-12, atol=1e-12)
    assert np.allclose(LU.sum(axis=1), A.sum(axis=1), rtol=1e-11, atol=1e-11)
    plain, _, _ = O.ilu0(rp, ci, v)
    assert not np.array_equal(plain, lu)          # fill-in was dropped, so MILU differs


def test_milu0_equals_ilu0_without_fill():
    # no update ever falls outside a tridiagonal pattern
    n = 200
    rp, ci, v = W.stencil((n, 1, 1), [(-1, 0, 0), (1, 0, 0)], [-1.0, -1.0], 4.0)
    a, _, _ = O.ilu0(rp, ci, v)
    b, _, _ = O.ilu0(rp, ci, v, milu=True)
    assert np.array_equal(a, b)
    a32, _, _ = O.ilu0(rp, ci, v, dtype=np.float32)
    b32, _, _ = O.ilu0(rp, ci, v, dtype=np.float32, milu=True)
    assert np.array_equal(a32, b32)


def test_milu0_f32_twin_close():
    rp, ci, v = W.lap5(12)
    a, _, _ = O.ilu0(rp, ci, v, milu=True)
    b, _, _ = O.ilu0(rp, ci, v, dtype=np.float32, milu=True)
    assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()


# ------------------------------------------------------ ILU(k) symbolic fill
def _fill_path_levels(rp, ci, K):
    """Brute force by the fill-path characterisation (a different algorithm
    from the oracle's row sweep): (i, j) has level of fill L - 1 where L is
    the length of the shortest path i -> j in the graph of A whose
    intermediate vertices are all numbered below min(i, j); keep L - 1 <= K."""
    n = len(rp) - 1
    adj = [list(ci[rp[i]:rp[i + 1]]) for i in range(n)]
    out = {}
    for i in range(n):
        for j in range(n):
            lim = min(i, j)
            dist = {i: 0}
            frontier = [i]
            found = None
            while frontier and found is None:
                nxt = []
                for u in frontier:
                    for w in adj[u]:
                        if w == j:
                            found = dist[u] + 1
                            break
                        if w < lim and w not in dist:
                            dist[w] = dist[u] + 1
                            nxt.append(w)
                    if found is not None:
                        break
                frontier = nxt
            if i == j:
                out[(i, j)] = 0
            elif found is not None and found - 1 <= K:
                out[(i, j)] = found - 1
    return out


@pytest.mark.parametrize("seed", range(6))
def test_iluk_pattern_matches_fill_paths(seed):
    n = 9 + seed
    rp, ci, _ = W.random_csr(n, 2.0 + seed % 3, seed=500 + seed)
    for K in range(4):
        frp, fci, flev = O.iluk_pattern(rp, ci, K)
        got = {(i, int(fci[p])): int(flev[p]) for i in range(n) for p in range(frp[i], frp[i + 1])}
        assert got == _fill_path_levels(rp, ci, K), (seed, K)


def test_iluk_level_zero_is_the_pattern_of_a():
    rp, ci, _ = W.random_csr(300, 5.0, seed=7)
    frp, fci, flev = O.iluk_pattern(rp, ci, 0)
    assert np.array_equal(frp, rp) and np.array_equal(fci, ci) and not flev.any()


def test_iluk_full_fill_is_the_lu_fill_and_exact_lu():
    # with K >= n every fill is kept: the pattern is the no-pivoting LU fill
    # (boolean right-looking elimination) and ILU on it is exact LU
    n = 14
    rp, ci, v = W.random_csr(n, 2.5, seed=77, dominant=True)
    S = np.zeros((n, n), dtype=bool)
    for i in range(n):
        S[i, ci[rp[i]:rp[i + 1]]] = True
    for k in range(n):
        for i in range(k + 1, n):
            if S[i, k]:
                S[i, k + 1:] |= S[k, k + 1:]
    frp, fci, _ = O.iluk_pattern(rp, ci, n)
    F = np.zeros((n, n), dtype=bool)
    for i in range(n):
        F[i, fci[frp[i]:frp[i + 1]]] = True
    assert np.array_equal(F, S)
    fv = O.scatter_values(rp, ci, v, frp, fci)
    lu, st, _ = O.ilu0(frp, fci, fv)
    assert st == O.OK
    A = np.zeros((n, n))
    for i in range(n):
        A[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    # dense Doolittle without pivoting, plain loops
    U = A.copy()
    L = np.eye(n)
    for k in range(n):
        for i in range(k + 1, n):
            L[i, k] = U[i, k] / U[k, k]
            U[i, k:] -= L[i, k] * U[k, k:]
    dense = np.tril(L, -1) + np.triu(U)
    got = np.zeros((n, n))
    for i in range(n):
        got[i, fci[frp[i]:frp[i + 1]]] = lu[frp[i]:frp[i + 1]]
    assert np.allclose(got[F], dense[F], rtol=1e-12, atol=1e-14)


def test_iluk_one_on_5pt_laplacian_adds_the_two_known_diagonals():
    m = 9
    rp, ci, _ = W.lap5(m)
    frp, fci, flev = O.iluk_pattern(rp, ci, 1)
    i = 4 * m + 4                                   # an interior row
    cols = fci[frp[i]:frp[i + 1]] - i
    assert list(cols) == [-m, -m + 1, -1, 0, 1, m - 1, m]
    lv = dict(zip(cols, flev[frp[i]:frp[i + 1]]))
    assert lv[-m + 1] == 1 and lv[m - 1] == 1 and lv[-1] == 0


def test_ilu0_tridiagonal_golden_pivots():
    rows = _read_golden("tridiag_pivots.txt")
    n = len(rows)
    main = np.full(n, 4.0)
    off = np.full(n - 1, -1.0)
    A = sp.diags([off, main, off], [-1, 0, 1], format="csr")
    A.sort_indices()
    lu, st, _ = O.ilu0(A.indptr, A.indices, A.data)
    diag = O.diag_ptr(A.indptr, A.indices)
    for k, num, den in rows:
        want = int(num) / int(den)
        assert abs(lu[diag[int(k)]] - want) <= 2e-16 * want * (int(k) + 1)
    # exact LU agrees (tridiagonal: no fill to drop)
    P, L, U = sla.lu(A.toarray())
    assert np.array_equal(P, np.eye(n))
    Lg, Ug = _split_lu(A.indptr, A.indices, lu)
    assert np.allclose(Lg, L, rtol=1e-14, atol=1e-15) and np.allclose(Ug, U, rtol=1e-14)


def test_ilu0_grid3x3_golden():
    rp, ci, v = W.lap5(3)
    lu, st, _ = O.ilu0(rp, ci, v)
    diag = O.diag_ptr(rp, ci)
    upiv = {}
    for p, x, y, num, den in _read_golden("grid3x3_ilu0.txt"):
        p = int(p)
        upiv[p] = Fraction(int(num), int(den))
        assert abs(lu[diag[p]] - float(upiv[p])) <= 4e-16 * float(upiv[p])
    for i in range(9):
        for q in range(rp[i], rp[i + 1]):
            j = ci[q]
            if j < i:
                assert abs(lu[q] - float(-1 / upiv[j])) <= 4e-16
            elif j > i:
                assert lu[q] == -1.0


@pytest.mark.parametrize("kind", ["dense", "blockdiag"])
def test_ilu0_no_fill_equals_exact_lu(kind):
    rng = np.random.default_rng(7)
    if kind == "dense":
        n = 10
        M = rng.uniform(-1, 1, (n, n))
        M += np.diag(np.abs(M).sum(axis=0) + 1.0)          # column diagonally dominant
        A = sp.csr_matrix(M)
    else:
        blocks = []
        for b in range(4):
            Bk = rng.uniform(-1, 1, (5, 5))
            Bk += np.diag(np.abs(Bk).sum(axis=0) + 1.0)
            blocks.append(Bk)
        A = sp.csr_matrix(sp.block_diag([sp.coo_matrix(b) for b in blocks]))
    A.sort_indices()
    n = A.shape[0]
    P, L, U = sla.lu(A.toarray())
    assert np.array_equal(P, np.eye(n))                     # no pivoting was needed
    lu, st, _ = O.ilu0(A.indptr, A.indices, A.data)
    Lg, Ug = _split_lu(A.indptr, A.indices, lu)
    assert np.allclose(Lg, L, rtol=1e-12, atol=1e-13) and np.allclose(Ug, U, rtol=1e-12, atol=1e-13)


def test_ilu0_triangular_inputs():
    rp, ci, v = W.random_csr(30, 4.0, seed=9, lower_only=True)
    lu, st, _ = O.ilu0(rp, ci, v)
    A = _csr(rp, ci, v).toarray()
    L, U = _split_lu(rp, ci, lu)
    d = np.diag(A)
    assert np.allclose(U, np.diag(d), rtol=0, atol=0)
    assert np.allclose(L, np.tril(A, -1) / d[None, :] + np.eye(30), rtol=1e-15)
    rp, ci, v = W.random_csr(30, 4.0, seed=10, upper_only=True)
    lu, st, _ = O.ilu0(rp, ci, v)
    L, U = _split_lu(rp, ci, lu)
    assert np.array_equal(L, np.eye(30)) and np.array_equal(U, _csr(rp, ci, v).toarray())


def test_ilu0_symmetric_gives_u_equals_d_lt():
    rp, ci, v = W.lap7(5)
    lu, st, _ = O.ilu0(rp, ci, v)
    L, U = _split_lu(rp, ci, lu)
    assert np.allclose(U, np.diag(np.diag(U)) @ L.T, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_ilu0_stencil_pivot_recurrence(dim):
    m = 7
    rp, ci, v = W.lap5(m) if dim == 2 else W.lap7(m)
    d = 4.0 if dim == 2 else 6.0 + 1e-3
    n = m ** dim
    u = np.zeros(n)
    for p in range(n):
        s = d
        for stride in ([1, m] if dim == 2 else [1, m, m * m]):
            # the neighbour at -stride exists when the coordinate is nonzero
            if (p // stride) % m > 0:
                s -= 1.0 / u[p - stride]
        u[p] = s
    lu, st, _ = O.ilu0(rp, ci, v)
    diag = O.diag_ptr(rp, ci)
    assert np.allclose(lu[diag], u, rtol=1e-14)


def test_ilu0_zero_pivot_reported():
    A = sp.csr_matrix(np.array([[1.0, 1.0, 0.0], [1.0, 1.0, 1.0], [0.0, 1.0, 3.0]]))
    A.sort_indices()
    _, st, bad = O.ilu0(A.indptr, A.indices, A.data)
    assert st == O.ERR_ZERO_PIVOT and bad == 1
    A = sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 2.0]]))
    rp, ci = np.array([0, 2, 4]), np.array([0, 1, 0, 1])
    _, st, bad = O.ilu0(rp, ci, np.array([0.0, 1.0, 1.0, 2.0]))
    assert st == O.ERR_ZERO_PIVOT and bad == 0


def test_ilu0_f32_twin_close_to_exact():
    rp, ci, v = W.random_csr(14, 3.0, seed=31)
    lu32, st, _ = O.ilu0(rp, ci, v.astype(np.float32), dtype=np.float32)
    assert st == O.OK and lu32.dtype == np.float32
    exact = _ilu0_fraction(rp, ci, v.astype(np.float32).astype(np.float64))
    for got, want in zip(lu32, exact):
        assert abs(float(got) - float(want)) <= 1e-5 * max(1.0, abs(float(want)))


# --------------------------------------------------------------------- solves
@pytest.mark.parametrize("nrhs", [1, 3])
def test_solves_match_dense_triangular(nrhs):
    rp, ci, v = W.random_csr(60, 4.0, seed=12)
    lu, st, _ = O.ilu0(rp, ci, v)
    diag = O.diag_ptr(rp, ci)
    L, U = _split_lu(rp, ci, lu)
    b = W.rhs(60, nrhs, seed=13)
    assert np.allclose(O.lsolve(rp, ci, diag, lu, b), sla.solve_triangular(L, b, lower=True),
                       rtol=1e-12, atol=1e-13)
    assert np.allclose(O.usolve(rp, ci, diag, lu, b), sla.solve_triangular(U, b, lower=False),
                       rtol=1e-12, atol=1e-13)
    assert np.allclose(O.lsolve_t(rp, ci, diag, lu, b),
                       sla.solve_triangular(L, b, lower=True, trans="T"), rtol=1e-12, atol=1e-13)
    assert np.allclose(O.usolve_t(rp, ci, diag, lu, b),
                       sla.solve_triangular(U, b, lower=False, trans="T"), rtol=1e-12, atol=1e-13)


def test_spmv_matches_scipy():
    rp, ci, v = W.random_csr(90, 6.0, seed=14)
    x = W.rhs(90, 1, seed=15)
    y0 = W.rhs(90, 1, seed=16)
    A = _csr(rp, ci, v)
    assert np.allclose(O.spmv(rp, ci, v, x), A @ x, rtol=1e-14, atol=1e-14)
    assert np.allclose(O.spmv(rp, ci, v, x, y0, alpha=-2.0, beta=0.5), -2.0 * (A @ x) + 0.5 * y0,
                       rtol=1e-14, atol=1e-14)


def test_masked_outer_matches_dense():
    rp, ci, _ = W.random_csr(25, 4.0, seed=17)
    diag = O.diag_ptr(rp, ci)
    a, b = W.rhs(25, 4, seed=18), W.rhs(25, 4, seed=19)
    full = a @ b.T
    mask = _csr(rp, ci, np.arange(len(ci), dtype=np.float64) + 1).toarray()
    gl = O.masked_outer(rp, ci, diag, 0, a, b, alpha=-1.0)
    gu = O.masked_outer(rp, ci, diag, 1, a, b, alpha=-1.0)
    for i in range(25):
        for p in range(rp[i], rp[i + 1]):
            j = ci[p]
            want = -full[i, j]
            if j < i:
                assert abs(gl[p] - want) < 1e-14 and gu[p] == 0.0
            else:
                assert abs(gu[p] - want) < 1e-14 and gl[p] == 0.0
    assert mask.shape == (25, 25)


def test_adjoint_matches_torch_autograd():
    """z = U^-1 L^-1 r; the oracle's adjoint (transposed solves + masked
    outer products) must equal dense autograd restricted to the pattern."""
    torch = pytest.importorskip("torch")
    rp, ci, v = W.random_csr(30, 4.0, seed=20)
    lu, _, _ = O.ilu0(rp, ci, v)
    diag = O.diag_ptr(rp, ci)
    r = W.rhs(30, 3, seed=21)
    gz = W.rhs(30, 3, seed=22)
    Ld, Ud = _split_lu(rp, ci, lu)
    Lt = torch.tensor(np.tril(Ld, -1), dtype=torch.float64, requires_grad=True)
    Ut = torch.tensor(Ud, dtype=torch.float64, requires_grad=True)
    rt = torch.tensor(r, dtype=torch.float64, requires_grad=True)
    eye = torch.eye(30, dtype=torch.float64)
    y = torch.linalg.solve_triangular(Lt + eye, rt, upper=False, unitriangular=True)
    z = torch.linalg.solve_triangular(Ut, y, upper=True)
    (z * torch.tensor(gz)).sum().backward()
    yo = O.lsolve(rp, ci, diag, lu, r)
    zo = O.usolve(rp, ci, diag, lu, yo)
    assert np.allclose(zo, z.detach().numpy(), rtol=1e-12, atol=1e-13)
    gy = O.usolve_t(rp, ci, diag, lu, gz)
    gr = O.lsolve_t(rp, ci, diag, lu, gy)
    assert np.allclose(gr, rt.grad.numpy(), rtol=1e-12, atol=1e-13)
    g = O.masked_outer(rp, ci, diag, 0, gr, yo, -1.0) + O.masked_outer(rp, ci, diag, 1, gy, zo, -1.0)
    gl_dense, gu_dense = Lt.grad.numpy(), Ut.grad.numpy()
    for i in range(30):
        for p in range(rp[i], rp[i + 1]):
            j = ci[p]
            want = gl_dense[i, j] if j < i else gu_dense[i, j]
            assert abs(g[p] - want) <= 1e-12 * max(1.0, abs(want))


# --------------------------------------------------------------------- Krylov
def test_pcg_exact_preconditioner_one_iteration():
    n = 50
    A = sp.diags([np.full(n - 1, -1.0), np.full(n, 4.0), np.full(n - 1, -1.0)], [-1, 0, 1],
                 format="csr")
    A.sort_indices()
    lu, _, _ = O.ilu0(A.indptr, A.indices, A.data)
    b = W.rhs(n, 1, seed=23)
    x, it, rel = O.pcg(A.indptr, A.indices, A.data, lu, b, tol=1e-12)
    assert it == 1 and rel < 1e-13
    x, it, rel = O.fgmres(A.indptr, A.indices, A.data, lu, b, tol=1e-12)
    assert it == 1 and rel < 1e-13


def test_pcg_matches_scipy_cg_iterations_and_solution():
    rp, ci, v = W.lap5(24)
    A = _csr(rp, ci, v)
    lu, _, _ = O.ilu0(rp, ci, v)
    diag = O.diag_ptr(rp, ci)
    b = W.rhs(A.shape[0], 1, seed=24)
    x, it, rel = O.pcg(rp, ci, v, lu, b, tol=1e-8)
    assert rel <= 1e-8
    xs = spla.spsolve(A.tocsc(), b)
    assert np.allclose(x, xs, rtol=1e-6, atol=1e-7)
    count = [0]
    M = spla.LinearOperator(A.shape, matvec=lambda r: O.usolve(rp, ci, diag, lu,
                                                              O.lsolve(rp, ci, diag, lu, r)))
    spla.cg(A, b, rtol=1e-8, atol=0.0, M=M, callback=lambda xk: count.__setitem__(0, count[0] + 1))
    assert abs(count[0] - it) <= 1


def test_fgmres_minimises_residual_over_krylov_space():
    rp, ci, v, _ = W.cd27(4)
    A = _csr(rp, ci, v).toarray()
    n = A.shape[0]
    lu, _, _ = O.ilu0(rp, ci, v)
    diag = O.diag_ptr(rp, ci)
    b = W.rhs(n, 1, seed=25)
    Minv = lambda r: O.usolve(rp, ci, diag, lu, O.lsolve(rp, ci, diag, lu, r))
    for k in (1, 2, 4, 6):
        _, it, rel = O.fgmres(rp, ci, v, lu, b, m=k, tol=0.0, max_restarts=1)
        # brute force: min over y in K_k(A M^-1, b) of ||b - A M^-1 y||
        K = [b.copy()]
        for _ in range(k - 1):
            K.append(A @ Minv(K[-1]))
        K = np.stack(K, axis=1)
        Q, _ = np.linalg.qr(K)
        AMQ = np.stack([A @ Minv(Q[:, t]) for t in range(k)], axis=1)
        c, *_ = np.linalg.lstsq(AMQ, b, rcond=None)
        best = np.linalg.norm(b - AMQ @ c) / np.linalg.norm(b)
        assert abs(rel - best) <= 1e-9 * max(best, 1e-3)


def test_fgmres_solution_nonsymmetric():
    rp, ci, v, _ = W.cd27(6)
    A = _csr(rp, ci, v)
    lu, _, _ = O.ilu0(rp, ci, v)
    b = W.rhs(A.shape[0], 1, seed=26)
    x, it, rel = O.fgmres(rp, ci, v, lu, b, m=30, tol=1e-10)
    assert it > 0 and rel <= 1e-10
    assert np.allclose(x, spla.spsolve(A.tocsc(), b), rtol=1e-8, atol=1e-9)


def test_solve_scale_bounds_other_summation_orders():
    # the scale the GPU tests measure tree-summed solve rows against: a
    # forward substitution that adds each row's terms in another order (here
    # reversed, in plain Python) stays within a few eps of the serial one
    # relative to s = (|I - N|)^-1 |b|, even where the result itself cancels
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from jvutil import close_scaled, solve_scale
    rp, ci, v = W.random_csr(300, 12.0, seed=91, dominant=False)
    diag = O.diag_ptr(rp, ci)
    lu, st, _ = O.ilu0(rp, ci, v, diag)
    if st != O.OK:
        lu = v.copy()
    b = W.rhs(300, 1, seed=92)
    x = O.lsolve(rp, ci, diag, lu, b)
    y = np.zeros(300)
    for r in range(300):
        s = 0.0
        for q in range(diag[r] - 1, rp[r] - 1, -1):
            s += lu[q] * y[ci[q]]
        y[r] = b[r] - s
    scale = solve_scale(O.lsolve, rp, ci, diag, lu, b)
    assert np.all(scale >= np.abs(x) * (1 - 1e-12))
    ok, err = close_scaled(y, x, scale, rel=1e-13)
    assert ok, err


def test_spmv_scale_bounds_lane_and_tree_order():
    # the criterion the GPU tests apply to spmv rows summed by lanes and a
    # tree: each of 32 lanes adds its share (entries l, l + 32, ...) in
    # order, then a butterfly adds the partial sums.  That order stays within
    # a few eps of the serial oracle relative to sum |a_rj x_j|, while a
    # dropped term does not
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from jvutil import close_scaled
    rp, ci, v = W.powerlaw(3000, kmin=4, kmax=1500, mean=40, seed_pattern=41, seed_values=42)
    n = len(rp) - 1
    x = W.rhs(n, 1, seed=43)
    want = O.spmv(rp, ci, v, x)
    scale = O.spmv(rp, ci, np.abs(v), np.abs(x))
    got = np.empty(n)
    dropped = want.copy()
    for r in range(n):
        part = [0.0] * 32
        for q in range(rp[r], rp[r + 1]):
            part[(q - rp[r]) % 32] += v[q] * x[ci[q]]
        o = 16
        while o:
            part = [part[l] + part[l ^ o] for l in range(32)]
            o >>= 1
        got[r] = part[0]
        if rp[r + 1] - rp[r] > 128:
            dropped[r] = want[r] - v[rp[r]] * x[ci[rp[r]]]
    assert (np.diff(rp) > 128).sum() > 50
    ok, err = close_scaled(got, want, scale, rel=1e-13)
    assert ok, err
    assert not close_scaled(dropped, want, scale)[0]


def _fma(a, b, c):
    # one correctly rounded a*b + c: exact rational arithmetic, then a single
    # rounding (Fraction -> float rounds to nearest)
    from fractions import Fraction
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def test_factor_diagonal_tree_order_within_bound():
    # the default FP64 factor sums a hub row's diagonal updates (more than 32)
    # over 32 lanes and a butterfly.  On a power-law matrix: the oracle's
    # diagonal is the serial chain of fused multiply-adds over its final l_ik
    # and u_ki (bit for bit), the lane-and-tree order stays within the 1e-12
    # bound the GPU tests apply, and a dropped update does not
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from jvutil import close
    rp, ci, v = W.powerlaw(800, kmin=4, kmax=300, mean=24, seed_pattern=51, seed_values=52)
    n = len(rp) - 1
    diag = O.diag_ptr(rp, ci)
    lu, st, _ = O.ilu0(rp, ci, v, diag)
    assert st == O.OK
    pos = [dict(zip(ci[rp[r]:rp[r + 1]].tolist(), range(rp[r], rp[r + 1]))) for r in range(n)]
    serial, tree, dropped = lu.copy(), lu.copy(), lu.copy()
    hubs = 0
    for r in range(n):
        terms = [(lu[p], lu[pos[k][r]]) for p, k in zip(range(rp[r], diag[r]), ci[rp[r]:diag[r]])
                 if r in pos[k]]
        d = v[diag[r]]
        for l, u in terms:
            d = _fma(-l, u, d)
        serial[diag[r]] = d
        if len(terms) > 32:
            hubs += 1
            part = [0.0] * 32
            for t, (l, u) in enumerate(terms):
                part[t % 32] = _fma(-l, u, part[t % 32])
            o = 16
            while o:
                part = [part[i] + part[i ^ o] for i in range(32)]
                o >>= 1
            tree[diag[r]] = v[diag[r]] + part[0]
            dropped[diag[r]] = tree[diag[r]] + terms[0][0] * terms[0][1]
    assert hubs > 20
    assert np.array_equal(serial, lu)
    ok, err = close(tree, lu)
    assert ok, err
    assert not close(dropped, lu)[0]
