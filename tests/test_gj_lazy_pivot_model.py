"""Host model of the blocked Gauss-Jordan inversion that the FP32 look-ahead kernel runs
(batched block inverses of the block-cyclic-reduction factor).

The kernel never swaps rows: the pivot of column k is the physical row piv[k] with the
largest |re| + |im| among the rows not yet used (ties to the lowest row), each panel of
16 columns is reduced in place, the other columns get the panel's rank-16 update with the
panel's pivot rows starting from zero, and the inverse is written out as
M[piv[i]][pinv[j]] of the in-place result M.  These tests check that identity against
numpy's inverse, and that the numbers equal those of the same algorithm with explicit
row swaps whenever no two pivot candidates tie."""
import numpy as np
import pytest

NB = 16


def _cabs1(z):
    return np.abs(z.real) + np.abs(z.imag)


def gj_recorded_pivots(A, nb=NB):
    """Blocked in-place Gauss-Jordan with recorded pivot rows; returns (inverse, singular)."""
    n = A.shape[0]
    a = A.astype(np.complex128).copy()
    used = np.zeros(n, bool)
    piv = np.zeros(n, int)
    rowpanel = np.full(n, -1)
    singular = False
    for c0 in range(0, n, nb):
        w = min(nb, n - c0)
        cols = np.arange(c0, c0 + w)
        for kt in range(w):
            k = c0 + kt
            cand = np.where(used, -1.0, _cabs1(a[:, k]))
            p = int(np.argmax(cand))                    # first maximum: lowest row on ties
            singular |= cand[p] <= 0
            used[p] = True
            piv[k] = p
            rowpanel[p] = c0
            col = a[:, k].copy()
            pinv = 1.0 / col[p] if col[p] != 0 else 0.0
            rk = a[p, cols] * pinv
            rk[kt] = pinv
            others = np.arange(n) != p
            a[np.ix_(others, cols)] -= np.outer(col[others], rk)
            a[others, k] = -col[others] * pinv
            a[p, cols] = rk
        rest = np.r_[0:c0, c0 + w:n]
        if rest.size:
            T = a[np.ix_(piv[c0:c0 + w], rest)].copy()
            base = a[:, rest].copy()
            base[rowpanel == c0] = 0
            a[:, rest] = base + a[:, cols] @ T
    pinv_perm = np.argsort(piv)
    return a[piv][:, pinv_perm], singular


def gj_explicit_swaps(A):
    """Unblocked Gauss-Jordan with row swaps and the final column permutation."""
    n = A.shape[0]
    a = A.astype(np.complex128).copy()
    perm = np.zeros(n, int)
    for k in range(n):
        p = k + int(np.argmax(_cabs1(a[k:, k])))
        perm[k] = p
        a[[k, p]] = a[[p, k]]
        # the same array expressions as gj_recorded_pivots (numpy's loops round alike)
        col = a[:, k].copy()
        pinv = 1.0 / col[k]
        rk = a[k, :] * pinv
        rk[k] = pinv
        others = np.arange(n) != k
        a[np.ix_(others, np.arange(n))] -= np.outer(col[others], rk)
        a[others, k] = -col[others] * pinv
        a[k, :] = rk
    idx = np.arange(n)
    for k in range(n - 1, -1, -1):
        idx[[k, perm[k]]] = idx[[perm[k], k]]
    return a[:, idx]


def _random(n, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))


@pytest.mark.parametrize("n", [1, 2, 7, 16, 17, 31, 32, 50, 100, 150, 160])
def test_recorded_pivots_give_the_inverse(n):
    A = _random(n, n)
    X, singular = gj_recorded_pivots(A)
    assert not singular
    assert np.allclose(X @ A, np.eye(n), atol=1e-9 * n)


@pytest.mark.parametrize("n", [5, 16, 40, 160])
def test_recorded_pivots_equal_explicit_swaps_without_ties(n):
    # a block of the kind the factorisation inverts: strong diagonal, unit coupling, noise
    rng = np.random.default_rng(100 + n)
    A = 5 * (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    A += np.diag(np.full(n, -1600.0 + 3j)) + 400.0 * (np.eye(n, k=1) + np.eye(n, k=-1))
    X1, _ = gj_recorded_pivots(A, nb=1 << 30)      # one panel: the unblocked order of updates
    X2 = gj_explicit_swaps(A)
    assert np.array_equal(X1, X2)
    X3, _ = gj_recorded_pivots(A)
    assert np.allclose(X3, X2, rtol=0, atol=1e-12 * np.abs(X2).max())


def test_ties_go_to_the_lowest_unused_row():
    # every column of a permutation matrix times a constant has one candidate; equal
    # magnitudes in column 0 (rows 1 and 3) must pick row 1
    A = np.array([[0, 1, 0, 0], [2, 0, 0, 0], [0, 0, 1, 0], [2j, 0, 0, 1]], complex)
    X, singular = gj_recorded_pivots(A)
    assert not singular
    assert np.allclose(X @ A, np.eye(4))


def test_singular_block_is_flagged():
    A = _random(20, 3)
    A[:, 7] = 0
    _, singular = gj_recorded_pivots(A)
    assert singular
