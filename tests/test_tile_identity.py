"""Host checks of the Hermitian tile decomposition the direct form's tile pass
uses (Section III-B's direct branch, u_b = L_b q_b with L_b = (H_b^H H_b + rho I)^{-1}
Hermitian).  With L cut into 64 x 64 tiles and only the lower triangle kept,

    u_I = sum_{J <= I} L_IJ q_J + sum_{I' > I} L_I'I^H q_I',

and the pass visits tiles tile column by tile column (then block, then tile
row).  These tests restate that identity and that order in numpy; they need no
GPU and touch neither the oracle nor the library."""

import numpy as np
import pytest

T = 64


def hermitian_pd(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((2 * n, n)) + 1j * rng.standard_normal((2 * n, n))
    return np.linalg.inv(A.conj().T @ A + 0.5 * np.eye(n))


def tiled_apply(L, q):
    """u = L q from the lower-triangle tiles only: each tile's row sums and,
    below the diagonal, its column sums, added per row in tile order."""
    n = L.shape[0]
    NT = -(-n // T)
    Lp = np.zeros((NT * T, NT * T), dtype=complex)
    Lp[:n, :n] = np.tril(L)            # the tiles hold the lower triangle (diagonal tiles whole)
    for I in range(NT):                # diagonal tiles are kept whole
        Lp[I * T:(I + 1) * T, I * T:(I + 1) * T] = 0
        blk = L[I * T:min((I + 1) * T, n), I * T:min((I + 1) * T, n)]
        Lp[I * T:I * T + blk.shape[0], I * T:I * T + blk.shape[1]] = blk
    qp = np.zeros(NT * T, dtype=complex)
    qp[:n] = q
    RP, CP = {}, {}
    for I in range(NT):
        for J in range(I + 1):
            tile = Lp[I * T:(I + 1) * T, J * T:(J + 1) * T]
            RP[I, J] = tile @ qp[J * T:(J + 1) * T]
            if J < I:
                CP[I, J] = tile.conj().T @ qp[I * T:(I + 1) * T]
    u = np.zeros(NT * T, dtype=complex)
    for X in range(NT):
        acc = np.zeros(T, dtype=complex)
        for k in range(NT):            # fixed order: row sums of (X, k <= X), then column sums of (k > X, X)
            acc += RP[X, k] if k <= X else CP[k, X]
        u[X * T:(X + 1) * T] = acc
    return u[:n]


@pytest.mark.parametrize("n,seed", [(64, 1), (200, 2), (257, 3), (1030, 4)])
def test_lower_triangle_tiles_reproduce_the_full_product(n, seed):
    L = hermitian_pd(n, seed)
    assert np.allclose(L, L.conj().T, atol=1e-12)
    q = np.random.default_rng(seed + 10).standard_normal(n) + 1j * np.random.default_rng(seed + 20).standard_normal(n)
    u = tiled_apply(L, q)
    assert np.linalg.norm(u - L @ q) <= 1e-12 * np.linalg.norm(L @ q)


def test_dropping_the_column_sums_breaks_the_identity():
    """The column sums (the conjugate-transposed tiles) are what makes half the
    bytes enough: without them u is the product with tril(L) only."""
    n = 200
    L = hermitian_pd(n, 5)
    q = np.ones(n, dtype=complex)
    NT = -(-n // T)
    u_rows_only = np.zeros(n, dtype=complex)
    for I in range(NT):
        for J in range(I + 1):
            r0, r1 = I * T, min((I + 1) * T, n)
            c0, c1 = J * T, min((J + 1) * T, n)
            u_rows_only[r0:r1] += L[r0:r1, c0:c1] @ q[c0:c1]
    assert np.linalg.norm(u_rows_only - L @ q) > 1e-3 * np.linalg.norm(L @ q)


def pass_order(nts):
    """(p, I, J) in the tile pass's order for blocks with nts[p] tile panels."""
    return [(p, I, J) for J in range(max(nts)) for p in range(len(nts)) for I in range(J, nts[p])]


@pytest.mark.parametrize("nts", [[32] * 8, [4, 4, 4], [5, 3, 7], [1]])
def test_pass_order_visits_every_tile_once_and_completes_panels_in_order(nts):
    order = pass_order(nts)
    want = {(p, I, J) for p, nt in enumerate(nts) for I in range(nt) for J in range(I + 1)}
    assert len(order) == len(want) and set(order) == want
    # panel X of block p needs tiles (X, J <= X) and (I > X, X): all of them
    # come no later than the last tile of tile column X
    last_of_column = {}
    for pos, (p, I, J) in enumerate(order):
        last_of_column[J] = pos
    for p, nt in enumerate(nts):
        for X in range(nt):
            need = [(p, X, J) for J in range(X + 1)] + [(p, I, X) for I in range(X + 1, nt)]
            assert max(order.index(t) for t in need) <= last_of_column[X]
