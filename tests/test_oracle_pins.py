"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these tests compares the oracle with itself: each side of every
assertion comes from a closed form, a printed number of the paper, a textbook
solver of a different kind (dense LAPACK solve, QR least squares, FISTA), or
brute-force enumeration.
"""

import itertools
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import admm_fp64 as A

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_c(rng, shape, scale=1.0):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * scale


def shrink_independent(a, t):
    """Complex shrinkage written as a * max(0, 1 - t/|a|) (textbook prox of t|.|)."""
    a = np.asarray(a, dtype=np.complex128)
    mag = np.abs(a)
    with np.errstate(divide="ignore", invalid="ignore"):
        scale = np.where(mag > t, 1.0 - t / np.where(mag > 0, mag, 1.0), 0.0)
    return a * scale


def fista(H, g, lam, iters=20000, tol=1e-15):
    """FISTA (Beck & Teboulle) for min 1/2||Hu - g||^2 + lam ||u||_1 over C^n."""
    L = np.linalg.norm(H, 2) ** 2
    x = np.zeros(H.shape[1], dtype=np.complex128)
    y, t = x.copy(), 1.0
    for _ in range(iters):
        grad = H.conj().T @ (H @ y - g)
        x_new = shrink_independent(y - grad / L, lam / L)
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        y = x_new + ((t - 1.0) / t_new) * (x_new - x)
        if np.linalg.norm(x_new - x) <= tol * max(1.0, np.linalg.norm(x_new)):
            x = x_new
            break
        x, t = x_new, t_new
    return x


def kkt_violation(H, g, v, lam):
    """Complex lasso optimality: c = H^*(g - Hv); c_k = lam v_k/|v_k| on the
    support, |c_k| <= lam off it.  Returns the largest violation / lam."""
    c = H.conj().T @ (g - H @ v)
    on = np.abs(v) > 0
    viol_on = np.abs(c[on] - lam * v[on] / np.abs(v[on])) if on.any() else np.zeros(1)
    viol_off = np.maximum(np.abs(c[~on]) - lam, 0.0) if (~on).any() else np.zeros(1)
    return float(max(viol_on.max(), viol_off.max()) / lam)


def small_problem(m=20, n=48, nnz=4, seed=3, rho=1.0, lam_frac=0.1):
    return synth.gaussian_problem(m, n, nnz, seed, lam_frac=lam_frac, rho=rho, c64=False)


SPLITS = [(1, 1), (2, 1), (4, 1), (1, 2), (1, 3), (2, 2), (3, 2)]


# ----------------------------------------------------------------------------
# soft-threshold, Eq. (softhresholding)
# ----------------------------------------------------------------------------

def test_soft_threshold_golden_values():
    rows = np.loadtxt(os.path.join(GOLDEN, "soft_threshold.txt"), comments="#")
    for re_a, im_a, kappa, re_s, im_s in rows:
        out = oracle.soft_threshold(np.array([re_a + 1j * im_a]), kappa)[0]
        assert abs(out - (re_s + 1j * im_s)) <= 1e-12, (re_a, im_a, kappa, out)


def test_soft_threshold_is_the_prox_of_the_modulus():
    """S_kappa(a) = argmin_x kappa|x| + 1/2|x - a|^2; checked on a dense grid."""
    rng = np.random.default_rng(0)
    grid = np.linspace(-3, 3, 601)
    X = grid[:, None] + 1j * grid[None, :]
    for _ in range(20):
        a = complex(*rng.uniform(-2, 2, 2))
        kappa = float(rng.uniform(0, 2))
        obj = kappa * np.abs(X) + 0.5 * np.abs(X - a) ** 2
        best = X.ravel()[np.argmin(obj)]
        assert abs(oracle.soft_threshold(np.array([a]), kappa)[0] - best) <= 0.011


def test_soft_threshold_keeps_phase_and_shrinks_modulus():
    rng = np.random.default_rng(1)
    a = _rand_c(rng, 1000, 2.0)
    kappa = 0.7
    out = oracle.soft_threshold(a, kappa)
    big = np.abs(a) > kappa
    assert np.allclose(np.abs(out[big]), np.abs(a[big]) - kappa, rtol=0, atol=1e-14)
    assert np.allclose(np.angle(out[big]), np.angle(a[big]), atol=1e-12)
    assert np.all(out[~big] == 0)


# ----------------------------------------------------------------------------
# u-step: inversion lemma vs a dense solve, Eq. (inversion_lemma)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("rows,cols,rho", [(8, 64, 1.0), (30, 200, 0.05), (64, 70, 17.0),
                                           (12, 12, 2.0), (40, 16, 0.5)])
def test_block_solver_matches_dense_solve(rows, cols, rho):
    rng = np.random.default_rng(rows * 1000 + cols)
    Hb = _rand_c(rng, (rows, cols), 1 / np.sqrt(rows))
    q = _rand_c(rng, cols)
    dense = np.linalg.solve(Hb.conj().T @ Hb + rho * np.eye(cols), q)
    sv = A.BlockSolver(Hb, rho)
    assert sv.lemma == (rows < cols)
    got = sv.solve(q)
    assert np.linalg.norm(got - dense) <= 1e-12 * np.linalg.norm(dense)


# ----------------------------------------------------------------------------
# one iteration of every split against a QR least-squares u-step
# ----------------------------------------------------------------------------

def _blocks_of(res, m, n, M, N):
    rows = A.balanced_blocks(m, M)
    cols = A.balanced_blocks(n, N)
    return rows, cols


def _ls_step(Hb, target, z, rho):
    """argmin_u 1/2||Hb u - target||^2 + rho/2||u - z||^2 via lstsq of the stacked system."""
    k = Hb.shape[1]
    Aug = np.vstack([Hb, np.sqrt(rho) * np.eye(k)])
    rhs = np.concatenate([target, np.sqrt(rho) * z])
    return np.linalg.lstsq(Aug, rhs, rcond=None)[0]


@pytest.mark.parametrize("M,N", SPLITS)
@pytest.mark.parametrize("k", [0, 1, 7])
@pytest.mark.parametrize("mn", [(20, 48), (60, 12)])   # wide blocks (lemma) and tall ones (direct)
def test_one_iteration_matches_least_squares_step(M, N, k, mn):
    """From the oracle's state after k iterations, iteration k+1 must be:
    u-step = the prox-regularised least squares of Sections III-A..C with the
    estimated data of the *previous* iterate; v-step = shrinkage of the replica
    means with kappa = lam/(M rho); dual step s + u - v.  On the 60 x 12
    problem every block has at least as many rows as columns, so the oracle
    takes its direct branch throughout."""
    if mn[1] < N:
        pytest.skip("more column blocks than columns")
    p = small_problem(m=mn[0], n=mn[1], nnz=3, rho=3.0 * (N if N > 1 else 1))
    m, n = p.H.shape
    H, g = p.H, p.g
    before = oracle.run_split(H, g, M, N, p.lam, p.rho, k)
    after = oracle.run_split(H, g, M, N, p.lam, p.rho, k + 1)
    rows, cols = _blocks_of(before, m, n, M, N)
    if k == 0:
        v0 = np.zeros(n, complex); s0 = np.zeros((M, n), complex); u0 = np.zeros((M, n), complex)
    else:
        v0, s0, u0 = before.v, before.s, before.u
    u1 = np.zeros((M, n), complex)
    for i, (r0, r1) in enumerate(rows):
        for j, (c0, c1) in enumerate(cols):
            target = g[r0:r1].copy()
            for q, (d0, d1) in enumerate(cols):
                if q != j:
                    target -= H[r0:r1, d0:d1] @ u0[i, d0:d1]
            z = v0[c0:c1] - s0[i, c0:c1]
            u1[i, c0:c1] = _ls_step(H[r0:r1, c0:c1], target, z, p.rho)
    assert np.linalg.norm(after.u - u1) <= 1e-10 * max(1.0, np.linalg.norm(u1))
    kappa = p.lam / (M * p.rho)
    v1 = shrink_independent(u1.mean(axis=0) + s0.mean(axis=0), kappa)
    assert np.linalg.norm(after.v - v1) <= 1e-10 * max(1.0, np.linalg.norm(v1))
    s1 = s0 + u1 - v1[None, :]
    assert np.linalg.norm(after.s - s1) <= 1e-10 * max(1.0, np.linalg.norm(s1))
    # residual vectors as stacked in Sections III-A..C, then their squared norms
    r_p = np.concatenate([u1[i] - v1 for i in range(M)])
    r_d = np.concatenate([-p.rho * (v1 - v0) for _ in range(M)])
    rec = after.hist[-1]
    assert abs(rec[0] - np.vdot(r_p, r_p).real) <= 1e-9 * max(1.0, rec[0])
    assert abs(rec[1] - np.vdot(r_d, r_d).real) <= 1e-9 * max(1.0, rec[1])


def test_estimated_data_is_blockwise_product():
    """ghat returned for the column splits equals H_iq u_q^i of the final iterate (Eq. g_columns)."""
    p = small_problem()
    for M, N in [(1, 3), (2, 2)]:
        r = oracle.run_split(p.H, p.g, M, N, p.lam, 6.0, 5)
        rows = A.balanced_blocks(p.m, M)
        cols = A.balanced_blocks(p.n, N)
        for i, (r0, r1) in enumerate(rows):
            for q, (c0, c1) in enumerate(cols):
                want = p.H[r0:r1, c0:c1] @ r.u[i, c0:c1]
                assert np.allclose(r.ghat[q, r0:r1], want, rtol=0, atol=1e-12)


# ----------------------------------------------------------------------------
# structure: M = N = 1, and the reductions between splits
# ----------------------------------------------------------------------------

def test_unsplit_case_is_identical_across_all_four_code_paths():
    p = small_problem()
    ref = A.lasso_admm(p.H, p.g, p.lam, p.rho, 40)
    for fn in (lambda: A.consensus_admm(p.H, p.g, 1, p.lam, p.rho, 40),
               lambda: A.sectioning_admm(p.H, p.g, 1, p.lam, p.rho, 40),
               lambda: A.cs_admm(p.H, p.g, 1, 1, p.lam, p.rho, 40)):
        r = fn()
        assert np.array_equal(r.v, ref.v)
        assert np.array_equal(r.s, ref.s)
        assert np.array_equal(r.hist, ref.hist)


def test_cs_reduces_to_consensus_and_sectioning():
    p = small_problem()
    a = A.cs_admm(p.H, p.g, 3, 1, p.lam, p.rho, 25)
    b = A.consensus_admm(p.H, p.g, 3, p.lam, p.rho, 25)
    assert np.allclose(a.v, b.v, rtol=0, atol=1e-12) and np.allclose(a.hist, b.hist, rtol=1e-10)
    a = A.cs_admm(p.H, p.g, 1, 3, p.lam, 9.0, 25)
    b = A.sectioning_admm(p.H, p.g, 3, p.lam, 9.0, 25)
    assert np.allclose(a.v, b.v, rtol=0, atol=1e-12) and np.allclose(a.hist, b.hist, rtol=1e-10)


def test_block_diagonal_columns_decouple_sectioning():
    """If H = blockdiag(H_1, H_2) by rows and columns, the column split is two
    independent unsplit lasso ADMMs (H_1^* H_2 = 0 makes the estimated data of
    the other block invisible to each u-step)."""
    rng = np.random.default_rng(5)
    H1 = _rand_c(rng, (6, 20), 0.4); H2 = _rand_c(rng, (6, 20), 0.4)
    H = np.zeros((12, 40), complex); H[:6, :20] = H1; H[6:, 20:] = H2
    g = _rand_c(rng, 12)
    lam, rho = 0.2, 2.0
    sec = A.sectioning_admm(H, g, 2, lam, rho, 60)
    r1 = A.lasso_admm(H1, g[:6], lam, rho, 60)
    r2 = A.lasso_admm(H2, g[6:], lam, rho, 60)
    assert np.allclose(sec.v, np.concatenate([r1.v, r2.v]), rtol=0, atol=1e-12)


# ----------------------------------------------------------------------------
# fixed point: every split reaches the lasso minimiser
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("M,N", SPLITS)
def test_every_split_converges_to_the_lasso_minimiser(M, N):
    p = small_problem(m=16, n=40, nnz=3, seed=11, lam_frac=0.15)
    ref = fista(p.H, p.g, p.lam)
    assert kkt_violation(p.H, p.g, ref, p.lam) < 1e-9
    rho = 1.0 if N == 1 else N * max(np.linalg.norm(p.H[:, c0:c1], 2) ** 2
                                     for c0, c1 in A.balanced_blocks(p.n, N))
    r = oracle.run_split(p.H, p.g, M, N, p.lam, rho, 20000, eps=(1e-13, 1e-12))
    assert r.stopped_at is not None
    assert np.linalg.norm(r.v - ref) <= 1e-8 * np.linalg.norm(ref)
    assert kkt_violation(p.H, p.g, r.v, p.lam) < 1e-7
    assert np.array_equal(np.abs(r.v) > 0, np.abs(ref) > 1e-12)


def test_diagonal_sensing_matrix_has_closed_form():
    """H = diag(h): the lasso decouples, u_k = S_{lam/|h_k|^2}(g_k / h_k)."""
    rng = np.random.default_rng(7)
    n = 24
    h = _rand_c(rng, n)
    H = np.diag(h)
    g = _rand_c(rng, n)
    lam = 0.6
    want = np.array([A.soft_threshold(np.array([g[k] / h[k]]), lam / abs(h[k]) ** 2)[0]
                     for k in range(n)])
    # independent form of the same closed form
    want2 = shrink_independent(g / h, lam / np.abs(h) ** 2)
    assert np.allclose(want, want2, rtol=0, atol=1e-14)
    for M, N in [(2, 1), (1, 2), (2, 2), (3, 1)]:
        rho = 1.0 if N == 1 else N * np.max(np.abs(h)) ** 2
        r = oracle.run_split(H, g, M, N, lam, rho, 20000, eps=(1e-14, 1e-13))
        assert np.allclose(r.v, want2, rtol=0, atol=1e-9), (M, N)


def test_identity_sensing_matrix_gives_plain_shrinkage():
    rng = np.random.default_rng(8)
    n = 30
    g = _rand_c(rng, n)
    lam = 0.8
    for M, N in [(1, 1), (3, 1), (1, 3), (3, 3)]:
        rho = 1.0 if N == 1 else 1.0 * N
        r = oracle.run_split(np.eye(n, dtype=complex), g, M, N, lam, rho, 20000,
                             eps=(1e-14, 1e-13))
        assert np.allclose(r.v, shrink_independent(g, lam), rtol=0, atol=1e-9), (M, N)


def _bruteforce_real_lasso(H, g, lam):
    """Enumerate every sign pattern in {-1,0,1}^n; return the unique KKT point."""
    m, n = H.shape
    sols = []
    for pattern in itertools.product((-1, 0, 1), repeat=n):
        sig = np.array(pattern, dtype=float)
        S = np.flatnonzero(sig)
        u = np.zeros(n)
        if S.size:
            if S.size > m:
                continue
            HS = H[:, S]
            G = HS.T @ HS
            if np.linalg.cond(G) > 1e10:
                continue
            uS = np.linalg.solve(G, HS.T @ g - lam * sig[S])
            if np.any(np.sign(uS) != sig[S]):
                continue
            u[S] = uS
        c = H.T @ (g - H @ u)
        off = np.setdiff1d(np.arange(n), S)
        if off.size and np.any(np.abs(c[off]) > lam * (1 + 1e-12)):
            continue
        sols.append(u)
    return sols


def test_tiny_real_instance_matches_bruteforce_lasso():
    rng = np.random.default_rng(21)
    m, n = 5, 8
    H = rng.standard_normal((m, n)) / np.sqrt(m)
    g = rng.standard_normal(m)
    lam = 0.25 * np.max(np.abs(H.T @ g))
    sols = _bruteforce_real_lasso(H, g, lam)
    assert len(sols) == 1
    exact = sols[0]
    Hc, gc = H.astype(complex), g.astype(complex)
    for M, N in [(1, 1), (2, 1), (1, 2), (2, 2)]:
        rho = 1.0 if N == 1 else N * max(np.linalg.norm(H[:, c0:c1], 2) ** 2
                                         for c0, c1 in A.balanced_blocks(n, N))
        r = oracle.run_split(Hc, gc, M, N, lam, rho, 50000, eps=(1e-14, 1e-13))
        assert np.max(np.abs(r.v.imag)) == 0.0          # real data stays real
        assert np.allclose(r.v.real, exact, rtol=0, atol=1e-8), (M, N)
        assert np.array_equal(r.v != 0, exact != 0)


def test_planted_two_sparse_recovery_noiseless():
    rng = np.random.default_rng(4)
    m, n = 12, 32
    H = _rand_c(rng, (m, n), 1 / np.sqrt(2 * m))
    support = np.array([5, 19])
    u = np.zeros(n, complex)
    u[support] = np.exp(1j * np.array([0.3, 2.1]))
    g = H @ u
    # l0: the planted pair is the only 2-column subset that explains g exactly
    exact_pairs = []
    for a, b in itertools.combinations(range(n), 2):
        Hs = H[:, [a, b]]
        x = np.linalg.lstsq(Hs, g, rcond=None)[0]
        if np.linalg.norm(Hs @ x - g) < 1e-10 * np.linalg.norm(g):
            exact_pairs.append((a, b))
    assert exact_pairs == [tuple(support)]
    lam = 1e-3 * np.max(np.abs(H.conj().T @ g))
    for M, N in [(1, 1), (3, 1), (1, 2), (3, 2)]:
        rho = 0.3 if N == 1 else N * max(np.linalg.norm(H[:, c0:c1], 2) ** 2
                                         for c0, c1 in A.balanced_blocks(n, N))
        r = oracle.run_split(H, g, M, N, lam, rho, 60000, eps=(1e-15, 1e-13))
        assert list(np.flatnonzero(r.v)) == list(support), (M, N)
        assert np.linalg.norm(r.v - u) < 1e-2


# ----------------------------------------------------------------------------
# partitioner and Tables I-III
# ----------------------------------------------------------------------------

def test_partition_reproduces_table2_shapes():
    Nm, Np = 2160, 22500
    for line in open(os.path.join(GOLDEN, "table2_blocks.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, M, N, br, bc, lr, lc = line.split()
        M, N, br, bc, lr, lc = map(int, (M, N, br, bc, lr, lc))
        rows = A.balanced_blocks(Nm, M)
        cols = A.balanced_blocks(Np, N)
        assert {r1 - r0 for r0, r1 in rows} == {br}
        assert {c1 - c0 for c0, c1 in cols} == {bc}
        assert A.lemma_applies(br, bc)
        assert (lr, lc) == (br, br)


def test_partition_ragged_sizes():
    for total, parts in [(10, 3), (7, 7), (1440, 8), (101, 4), (5, 1)]:
        blocks = A.balanced_blocks(total, parts)
        sizes = [b - a for a, b in blocks]
        assert sum(sizes) == total and max(sizes) - min(sizes) <= 1
        assert sizes == sorted(sizes, reverse=True)
        assert blocks[0][0] == 0 and blocks[-1][1] == total
    with pytest.raises(ValueError):
        A.balanced_blocks(3, 4)


def test_communication_counts_table1_and_table3():
    printed = {}
    for line in open(os.path.join(GOLDEN, "table3_comm.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, elems, pct = line.split()
        printed[name] = (int(elems), float(pct))
    c = oracle.comm_elements(4, 3, 2160, 22500)
    assert c["consensus"] == printed["consensus"][0]
    assert c["sectioning"] == printed["sectioning"][0]
    assert round(100 * (1 - c["sectioning"] / c["consensus"]), 1) == printed["sectioning"][1]
    # Table I's C&S formula gives 16,620; the printed 12,870 does not follow from
    # it (the printed count and percentage agree only with each other).
    assert c["cs"] == 16620
    assert printed["cs"][0] != c["cs"]
    assert round(100 * (1 - printed["cs"][0] / c["consensus"]), 1) == printed["cs"][1]


def test_efficiency_inequalities_agree_with_table1():
    """Section IV-B: columns beat rows iff N < 2R; both beat rows iff
    N^2/(2M(N-1)) < R; both beat columns iff R < N^2 (M-1)/(2M), i.e.
    M > N^2/(N^2 - 2R) when N^2 > 2R."""
    for Nm in (100, 360):
        for Np in (150, 1000, 22500):
            R = Np / Nm
            for M in range(1, 9):
                for N in range(2, 12):
                    c = oracle.comm_elements(M, N, Nm, Np)
                    assert (c["sectioning"] < c["consensus"]) == (N < 2 * R)
                    assert (c["cs"] < c["consensus"]) == (N * N / (2 * M * (N - 1)) < R)
                    both_beat_cols = c["cs"] < c["sectioning"]
                    assert both_beat_cols == (R < N * N * (M - 1) / (2 * M))
                    if N * N > 2 * R:
                        assert both_beat_cols == (M > N * N / (N * N - 2 * R))


# ----------------------------------------------------------------------------
# stopping rule
# ----------------------------------------------------------------------------

def test_stop_rule_hand_worked_records():
    """Boyd et al. Section 3.3.1 (the residuals the paper cites): stop when
    ||r_p|| <= sqrt(p) eps_abs + eps_rel max(||Ax||, ||Bz||) and
    ||r_d|| <= sqrt(p) eps_abs + eps_rel ||A^T y||, with y = rho s the unscaled
    dual.  Records are (||r_p||^2, ||r_d||^2, ||u||^2, ||v||^2, ||s||^2); every
    number below is a power of two or a short sum of them, so the boundary
    cases are exact.  With p = 4, eps_abs = 1/8, eps_rel = 1/2, rho = 2:
    sqrt(p) eps_abs = 1/4; ||u|| = 2, ||v|| = 4 gives eps_pri = 1/4 + 2 = 9/4;
    ||s|| = 1 gives eps_dual = 1/4 + (1/2)(2)(1) = 5/4."""
    p, ea, er, rho = 4, 0.125, 0.5, 2.0
    # both norms exactly on their tolerance: stop (the test is "<=")
    assert A.stop_test(np.array([2.25 ** 2, 1.25 ** 2, 4.0, 16.0, 1.0]), p, rho, ea, er) is True
    # only the primal test fails: ||r_p|| = 5/2 > 9/4, ||r_d|| = 1 <= 5/4
    assert A.stop_test(np.array([2.5 ** 2, 1.0, 4.0, 16.0, 1.0]), p, rho, ea, er) is False
    # only the dual test fails: ||r_p|| = 2 <= 9/4, ||r_d|| = 3/2 > 5/4
    assert A.stop_test(np.array([4.0, 1.5 ** 2, 4.0, 16.0, 1.0]), p, rho, ea, er) is False
    # the larger of ||u|| and ||v|| sets eps_pri: ||u|| = 6 gives 1/4 + 3 = 13/4
    assert A.stop_test(np.array([3.25 ** 2, 1.0, 36.0, 16.0, 1.0]), p, rho, ea, er) is True
    assert A.stop_test(np.array([3.5 ** 2, 1.0, 36.0, 16.0, 1.0]), p, rho, ea, er) is False
    # rho scales the dual tolerance: rho = 4 gives eps_dual = 1/4 + 2 = 9/4
    assert A.stop_test(np.array([1.0, 2.25 ** 2, 4.0, 16.0, 1.0]), p, 4.0, ea, er) is True
    assert A.stop_test(np.array([1.0, 2.25 ** 2, 4.0, 16.0, 1.0]), p, rho, ea, er) is False
    # sqrt(p) scales the absolute part of both: p = 64 gives 1 + 2 = 3 and 1 + 1 = 2
    assert A.stop_test(np.array([9.0, 4.0, 4.0, 16.0, 1.0]), 64, rho, ea, er) is True
    assert A.stop_test(np.array([9.0, 4.0, 4.0, 16.0, 1.0]), 16, rho, ea, er) is False


def test_threshold_margin_hand_values():
    """min_k | |a_k| - kappa | / kappa: |3+4j| = 5, |1| = 1, |0| = 0 against kappa = 2
    give 3/2, 1/2 and 1, so 1/2; a tie gives 0; kappa = 0 (no shrinkage) gives inf."""
    a = np.array([3 + 4j, 1.0, 0.0])
    assert A.threshold_margin(a, 2.0) == 0.5
    assert A.threshold_margin(np.array([2j, 7.0]), 2.0) == 0.0
    assert A.threshold_margin(a, 0.0) == float("inf")


def _stacked_state(res, M, n):
    """(u, v, s) of an oracle result as (M, n) replicas, the image and the duals."""
    return res.u.reshape(M, n), res.v.copy(), res.s.reshape(M, n)


@pytest.mark.parametrize("M,N", [(1, 1), (3, 1), (1, 3), (2, 2)])
@pytest.mark.parametrize("k", [0, 4])
def test_recorded_norms_follow_the_stacked_definitions(M, N, k):
    """The norms the stopping rule reads, rebuilt from the state alone.

    Boyd's stacked form of the split: x = (u^1, ..., u^M) (one replica per
    row block; the column segments of a replica side by side), z = v,
    constraint x - [v; ...; v] = 0, so ||Ax|| = ||x||, ||Bz|| = ||[v; ...; v]||
    and ||A^T y|| = rho ||s|| over the stacked duals.  The primal residual is
    x - [v; ...; v].  The dual residual is taken from its definition as the
    defect of dual feasibility after the step: block b's gradient of
    1/2||H_b u_b - gt_b||^2 (gt_b the data the block fits, with the previous
    iterate's estimated data of the other column blocks) plus its unscaled
    dual rho s_b; stacked over all blocks its squared norm is ||r_d||^2."""
    p = small_problem(m=20, n=48, nnz=3, rho=3.0 * N)
    H, g, n = p.H, p.g, p.n
    before = oracle.run_split(H, g, M, N, p.lam, p.rho, k)
    after = oracle.run_split(H, g, M, N, p.lam, p.rho, k + 1)
    rows = A.balanced_blocks(p.m, M)
    cols = A.balanced_blocks(n, N)
    if k == 0:
        u0 = np.zeros((M, n), complex)
    else:
        u0 = before.u.reshape(M, n)
    u1, v1, s1 = _stacked_state(after, M, n)
    x = u1.reshape(-1)
    bz = np.tile(v1, M)
    defect = []
    for i, (r0, r1) in enumerate(rows):
        for j, (c0, c1) in enumerate(cols):
            gt = g[r0:r1].copy()
            for q, (d0, d1) in enumerate(cols):
                if q != j:
                    gt -= H[r0:r1, d0:d1] @ u0[i, d0:d1]
            Hb = H[r0:r1, c0:c1]
            defect.append(Hb.conj().T @ (Hb @ u1[i, c0:c1] - gt) + p.rho * s1[i, c0:c1])
    defect = np.concatenate(defect)
    rec = after.hist[-1]
    want = [np.linalg.norm(x - bz) ** 2, np.linalg.norm(defect) ** 2, np.linalg.norm(x) ** 2,
            np.linalg.norm(bz) ** 2, np.linalg.norm(s1.reshape(-1)) ** 2]
    for got, ref in zip(rec, want):
        assert abs(got - ref) <= 1e-9 * max(1.0, ref), (rec, want)


@pytest.mark.parametrize("M,N", [(1, 1), (4, 1), (1, 3), (2, 2)])
def test_stopping_iteration_follows_boyd(M, N):
    """The oracle stops at the first iteration whose state meets Boyd's test
    with p = the length of the stacked constraint (M n entries), the norms
    taken from the state as in the previous test.  The tolerances are chosen
    so that p = n instead would stop at another iteration."""
    p = small_problem(m=20, n=48, nnz=3, rho=3.0 * N)
    H, g, n = p.H, p.g, p.n
    eps_abs, eps_rel = 2e-4, 0.0
    K = 120
    stop = oracle.run_split(H, g, M, N, p.lam, p.rho, K, eps=(eps_abs, eps_rel))
    full = oracle.run_split(H, g, M, N, p.lam, p.rho, K)
    first = {}
    for plen in (M * n, n):
        for k in range(K):
            rp, rd = np.sqrt(full.hist[k, 0]), np.sqrt(full.hist[k, 1])
            if rp <= np.sqrt(plen) * eps_abs and rd <= np.sqrt(plen) * eps_abs:
                first[plen] = k + 1
                break
    assert M * n in first, "the tolerance is never met within the run"
    assert stop.stopped_at == first[M * n] == stop.iters
    if M > 1:
        assert first.get(n) != first[M * n]
    # and the recorded norms of the stopping iteration are those of the state
    u1, v1, s1 = _stacked_state(stop, M, n)
    assert abs(stop.hist[-1, 0] - np.linalg.norm(u1.reshape(-1) - np.tile(v1, M)) ** 2) <= 1e-12


# ----------------------------------------------------------------------------
# the stored FP64 solution of the time-to-tolerance workload
# ----------------------------------------------------------------------------

def load_vstar():
    """(header dict, v*) from tests/golden/vstar_gaussian_2048x16384_c8.txt."""
    path = os.path.join(GOLDEN, "vstar_gaussian_2048x16384_c8.txt")
    head, rows = {}, []
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                parts = line[1:].split()
                if parts and parts[0] in ("lambda", "rho", "iterations", "nonzeros"):
                    head[parts[0]] = float(parts[1])
                continue
            k, re, im = line.split()
            rows.append((int(k), float(re), float(im)))
    v = np.zeros(16384, dtype=np.complex128)
    for k, re, im in rows:
        v[k] = re + 1j * im
    return head, v


def test_stored_solution_satisfies_the_lasso_optimality_conditions():
    """v* minimises 1/2||Hv - g||^2 + lambda ||v||_1 (independent of ADMM):
    with c = H^H (g - H v*), c_k = lambda v_k / |v_k| on the support and
    |c_k| <= lambda elsewhere."""
    head, v = load_vstar()
    p = synth.gaussian_problem(2048, 16384, 128, seed=5)
    assert head["lambda"] == p.lam and head["rho"] == p.rho
    c = p.H.conj().T @ (p.g - p.H @ v)
    sup = v != 0
    assert sup.sum() == head["nonzeros"]
    assert np.max(np.abs(c[sup] - p.lam * v[sup] / np.abs(v[sup]))) <= 1e-9 * p.lam
    assert np.max(np.abs(c[~sup])) <= p.lam * (1 + 1e-9)
    # the planted scene is recovered on its support
    assert set(np.flatnonzero(p.u_true)) <= set(np.flatnonzero(v))


def test_stored_mixed_precision_solution_satisfies_the_lasso_optimality_conditions():
    """v* of the 8192 x 131072 workload (tests/golden/make_vstar_config3.py):
    with c = H^H (g - H v*), c_k = lambda v_k / |v_k| on the support and
    |c_k| <= lambda elsewhere; the stored lambda is 0.05 max|H^H g| of the
    recipe.  H is drawn again chunk by chunk (64 rows at a time), never held."""
    from concurrent.futures import ThreadPoolExecutor
    path = os.path.join(GOLDEN, "vstar_gaussian_8192x131072_c16.txt")
    head, rows = {}, []
    for line in open(path):
        if line.startswith("#"):
            parts = line[1:].split()
            if parts and parts[0] in ("lambda", "rho", "nonzeros"):
                head[parts[0]] = float(parts[1])
            continue
        k, re, im = line.split()
        rows.append((int(k), float(re) + 1j * float(im)))
    c3 = synth.CONFIG3
    m, n = c3["m"], c3["n"]
    idx = np.array([k for k, _ in rows])
    vals = np.array([x for _, x in rows])
    # pass 1: g (its noise scale needs every row of H u)
    _, g, u, _ = synth.chunked_gaussian_problem(m, n, c3["nnz"], c3["seed"], sink=lambda r0, blk: None,
                                                lam=-1.0)
    # pass 2: H^H g and H^H (g - H v*), summed in chunk order
    chunks = (m + synth.ROWS_PER_DRAW - 1) // synth.ROWS_PER_DRAW

    def part(c):
        blk = synth.chunked_gaussian_rows(m, n, c3["seed"], c).astype(np.complex128)
        r0 = c * synth.ROWS_PER_DRAW
        gc = g[r0:r0 + blk.shape[0]]
        res = gc - blk[:, idx] @ vals
        return np.conj(blk.T @ np.conj(gc)), np.conj(blk.T @ np.conj(res))

    hg = np.zeros(n, dtype=np.complex128)
    cvec = np.zeros(n, dtype=np.complex128)
    with ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:
        for a, b in ex.map(part, range(chunks)):
            hg += a
            cvec += b
    lam = head["lambda"]
    assert abs(lam - c3["lam_frac"] * np.max(np.abs(hg))) <= 1e-12 * lam
    assert head["rho"] == c3["rho"] and len(rows) == head["nonzeros"]
    v = np.zeros(n, dtype=np.complex128)
    v[idx] = vals
    sup = v != 0
    assert np.max(np.abs(cvec[sup] - lam * v[sup] / np.abs(v[sup]))) <= 1e-8 * lam
    assert np.max(np.abs(cvec[~sup])) <= lam * (1 + 1e-8)
    # the planted scene's support is recovered
    assert set(np.flatnonzero(u)) <= set(idx.tolist())
