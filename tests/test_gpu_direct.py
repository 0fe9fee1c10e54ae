"""GPU parity of the direct factor form (ADMM_FORM_DIRECT: the n_b x n_b
factor (H_b^H H_b + rho I)^{-1} of Section III-B) against the FP64 oracle,
whose blocks with m_b >= n_b take the same direct branch.  Same bar as the
lemma form: relative iterate error <= 1e-5, support identical outside the
FP32 band of the threshold."""

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import admm_fp64 as A
from test_gpu_parity import _rho_cols, compare_all, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_05571_gb300 as P
    P.load()


def direct_run(p, M, N, iters, rho=None, form="direct", lam=None, factor_pass=0):
    import paper_1811_05571_gb300 as P
    H = torch.from_numpy(p.H_c64()).cuda()
    g = torch.from_numpy(p.g_c64()).cuda()
    s = P.Solver(H, g, M, N, p.lam if lam is None else lam, p.rho if rho is None else rho, form=form)
    if factor_pass:
        s.set_option(P.ADMM_OPT_DIR_FACTOR_PASS, factor_pass)
    s.iterate(iters)
    assert s.status() == 0
    return s


@pytest.mark.parametrize("m,n,M,N,iters", [
    (1200, 512, 2, 1, 120),     # overdetermined consensus, 600 x 512 blocks: H is never read
    (700, 203, 1, 4, 120),      # sectioning, ragged column blocks of 51 / 50
    (703, 130, 3, 2, 100),      # C&S, ragged rows, 234 x 65 blocks
    (300, 300, 1, 1, 100),      # square lasso (m_b = n_b)
    (2000, 70, 1, 1, 100),      # tall lasso, a single partial factor chunk
    (4100, 1030, 5, 3, 60),     # several column tiles, factor chunks and row tiles, ragged tails
    (5000, 2100, 2, 1, 40),     # blocks wider than 2048 columns: the plain-load factor pass
    (3000, 1500, 2, 1, 40),     # 1500-column blocks: the streamed factor pass, several items per CTA
    (4000, 2400, 2, 2, 30),     # the streamed factor pass with two column blocks (q from the column pass)
])
def test_direct_form_matches_the_oracle(m, n, M, N, iters):
    """The full-factor-row passes (ADMM_OPT_DIR_FACTOR_PASS 1)."""
    rows = A.balanced_blocks(m, M)
    cols = A.balanced_blocks(n, N)
    assert all(not A.lemma_applies(r1 - r0, c1 - c0) for r0, r1 in rows for c0, c1 in cols)
    p = synth.gaussian_problem(m, n, max(2, n // 32), seed=m + n + M + N + 1)
    rho = _rho_cols(p, N)
    ref = oracle_run(p, M, N, iters, rho=rho)
    s = direct_run(p, M, N, iters, rho=rho, factor_pass=1)
    info = s.info()
    assert info["factor_form"] == 1 and info["rows_per_stage"] != 64
    compare_all(s, ref, M, N)


def _tile_bytes(n, N):
    """Bytes of the lower-triangle 64 x 64 tiles of one replica's factors."""
    total = 0
    for c0, c1 in A.balanced_blocks(n, N):
        nt = -(-(c1 - c0) // 64)
        total += nt * (nt + 1) // 2 * 64 * 64 * 8
    return total


@pytest.mark.parametrize("m,n,M,N,iters,fp", [
    (1200, 512, 2, 1, 120, 2),   # 512 columns (8 tile panels), forced below the default width
    (3000, 1500, 2, 1, 40, 0),   # 1500 columns: the default from 1024 on; a ragged last panel of 28
    (5000, 2100, 2, 1, 40, 0),   # 2100 columns, 33 panels (several rounds of the panel sums)
    (4000, 2400, 2, 2, 30, 0),   # two column blocks: q from the column pass, the row pass after
    (3600, 300, 9, 1, 60, 2),    # nine replicas: the update's general path (more than eight)
    (700, 300, 1, 1, 80, 2),     # the lasso (one block): a panel's update right after its sums
    (2600, 770, 2, 3, 40, 2),    # ragged column blocks of 257 / 257 / 256
])
def test_tile_pass_matches_the_oracle(m, n, M, N, iters, fp):
    """The lower-triangle tile pass (ADMM_OPT_DIR_FACTOR_PASS 2, the default
    from 1024 columns): the same iterates as the oracle's direct branch, and
    exactly the tile bytes per iteration."""
    p = synth.gaussian_problem(m, n, max(2, n // 32), seed=m + n + M + N + 2)
    rho = _rho_cols(p, N)
    ref = oracle_run(p, M, N, iters, rho=rho)
    s = direct_run(p, M, N, iters, rho=rho, factor_pass=fp)
    info = s.info()
    assert info["rows_per_stage"] == 64
    assert info["factor_bytes"] == M * _tile_bytes(n, N)
    compare_all(s, ref, M, N)


def test_tile_and_row_passes_agree():
    """The two factor passes compute the same u_b = L_b q_b: after 60
    iterations of 1100 x 1100 blocks their images agree to FP32 rounding."""
    p = synth.gaussian_problem(3 * 1100, 1100, 30, seed=60)
    a = direct_run(p, 3, 1, 60, factor_pass=1)
    b = direct_run(p, 3, 1, 60, factor_pass=2)
    va, vb = a.v().cpu().numpy(), b.v().cpu().numpy()
    assert np.linalg.norm(va - vb) <= 1e-5 * np.linalg.norm(va)
    ra, rb = a.residuals(60), b.residuals(60)
    for q in range(5):
        x, y = np.sqrt(ra[:, q]), np.sqrt(rb[:, q])
        assert np.max(np.abs(x - y)) <= 1e-4 * np.max(x), q


def test_tile_pass_set_rho_restart_and_stop():
    """A new rho repacks the tiles; a restart from a checkpoint is bit exact
    (fixed summation order); the stopping test ends where the oracle's does."""
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(2048, 1024, 24, seed=61)
    s = direct_run(p, 2, 1, 10, rho=1.0)
    assert s.info()["rows_per_stage"] == 64
    s.set_rho(2.5)
    s.reset()
    s.iterate(60)
    compare_all(s, oracle_run(p, 2, 1, 60, rho=2.5), 2, 1)
    k, v, sd, gh = s.state()
    s.iterate(15)
    v_straight = s.v().cpu()
    s.set_state(k, v, sd, None)
    s.iterate(15)
    assert s.status() == 0 and torch.equal(s.v().cpu(), v_straight)
    t = P.Solver(torch.from_numpy(p.H_c64()).cuda(), torch.from_numpy(p.g_c64()).cuda(), 2, 1, p.lam, 1.0,
                 form="direct")
    done = t.solve(2000, 1e-5, 1e-4)
    ref = oracle.run_split(p.H, p.g, 2, 1, p.lam, 1.0, 2000, eps=(1e-5, 1e-4))
    assert ref.stopped_at is not None and abs(done - ref.stopped_at) <= 2, (done, ref.stopped_at)


def test_factor_pass_option_is_checked():
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(512, 128, 4, seed=62)
    s = direct_run(p, 2, 1, 2)          # 128-column blocks: no tiles
    with pytest.raises(P.AdmmError) as e:
        s.set_option(P.ADMM_OPT_DIR_FACTOR_PASS, 2)
    assert e.value.status == P.ADMM_EUNSUPPORTED
    with pytest.raises(P.AdmmError) as e:
        s.set_option(P.ADMM_OPT_DIR_FACTOR_PASS, 3)
    assert e.value.status == P.ADMM_EINVAL
    s.set_option(P.ADMM_OPT_DIR_FACTOR_PASS, 1)
    s.iterate(2)
    assert s.status() == 0 and s.state()[0] == 4


def test_streamed_factor_pass_with_more_items_than_its_chunk_table():
    """80 row blocks of 1024 x 1024: 5120 factor items over the CTAs, more than
    the 32 a CTA counts in shared memory, so the later items of a CTA count
    their rows in the global chunk counters at once."""
    p = synth.gaussian_problem(80 * 1024, 1024, 16, seed=44)
    ref = oracle_run(p, 80, 1, 3)
    s = direct_run(p, 80, 1, 3, factor_pass=1)
    info = s.info()
    assert info["rows_per_stage"] == 4 and 5120 > 32 * info["ctas"]
    compare_all(s, ref, 80, 1)


def test_direct_form_on_wide_blocks_is_the_same_algorithm():
    """The direct form is valid for any block shape (it is only costlier when
    m_b < n_b): on wide blocks it matches the oracle's lemma branch."""
    p = synth.gaussian_problem(96, 400, 6, seed=31)
    rho = _rho_cols(p, 2)
    ref = oracle_run(p, 2, 2, 80, rho=rho)
    s = direct_run(p, 2, 2, 80, rho=rho)
    compare_all(s, ref, 2, 2)


def test_auto_form_follows_the_block_shape():
    import paper_1811_05571_gb300 as P
    tall = synth.gaussian_problem(512, 128, 4, seed=32)
    wide = synth.gaussian_problem(64, 512, 4, seed=33)
    for p, M, N, want in [(tall, 2, 1, 1), (tall, 1, 2, 1), (wide, 1, 1, 0), (wide, 2, 1, 0)]:
        s = P.Solver(torch.from_numpy(p.H_c64()).cuda(), torch.from_numpy(p.g_c64()).cuda(), M, N,
                     p.lam, 1.0, form="auto")
        assert s.info()["factor_form"] == want, (p.m, p.n, M, N)


def test_lemma_and_direct_forms_agree_on_a_large_tall_problem():
    """8192 x 1024 in 4 x 2 blocks (2048 x 512): the two forms of the same
    iteration against each other after 80 iterations, and the direct form
    against the oracle."""
    p = synth.gaussian_problem(8192, 1024, 32, seed=34)
    rho = _rho_cols(p, 2)
    ref = oracle_run(p, 4, 2, 80, rho=rho)
    d = direct_run(p, 4, 2, 80, rho=rho)
    compare_all(d, ref, 4, 2)
    lem = direct_run(p, 4, 2, 80, rho=rho, form="lemma")
    vd, vl = d.v().cpu().numpy(), lem.v().cpu().numpy()
    assert np.linalg.norm(vd - vl) <= 2e-5 * np.linalg.norm(vl)


def test_new_data_vector_recomputes_the_cached_product():
    """With one column block the direct form caches H_i^H g_i; admm_set_g
    must replace it (and reset restarts from zero)."""
    p = synth.gaussian_problem(900, 200, 6, seed=35)
    q = synth.gaussian_problem(900, 200, 6, seed=36)
    s = direct_run(p, 3, 1, 20)
    s.set_g(torch.from_numpy(q.g_c64()).cuda())
    s.reset()
    s.iterate(90)
    assert s.status() == 0
    ref = oracle.run_split(p.H, q.g, 3, 1, p.lam, p.rho, 90)
    compare_all(s, ref, 3, 1)


def test_set_rho_refactors_the_direct_factor():
    p = synth.gaussian_problem(800, 160, 5, seed=37)
    s = direct_run(p, 2, 2, 10, rho=1.0)
    s.set_rho(3.0)
    s.reset()
    s.iterate(80)
    ref = oracle_run(p, 2, 2, 80, rho=3.0)
    compare_all(s, ref, 2, 2)


@pytest.mark.parametrize("M,N", [(2, 1), (1, 3), (2, 2)])
def test_checkpoint_restart_is_bit_exact(M, N):
    """The direct form sums in a fixed order: a restart from a checkpoint
    reproduces the uninterrupted iterates bit for bit."""
    p = synth.gaussian_problem(600, 150, 5, seed=38 + M + N)
    rho = _rho_cols(p, N)
    s = direct_run(p, M, N, 17, rho=rho)
    k, v, sd, gh = s.state()
    s.iterate(23)
    v_straight = s.v().cpu()
    s.set_state(k, v, sd, gh if N > 1 else None)
    s.iterate(23)
    assert s.status() == 0
    assert torch.equal(s.v().cpu(), v_straight)


def test_solve_stops_where_the_oracle_stops():
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(1024, 256, 8, seed=41)
    for M, N in [(4, 1), (2, 2)]:
        rho = _rho_cols(p, N)
        s = P.Solver(torch.from_numpy(p.H_c64()).cuda(), torch.from_numpy(p.g_c64()).cuda(), M, N,
                     p.lam, rho, form="direct")
        done = s.solve(3000, 1e-5, 1e-4)
        ref = oracle.run_split(p.H, p.g, M, N, p.lam, rho, 3000, eps=(1e-5, 1e-4))
        assert ref.stopped_at is not None
        assert abs(done - ref.stopped_at) <= 2, (M, N, done, ref.stopped_at)
        rec = s.residuals(1)[0]
        assert A.stop_test(rec, M * p.n, rho, 1e-5, 1e-4)
        # the state is that of the last iteration: continuing is a plain iterate
        k0 = s.state()[0]
        s.iterate(3)
        assert s.state()[0] == k0 + 3


def test_persistent_kernel_options_are_refused():
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(256, 64, 3, seed=42)
    s = direct_run(p, 2, 1, 1)
    for opt in (P.ADMM_OPT_H_FP16, P.ADMM_OPT_RECORD_ITERS, P.ADMM_OPT_TRACE_ITERS, P.ADMM_OPT_BARRIER_EXTRA):
        with pytest.raises(P.AdmmError) as e:
            s.set_option(opt, 1)
        assert e.value.status == P.ADMM_EUNSUPPORTED
    with pytest.raises(P.AdmmError) as e:
        P.Group([s])
    assert e.value.status == P.ADMM_EUNSUPPORTED
    s.tune()                  # nothing to tune; the state is untouched
    s.iterate(2)
    assert s.status() == 0 and s.state()[0] == 3


def test_lambda_zero_is_least_squares():
    """lambda = 0 with one block: the fixed point is the least-squares
    solution of the overdetermined system, reached by the direct form."""
    p = synth.gaussian_problem(400, 100, 4, seed=43)
    s = direct_run(p, 1, 1, 400, lam=0.0)
    x_ls = np.linalg.lstsq(p.H, p.g, rcond=None)[0]
    v = s.v().cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(v - x_ls) <= 1e-4 * np.linalg.norm(x_ls)


def test_tile_pass_solve_with_two_column_blocks():
    """With several column blocks the tile pass's update keeps the record and
    the row pass turns the stopping decision into the stop flag: a solve on
    2 x 2 blocks of 1024 x 512 (the tile pass forced) ends where the
    oracle's does."""
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(2048, 1024, 24, seed=63)
    rho = _rho_cols(p, 2)
    s = P.Solver(torch.from_numpy(p.H_c64()).cuda(), torch.from_numpy(p.g_c64()).cuda(), 2, 2, p.lam, rho,
                 form="direct")
    s.set_option(P.ADMM_OPT_DIR_FACTOR_PASS, 2)
    assert s.info()["rows_per_stage"] == 64
    done = s.solve(3000, 1e-5, 1e-4)
    ref = oracle.run_split(p.H, p.g, 2, 2, p.lam, rho, 3000, eps=(1e-5, 1e-4))
    assert ref.stopped_at is not None and abs(done - ref.stopped_at) <= 2, (done, ref.stopped_at)
    assert A.stop_test(s.residuals(1)[0], 2 * p.n, rho, 1e-5, 1e-4)


def test_tile_pass_new_data_vector_and_pass_switch():
    """admm_set_g replaces the cached H_i^H g_i under the tile pass; switching
    between the tile pass and the full-row pass mid-run continues the same
    iteration (the deferred record and the iteration count carry over)."""
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(3600, 1100, 30, seed=64)
    q = synth.gaussian_problem(3600, 1100, 30, seed=65)
    s = direct_run(p, 3, 1, 10)
    assert s.info()["rows_per_stage"] == 64
    s.set_g(torch.from_numpy(q.g_c64()).cuda())
    s.reset()
    s.iterate(17)                                   # one 16-graph and one 1-graph on the tile pass
    s.set_option(P.ADMM_OPT_DIR_FACTOR_PASS, 1)
    s.iterate(20)                                   # full rows
    s.set_option(P.ADMM_OPT_DIR_FACTOR_PASS, 2)
    s.iterate(23)                                   # tiles again
    assert s.status() == 0 and s.state()[0] == 60
    ref = oracle.run_split(p.H, q.g, 3, 1, p.lam, p.rho, 60)
    compare_all(s, ref, 3, 1)
