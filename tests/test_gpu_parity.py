"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Both sides receive the same seeded, complex64-representable inputs.  The
GPU computes in FP32; the bar is
  * relative iterate error ||v_gpu - v_fp64|| / ||v_fp64|| <= 1e-5, and the
    same bound element by element, |v_gpu - v_fp64|_k <= 1e-5 ||v_fp64||_inf;
  * the recovered support {k : v_k != 0} identical, except coordinates whose
    FP64 shrinkage argument lies within 1e-5 ||a||_inf of the threshold,
    where either decision is correct in FP32 (their count is reported).
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import admm_fp64 as A

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_05571_gb300 as P
    P.load()   # fails loudly when the library cannot be built or loaded


def gpu_run(p, M, N, iters, H=None, g=None, lam=None, rho=None, host_inputs=False):
    import paper_1811_05571_gb300 as P
    H = p.H_c64() if H is None else H
    g = p.g_c64() if g is None else g
    if not host_inputs:
        H = torch.from_numpy(H).cuda()
        g = torch.from_numpy(g).cuda()
    s = P.Solver(H, g, M, N, p.lam if lam is None else lam, p.rho if rho is None else rho)
    s.set_option(P.ADMM_OPT_TIMEOUT_NS, 2_000_000_000)
    s.iterate(iters)
    assert s.status() == 0
    return s


def oracle_run(p, M, N, iters, lam=None, rho=None):
    return oracle.run_split(p.H, p.g, M, N, p.lam if lam is None else lam,
                            p.rho if rho is None else rho, iters)


def assert_parity(v_gpu, ref, tol=TOL, what="v"):
    v_gpu = np.asarray(v_gpu, dtype=np.complex128)
    v_ref = ref.v
    scale = max(np.linalg.norm(v_ref), 1e-30)
    rel = np.linalg.norm(v_gpu - v_ref) / scale
    assert rel <= tol, f"{what}: relative error {rel:.3e} > {tol}"
    elem = np.max(np.abs(v_gpu - v_ref)) if v_ref.size else 0.0
    assert elem <= tol * max(np.max(np.abs(v_ref)), 1e-30), f"{what}: element error {elem:.3e}"
    # support, excluding coordinates within the FP32 band of the threshold
    band = tol * max(np.max(np.abs(ref.a_last)), 1e-30)
    ambiguous = np.abs(np.abs(ref.a_last) - ref.kappa) <= band
    sup_gpu, sup_ref = v_gpu != 0, v_ref != 0
    mismatch = (sup_gpu != sup_ref) & ~ambiguous
    assert not mismatch.any(), f"{what}: support differs at {np.flatnonzero(mismatch)[:10]}"
    return rel, int(ambiguous.sum())


def compare_all(s, ref, M, N):
    v = s.v().cpu().numpy()
    rel, amb = assert_parity(v, ref)
    u = s.u().cpu().numpy().astype(np.complex128)
    ru = np.linalg.norm(u - ref.u) / max(np.linalg.norm(ref.u), 1e-30)
    assert ru <= TOL, f"u relative error {ru:.3e}"
    k, vv, ss, gh = s.state()
    assert k == ref.iters
    # the scaled duals accumulate u - v differences, so their FP32 error scales
    # with ||u||, not with ||s|| (which can be much smaller, e.g. lambda = 0)
    ss = ss.numpy().astype(np.complex128)
    rs = np.linalg.norm(ss - ref.s) / max(np.linalg.norm(ref.s), np.linalg.norm(ref.u), 1e-30)
    assert rs <= 10 * TOL, f"s error {rs:.3e} (relative to max(||s||, ||u||))"
    if N > 1:
        gh = gh.numpy().astype(np.complex128)
        rg = np.linalg.norm(gh - ref.ghat) / max(np.linalg.norm(ref.ghat), 1e-30)
        assert rg <= TOL, f"estimated data relative error {rg:.3e}"
    hist = s.residuals()
    assert hist.shape == ref.hist.shape
    for q in range(5):
        a, b = np.sqrt(hist[:, q]), np.sqrt(ref.hist[:, q])
        err = np.max(np.abs(a - b)) / max(np.max(b), 1e-30)
        assert err <= 1e-4, f"history column {q}: {err:.3e}"
    return rel, amb


# ----------------------------------------------------------------------------
# the two single-matrix workloads at full size
# ----------------------------------------------------------------------------

def test_gaussian_256x4096_consensus4_300_iterations():
    p = synth.gaussian_problem(256, 4096, 16, seed=0)
    ref = oracle_run(p, 4, 1, 300)
    s = gpu_run(p, 4, 1, 300)
    rel, amb = compare_all(s, ref, 4, 1)
    assert amb == 0
    # the planted support is recovered
    assert set(np.flatnonzero(s.v().cpu().numpy())) == set(np.flatnonzero(p.u_true))


@pytest.fixture(scope="module")
def cra():
    return synth.cra_problem()


@pytest.mark.parametrize("M,N", [(8, 1), (1, 8), (4, 4)])
def test_cra_1440x32768_all_splits_300_iterations(cra, M, N):
    """300 iterations: the column splits' Jacobi exchange of estimated data is
    where FP32 drift would accumulate."""
    ref = oracle_run(cra, M, N, 300)
    s = gpu_run(cra, M, N, 300)
    compare_all(s, ref, M, N)


WIDE_CASES = [(96, 90000, 3, 1, 30), (96, 90000, 1, 3, 30), (96, 90000, 2, 2, 30),
              (64, 90001, 1, 160, 20)]


def _sms() -> int:
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("m,n,M,N,iters", WIDE_CASES)
def test_wide_slabs_run_two_column_groups(m, n, M, N, iters):
    """n = 90000: slabs of more than 256 column pairs, so every CTA runs two
    column groups of consumer warps (half the slab each, two partial products
    per row); ragged n (padding to 90016), and with 160 column blocks slabs
    that meet two blocks."""
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(m, n, max(2, m // 16), seed=m + n + M + N)
    plan, _ = P.admm_plan(m, n, M, N, num_sms=_sms(), smem_limit=232448)
    assert plan["groups"] == 2, plan
    rho = _rho_cols(p, N)
    ref = oracle_run(p, M, N, iters, rho=rho)
    s = gpu_run(p, M, N, iters, rho=rho)
    compare_all(s, ref, M, N)


# ----------------------------------------------------------------------------
# mid sizes: several tiles, ragged blocks, odd column boundaries
# ----------------------------------------------------------------------------

def _rho_cols(p, N):
    return 1.0 if N == 1 else N * max(np.linalg.norm(p.H[:, c0:c1], 2) ** 2
                                      for c0, c1 in A.balanced_blocks(p.n, N))


@pytest.mark.parametrize("m,n,M,N,iters", [
    (300, 3000, 7, 1, 200),     # ragged rows, several CTAs
    (300, 3001, 1, 5, 150),     # odd n: padded tail, odd column boundaries
    (300, 3003, 3, 4, 150),     # both
    (200, 6001, 5, 4, 100),
    (64, 4096, 1, 1, 200),      # unsplit lasso ADMM
    (37, 517, 3, 5, 120),       # tiny ragged everything
    (8, 200, 8, 1, 100),        # one row per block
    (96, 2048, 2, 16, 80),      # narrow column blocks (slab spans several)
])
def test_mid_size_parity(m, n, M, N, iters):
    p = synth.gaussian_problem(m, n, max(2, m // 16), seed=m + n + M + N)
    rho = _rho_cols(p, N)
    ref = oracle_run(p, M, N, iters, rho=rho)
    s = gpu_run(p, M, N, iters, rho=rho)
    compare_all(s, ref, M, N)


def test_lambda_zero_is_plain_consensus_least_squares():
    p = synth.gaussian_problem(64, 1024, 4, seed=5)
    ref = oracle_run(p, 4, 1, 100, lam=0.0)
    s = gpu_run(p, 4, 1, 100, lam=0.0)
    compare_all(s, ref, 4, 1)
    assert np.all(s.v().cpu().numpy() != 0)


def test_huge_lambda_gives_exact_zero_image():
    p = synth.gaussian_problem(64, 1024, 4, seed=6)
    lam = 10.0 * np.max(np.abs(p.H.conj().T @ p.g))
    s = gpu_run(p, 2, 2, 50, lam=lam, rho=_rho_cols(p, 2))
    assert np.all(s.v().cpu().numpy() == 0)


# ----------------------------------------------------------------------------
# API behaviour
# ----------------------------------------------------------------------------

def test_runs_are_bitwise_deterministic_and_resume_across_launches():
    p = synth.gaussian_problem(128, 2048, 8, seed=7)
    rho = _rho_cols(p, 2)
    a = gpu_run(p, 2, 2, 60, rho=rho)
    b = gpu_run(p, 2, 2, 0, rho=rho)
    for _ in range(6):
        b.iterate(10)
    assert torch.equal(a.v(), b.v()) and torch.equal(a.u(), b.u())
    assert np.array_equal(a.residuals(), b.residuals())


def test_checkpoint_restore_continues_exactly():
    p = synth.gaussian_problem(128, 2048, 8, seed=8)
    rho = _rho_cols(p, 3)
    full = gpu_run(p, 2, 3, 40, rho=rho)
    first = gpu_run(p, 2, 3, 25, rho=rho)
    k, v, s, gh = first.state()
    assert k == 25
    second = gpu_run(p, 2, 3, 0, rho=rho)
    second.set_state(k, v, s, gh)
    second.iterate(15)
    assert torch.equal(full.v(), second.v())
    assert second.info()["iterations"] == 40


def test_new_scene_and_lambda_without_refactoring():
    p = synth.gaussian_problem(128, 2048, 8, seed=9)
    q = synth.gaussian_problem(128, 2048, 8, seed=9)
    g2 = synth.round_to_c64(q.g * (1 + 0.5j))
    import paper_1811_05571_gb300 as P
    s = gpu_run(p, 4, 1, 20)
    s.set_g(torch.from_numpy(g2.astype(np.complex64)).cuda())
    s.set_lambda(0.5 * p.lam)
    s.reset()
    s.iterate(80)
    ref = oracle.run_split(p.H, g2, 4, 1, 0.5 * p.lam, p.rho, 80)
    compare_all(s, ref, 4, 1)


def test_set_rho_refactors_and_matches_fresh_setup():
    p = synth.gaussian_problem(128, 2048, 8, seed=10)
    a = gpu_run(p, 4, 1, 0, rho=1.0)
    a.set_rho(3.0)
    a.reset()
    a.iterate(50)
    ref = oracle_run(p, 4, 1, 50, rho=3.0)
    compare_all(a, ref, 4, 1)


def test_set_rho_keeps_unscaled_duals():
    p = synth.gaussian_problem(64, 1024, 4, seed=11)
    a = gpu_run(p, 2, 1, 30, rho=1.0)
    _, _, s_before, _ = a.state()
    a.set_rho(4.0)
    _, _, s_after, _ = a.state()
    assert torch.allclose(s_after * 4.0, s_before * 1.0, rtol=1e-6, atol=1e-7)


def test_solve_stops_where_the_oracle_stops():
    p = synth.gaussian_problem(128, 2048, 8, seed=12)
    import paper_1811_05571_gb300 as P
    H = torch.from_numpy(p.H_c64()).cuda()
    g = torch.from_numpy(p.g_c64()).cuda()
    s = P.Solver(H, g, 4, 1, p.lam, p.rho)
    done = s.solve(5000, 1e-5, 1e-4)
    ref = oracle.run_split(p.H, p.g, 4, 1, p.lam, p.rho, 5000, eps=(1e-5, 1e-4))
    assert ref.stopped_at is not None
    assert abs(done - ref.stopped_at) <= 2, (done, ref.stopped_at)
    rec = s.residuals(1)[0]
    assert A.stop_test(rec, 4 * p.n, p.rho, 1e-5, 1e-4)


def test_complex128_and_host_inputs_match_complex64_device_inputs():
    p = synth.gaussian_problem(96, 1500, 6, seed=13)
    a = gpu_run(p, 3, 2, 40, rho=_rho_cols(p, 2))
    b = gpu_run(p, 3, 2, 40, rho=_rho_cols(p, 2), H=np.ascontiguousarray(p.H),
                g=np.ascontiguousarray(p.g), host_inputs=True)
    assert torch.equal(a.v(), b.v())


@pytest.mark.parametrize("m,n,M,N,iters", [
    (300, 1000, 1, 5, 120),     # sectioning, 300 x 200 blocks
    (1200, 512, 2, 1, 120),     # overdetermined consensus, 600 x 512 blocks
    (400, 600, 2, 4, 100),      # C&S, 200 x 150 blocks
    (64, 64, 1, 1, 100),        # square: the direct branch at m_b = n_b
])
def test_tall_blocks_match_the_direct_branch(m, n, M, N, iters):
    """Blocks with m_b >= n_b: the oracle inverts H_b^H H_b + rho I (the
    direct branch); the GPU applies the same operator through K_b."""
    rows = A.balanced_blocks(m, M)
    cols = A.balanced_blocks(n, N)
    assert all(not A.lemma_applies(r1 - r0, c1 - c0) for r0, r1 in rows for c0, c1 in cols)
    p = synth.gaussian_problem(m, n, max(2, n // 32), seed=m + n + M + N)
    rho = _rho_cols(p, N)
    ref = oracle_run(p, M, N, iters, rho=rho)
    s = gpu_run(p, M, N, iters, rho=rho)
    compare_all(s, ref, M, N)


def test_nonfinite_input_is_rejected():
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(32, 256, 2, seed=14)
    H = p.H_c64()
    H[3, 7] = np.nan
    with pytest.raises(P.AdmmError) as e:
        P.Solver(torch.from_numpy(H).cuda(), torch.from_numpy(p.g_c64()).cuda(), 2, 1, p.lam, 1.0)
    assert e.value.status == P.ADMM_ENONFINITE


def test_barrier_timeout_is_reported_and_reset_recovers():
    """A grid barrier told to wait for CTAs that do not exist expires after its
    bound; the call reports ADMM_ETIMEOUT, the context stays usable, and
    admm_reset restores a working handle."""
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(64, 1024, 4, seed=15)
    s = gpu_run(p, 2, 1, 0)
    s.set_option(P.ADMM_OPT_TIMEOUT_NS, 20_000_000)
    s.set_option(P.ADMM_OPT_BARRIER_EXTRA, 1)
    s.iterate(3)
    assert s.status() == P.ADMM_ETIMEOUT
    with pytest.raises(P.AdmmError):
        s.iterate(1)
    s.set_option(P.ADMM_OPT_BARRIER_EXTRA, 0)
    s.set_option(P.ADMM_OPT_TIMEOUT_NS, 2_000_000_000)
    s.reset()
    s.iterate(30)
    assert s.status() == 0
    ref = oracle_run(p, 2, 1, 30)
    compare_all(s, ref, 2, 1)


def test_phase_trace_is_monotonic_and_covers_every_iteration():
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(128, 4096, 8, seed=16)
    s = gpu_run(p, 4, 1, 0)
    s.set_option(P.ADMM_OPT_TRACE_ITERS, 5)
    s.iterate(5)
    tr = s.trace(5)
    assert tr.shape == (2, 5, 8)
    for cta in range(2):
        flat = tr[cta].reshape(-1)
        assert np.all(flat > 0) and np.all(np.diff(flat) >= 0)
    s.set_option(P.ADMM_OPT_TRACE_ITERS, 0)
    s.iterate(2)
    assert s.status() == 0


def test_several_handles_with_different_plans_coexist():
    """Handles whose plans need different shared memory launch the same kernel
    instance in any order."""
    p = synth.gaussian_problem(256, 8192, 8, seed=17)
    rho = _rho_cols(p, 4)
    a = gpu_run(p, 8, 1, 0, rho=rho)
    b = gpu_run(p, 1, 4, 0, rho=rho)
    c = gpu_run(p, 4, 4, 0, rho=rho)
    for s in (a, b, c, a, c, b):
        s.iterate(3)
        assert s.status() == 0


def test_autotuned_l2_policy_keeps_parity(cra):
    import paper_1811_05571_gb300 as P
    s = P.Solver(torch.from_numpy(cra.H_c64()).cuda(), torch.from_numpy(cra.g_c64()).cuda(), 4, 4,
                 cra.lam, cra.rho)
    keep = s.tune()
    assert keep in [x << 20 for x in (0, 16, 32, 44, 52, 64, 80, 96)]
    assert s.info()["iterations"] == 0
    s.iterate(50)
    assert s.status() == 0
    compare_all(s, oracle_run(cra, 4, 4, 50), 4, 4)
