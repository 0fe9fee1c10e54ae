"""GPU parity of the FP16-H mode (ADMM_OPT_H_FP16) and of FP16 + complex64
polish iterations.

An FP16 run is exact ADMM on the matrix the FP16 storage encodes, so it is
compared, at the FP32 bar of the complex64 path (1e-5), with the FP64 oracle
run on ``oracle.quantize.dequantized(H)``.  A run that switches back to the
complex64 H continues from the FP16 iterate; its end point is compared with
the FP64 oracle solution of the original problem (relative error <= 1e-4).
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import quantize as Q
from test_gpu_parity import TOL, WIDE_CASES, _rho_cols, compare_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_05571_gb300 as P
    P.load()


def solver(p, M, N, lam=None, rho=None, fp16=True):
    import paper_1811_05571_gb300 as P
    H = torch.from_numpy(p.H_c64()).cuda()
    g = torch.from_numpy(p.g_c64()).cuda()
    s = P.Solver(H, g, M, N, p.lam if lam is None else lam, p.rho if rho is None else rho)
    s.set_option(P.ADMM_OPT_TIMEOUT_NS, 2_000_000_000)
    if fp16:
        s.use_fp16(True)
    return s


def oracle_fp16(p, M, N, iters, lam=None, rho=None, eps=None):
    return oracle.run_split(Q.dequantized(p.H), p.g, M, N, p.lam if lam is None else lam,
                            p.rho if rho is None else rho, iters, eps=eps)


def rel_err(x, ref):
    x = np.asarray(x, dtype=np.complex128)
    return np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-30)


@pytest.fixture(scope="module")
def cra():
    return synth.cra_problem()


@pytest.mark.parametrize("M,N", [(8, 1), (1, 8), (4, 4)])
def test_fp16_cra_1440x32768_all_splits(cra, M, N):
    s = solver(cra, M, N)
    info = s.info()
    assert info["h_fp16"] == 1 and info["h16_ready"] == 1
    assert info["h16_bytes"] == cra.m * cra.n * 4
    s.iterate(50)
    assert s.status() == 0
    compare_all(s, oracle_fp16(cra, M, N, 50), M, N)


def test_fp16_gaussian_256x4096_consensus4_300_iterations():
    p = synth.gaussian_problem(256, 4096, 16, seed=0)
    s = solver(p, 4, 1)
    s.iterate(300)
    compare_all(s, oracle_fp16(p, 4, 1, 300), 4, 1)
    assert set(np.flatnonzero(s.v().cpu().numpy())) == set(np.flatnonzero(p.u_true))


@pytest.mark.parametrize("m,n,M,N,iters", [
    (300, 3000, 7, 1, 200),     # ragged row groups (300 = 4 x 64 + 44)
    (300, 3001, 1, 5, 150),     # odd column boundaries: slab starts 2 mod 4
    (300, 3003, 3, 4, 150),
    (200, 6001, 5, 4, 100),
    (37, 517, 3, 5, 120),       # one partial row group
    (96, 2048, 2, 16, 80),      # slabs spanning several column blocks
])
def test_fp16_mid_size_parity(m, n, M, N, iters):
    _fp16_case(m, n, M, N, iters)


@pytest.mark.parametrize("m,n,M,N,iters", WIDE_CASES)
def test_fp16_wide_slabs_two_column_groups(m, n, M, N, iters):
    """The two-column-group kernel instance in the FP16 mode (slabs of more
    than 256 pairs; odd slab starts give boxes starting 2 columns early)."""
    _fp16_case(m, n, M, N, iters)


def _fp16_case(m, n, M, N, iters):
    p = synth.gaussian_problem(m, n, max(2, m // 16), seed=m + n + M + N)
    rho = _rho_cols(p, N)
    s = solver(p, M, N, rho=rho)
    s.iterate(iters)
    assert s.status() == 0
    compare_all(s, oracle_fp16(p, M, N, iters, rho=rho), M, N)


def test_rows_of_very_different_magnitude_keep_their_scales():
    # 64-row groups (and their data) weighted 1/2, 1, 4, 1/4, straddling the three
    # row blocks: every group has its own scale (the weights change the binade)
    # while the blocks stay well conditioned for the FP32 bar
    p = synth.gaussian_problem(256, 2048, 8, seed=21)
    w = np.repeat(np.array([0.5, 1.0, 4.0, 0.25]), 64)
    H = synth.round_to_c64(p.H * w[:, None])
    g = synth.round_to_c64(p.g * w)
    q = synth.Problem(H=H, g=g, u_true=p.u_true, lam=synth.lambda_from_fraction(H, g, 0.05),
                      rho=1.0, name="weighted rows")
    assert len(set(Q.group_scales(H))) == 4
    s = solver(q, 3, 1)
    s.iterate(100)
    compare_all(s, oracle_fp16(q, 3, 1, 100), 3, 1)


def test_switching_precision_is_a_state_handoff():
    """FP16 then complex64 in one handle equals an FP16 run checkpointed into a
    fresh complex64 handle: the state is shared, nothing else carries over."""
    p = synth.gaussian_problem(128, 2048, 8, seed=22)
    rho = _rho_cols(p, 2)
    a = solver(p, 2, 2, rho=rho)
    a.iterate(30)
    a.use_fp16(False)
    assert a.info()["h_fp16"] == 0 and a.info()["h16_ready"] == 1
    a.iterate(20)
    b = solver(p, 2, 2, rho=rho)
    b.iterate(30)
    k, v, st, gh = b.state()
    c = solver(p, 2, 2, rho=rho, fp16=False)
    c.set_state(k, v, st, gh)
    c.iterate(20)
    assert torch.equal(a.v(), c.v()) and torch.equal(a.u(), c.u())


def test_set_rho_refactors_the_fp16_factors_too():
    p = synth.gaussian_problem(128, 2048, 8, seed=23)
    s = solver(p, 4, 1, rho=1.0)
    s.set_rho(3.0)
    s.reset()
    s.iterate(50)
    compare_all(s, oracle_fp16(p, 4, 1, 50, rho=3.0), 4, 1)
    s.use_fp16(False)
    s.reset()
    s.iterate(50)
    compare_all(s, oracle.run_split(p.H, p.g, 4, 1, p.lam, 3.0, 50), 4, 1)


def test_fp16_solve_stops_where_the_oracle_stops():
    p = synth.gaussian_problem(128, 2048, 8, seed=12)
    s = solver(p, 4, 1)
    done = s.solve(5000, 1e-5, 1e-4)
    ref = oracle_fp16(p, 4, 1, 5000, eps=(1e-5, 1e-4))
    assert ref.stopped_at is not None
    assert abs(done - ref.stopped_at) <= 2, (done, ref.stopped_at)


@pytest.fixture(scope="module")
def converged():
    """Gaussian 1024 x 16384, 64 nonzeros, consensus over 4 row blocks: the FP64
    oracle solution v* (600 iterations: primal and dual residuals < 1e-10)."""
    p = synth.gaussian_problem(1024, 16384, 64, seed=0)
    ref = oracle.run_split(p.H, p.g, 4, 1, p.lam, p.rho, 600)
    assert np.sqrt(ref.hist[-1, 0]) < 1e-9 and np.sqrt(ref.hist[-1, 1]) < 1e-9
    return p, ref.v


def test_fp16_then_polish_reaches_the_fp64_solution(converged):
    p, vstar = converged
    s = solver(p, 4, 1)
    s.iterate(280)
    e16 = rel_err(s.v().cpu().numpy(), vstar)
    s.use_fp16(False)
    s.iterate(120)
    e_pol = rel_err(s.v().cpu().numpy(), vstar)
    plain = solver(p, 4, 1, fp16=False)
    plain.iterate(400)
    e32 = rel_err(plain.v().cpu().numpy(), vstar)
    # FP16 storage perturbs H by about 2^-11 relative; its fixed point stays within 1e-4
    assert e16 <= 1e-4, e16
    # polishing on the complex64 H removes the FP16 perturbation down to FP32 level
    assert e_pol <= 1e-5, e_pol
    assert e32 <= 1e-5, e32
    # and the support of the FP64 solution is recovered
    assert set(np.flatnonzero(s.v().cpu().numpy())) == set(np.flatnonzero(vstar))
