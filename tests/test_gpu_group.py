"""GPU parity of the multi-problem launch (admm_group_*): every problem of a
group, iterated together with the others on its share of the SMs, against
the FP64 oracle at the 1e-5 bar, and against the same problem run alone."""

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import admm_fp64 as A
from test_gpu_parity import TOL, compare_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_05571_gb300 as P
    P.load()


def _rho(p, N):
    if N == 1:
        return 1.0
    return N * max(np.linalg.norm(p.H[:, c0:c1], 2) ** 2 for c0, c1 in A.balanced_blocks(p.n, N))


SHAPES = [
    (256, 4096, 2, 1), (600, 8192, 3, 1), (300, 3001, 1, 5), (400, 6000, 2, 3),
    (96, 2048, 1, 1), (1000, 12000, 4, 1),
]


def _solvers(iters):
    import paper_1811_05571_gb300 as P
    probs, solvers = [], []
    for q, (m, n, M, N) in enumerate(SHAPES):
        p = synth.gaussian_problem(m, n, max(2, m // 16), seed=300 + q)
        rho = _rho(p, N)
        s = P.Solver(torch.from_numpy(p.H_c64()).cuda(), torch.from_numpy(p.g_c64()).cuda(), M, N, p.lam, rho)
        s.set_option(P.ADMM_OPT_TIMEOUT_NS, 2_000_000_000)
        probs.append((p, M, N, rho))
        solvers.append(s)
    return probs, solvers


def test_group_iterates_every_problem_like_the_oracle():
    import paper_1811_05571_gb300 as P
    probs, solvers = _solvers(60)
    g = P.Group(solvers)
    info = g.info()
    assert info["waves"] >= 1 and sum(info["ctas"]) <= 152 * info["waves"]
    g.iterate(40)
    g.iterate(20)              # resumes across launches
    for (p, M, N, rho), s in zip(probs, solvers):
        assert s.status() == 0
        assert s.info()["iterations"] == 60
        ref = oracle.run_split(p.H, p.g, M, N, p.lam, rho, 60)
        compare_all(s, ref, M, N)
    g.close()


def test_group_result_matches_the_problem_run_alone():
    import paper_1811_05571_gb300 as P
    probs, solvers = _solvers(30)
    _, alone = _solvers(30)
    g = P.Group(solvers)
    g.iterate(30)
    for s, a in zip(solvers, alone):
        a.iterate(30)
        v, va = s.v().cpu().numpy(), a.v().cpu().numpy()
        assert np.linalg.norm(v - va) <= 1e-5 * max(np.linalg.norm(va), 1e-30)
    g.close()


def test_group_of_several_waves_runs_in_one_launch():
    """A problem large enough to take a wave of its own (2048 x 16384) beside the
    six shared-wave shapes: at least two waves, all in one cooperative launch,
    every problem still the oracle's at the 1e-5 bar."""
    import paper_1811_05571_gb300 as P
    probs, solvers = _solvers(40)
    big = synth.gaussian_problem(2048, 16384, 64, seed=399)
    s_big = P.Solver(torch.from_numpy(big.H_c64()).cuda(), torch.from_numpy(big.g_c64()).cuda(), 8, 1,
                     big.lam, 1.0)
    probs.append((big, 8, 1, 1.0))
    solvers.append(s_big)
    g = P.Group(solvers)
    info = g.info()
    assert info["waves"] >= 2 and info["launches"] == 1, info
    g.iterate(25)
    g.iterate(15)
    assert g.info()["graph"] == 1, "the one launch is replayed from a captured CUDA graph"
    for (p, M, N, rho), s in zip(probs, solvers):
        assert s.status() == 0
        assert s.info()["iterations"] == 40
        compare_all(s, oracle.run_split(p.H, p.g, M, N, p.lam, rho, 40), M, N)
    g.close()
