"""The sharded iteration on the GPU: every rank of an Rr x Rc grid as its own
library handle (admm_shard_*) in this process, on one GPU, the exchanged sums
formed directly (sharded.LocalComm; no kernel waits for another).  The image,
the duals and the residual history must match the single-process FP64 oracle
at the FP32 bar of the other parity tests."""

import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import TOL, _rho_cols, assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_05571_gb300 as P
    P.load()


@pytest.mark.parametrize("m,n,M,N,world,grid,iters", [
    (256, 4096, 4, 1, 2, None, 60),        # consensus: row blocks on 2 ranks
    (300, 3001, 5, 1, 3, None, 60),        # ragged rows and columns
    (256, 4096, 1, 4, 2, None, 40),        # sectioning: column blocks on 2 ranks
    (256, 4096, 2, 2, 4, (2, 2), 40),      # consensus and sectioning on a 2 x 2 grid
    (300, 3003, 3, 4, 4, (2, 2), 40),      # ragged blocks on a 2 x 2 grid
])
def test_sharded_ranks_match_the_oracle(m, n, M, N, world, grid, iters):
    from paper_1811_05571_gb300 import sharded as SH
    p = synth.gaussian_problem(m, n, max(2, m // 16), seed=m + n + M + N + world)
    rho = _rho_cols(p, N)
    Rr, Rc = grid or SH.default_grid(M, N, world, m, n)
    lays = [SH.ShardLayout(m, n, M, N, Rr, Rc, r) for r in range(world)]
    H = torch.from_numpy(p.H_c64()).cuda()
    g = torch.from_numpy(p.g_c64()).cuda()
    engines = [SH.CudaShardEngine(H, g, lay, p.lam, rho) for lay in lays]
    sol = SH.ShardedSolver(list(zip(lays, engines)), SH.LocalComm(lays), rho).iterate(iters)
    ref = oracle.run_split(p.H, p.g, M, N, p.lam, rho, iters)
    v = np.zeros(n, np.complex128)
    s = np.zeros((M, n), np.complex128)
    for lay, e in zip(lays, engines):
        c0, c1 = lay.cols
        k, vv, ss, _ = e.state()
        assert k == iters
        if lay.row_group == 0:
            v[c0:c1] = vv.numpy()
        s[lay.blocks_i[0]:lay.blocks_i[1], c0:c1] = ss.numpy()
    assert_parity(v, ref)
    rs = np.linalg.norm(s - ref.s) / max(np.linalg.norm(ref.s), np.linalg.norm(ref.u), 1e-30)
    assert rs <= 10 * TOL, rs
    hist = sol.residuals()
    assert hist.shape == ref.hist.shape
    for q in range(5):
        a, b = np.sqrt(hist[:, q]), np.sqrt(ref.hist[:, q])
        assert np.max(np.abs(a - b)) <= 1e-4 * max(np.max(b), 1e-30), q
    for e in engines:
        e.close()
