"""The sharded iteration's host logic on CPU ranks (gloo): the blocks of one
split spread over 2 or 4 processes (Section IV, Table I), each rank's blocks
solved in FP64 by tests/shard_fp64.py, the estimated-data sums and the
consensus sums exchanged through torch.distributed sub-groups.  The result
must be the single-process FP64 oracle's, iterate by iterate (1e-12)."""

import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from conftest import ROOT
from paper_1811_05571_gb300 import sharded as SH


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, {root!r}); sys.path.insert(0, os.path.join({root!r}, "tests"))
import numpy as np, torch, torch.distributed as dist
dist.init_process_group("gloo")
import synth
from paper_1811_05571_gb300 import sharded as SH
from shard_fp64 import Fp64ShardEngine
m, n, M, N, K, rho, grid = {m}, {n}, {M}, {N}, {K}, {rho!r}, {grid!r}
p = synth.gaussian_problem(m, n, 5, seed=m + n + M + N)
rank, world = dist.get_rank(), dist.get_world_size()
lay = SH.ShardLayout(m, n, M, N, *(grid or SH.default_grid(M, N, world, m, n)), rank)
eng = Fp64ShardEngine(p.H, p.g, lay, p.lam, rho)
sol = SH.ShardedSolver([(lay, eng)], SH.TorchComm(lay), rho).iterate(K)
mine = {{"rank": rank, "rows": lay.blocks_i, "cols": lay.cols, "row_group": lay.row_group,
         "v": [eng.v.real.tolist(), eng.v.imag.tolist()],
         "s": [eng.s.real.tolist(), eng.s.imag.tolist()], "hist": sol.residuals().tolist()}}
allr = [None] * world
dist.all_gather_object(allr, mine)
if rank == 0:
    print(json.dumps(allr))
dist.destroy_process_group()
"""


def _run(m, n, M, N, K, rho, world, grid=None):
    port = _free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1",
                   OPENBLAS_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
        script = RANK_SCRIPT.format(root=ROOT, m=m, n=n, M=M, N=N, K=K, rho=rho, grid=grid)
        procs.append(subprocess.Popen([sys.executable, "-c", script], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-3000:]
        outs.append(out)
    return json.loads(outs[0].strip().splitlines()[-1])


@pytest.mark.parametrize("M,N,world,grid", [(4, 1, 2, None), (3, 1, 3, None), (1, 4, 2, None), (1, 3, 3, None),
                                              (2, 2, 2, None), (2, 3, 4, (2, 2)), (3, 2, 4, (2, 2))])
def test_sharded_iteration_equals_the_single_process_oracle(M, N, world, grid):
    m, n, K = 48, 160, 25
    p = synth.gaussian_problem(m, n, 5, seed=m + n + M + N)
    rho = 1.0 if N == 1 else synth.sectioning_rho(p.H, N)
    res = _run(m, n, M, N, K, rho, world, grid)
    ref = oracle.run_split(p.H, p.g, M, N, p.lam, rho, K)
    v = np.zeros(n, complex)
    s = np.zeros((M, n), complex)
    for r in res:
        c0, c1 = r["cols"]
        i0, i1 = r["rows"]
        if r["row_group"] == 0:
            v[c0:c1] = np.array(r["v"][0]) + 1j * np.array(r["v"][1])
        s[i0:i1, c0:c1] = np.array(r["s"][0]) + 1j * np.array(r["s"][1])
        # every rank agrees on the whole problem's residual history
        hist = np.array(r["hist"])
        assert np.allclose(hist, ref.hist, rtol=1e-10, atol=1e-13 * np.max(ref.hist))
    assert np.linalg.norm(v - ref.v) <= 1e-12 * max(np.linalg.norm(ref.v), 1.0)
    assert np.linalg.norm(s - ref.s) <= 1e-12 * max(np.linalg.norm(ref.s), 1.0)


def test_rank_grids_follow_the_split():
    """Consensus shards row blocks, sectioning column blocks; both splits take
    the grid whose ranks exchange the fewest elements (Table I: m/Rr estimated
    data when the columns are split, 2n/Rc consensus values when the rows
    are); the layouts of all ranks tile the blocks exactly once."""
    assert SH.default_grid(16, 1, 4, 8192, 131072) == (4, 1)
    assert SH.default_grid(1, 8, 4, 1440, 32768) == (1, 4)
    # 4 x 4 blocks of 100 x 700 on 4 ranks: (1,4) moves 100, (2,2) 50 + 700, (4,1) 1400
    assert SH.default_grid(4, 4, 4, 100, 700) == (1, 4)
    # 7000 x 100: (1,4) moves 7000, (2,2) 3500 + 100, (4,1) 200
    assert SH.default_grid(4, 4, 4, 7000, 100) == (4, 1)
    # 1000 x 1000 on 4 ranks of a 2 x 4 split: (1,4) 1000, (2,2) 500 + 1000
    assert SH.default_grid(2, 4, 4, 1000, 1000) == (1, 4)
    for M, N, world in [(4, 4, 4), (3, 5, 6), (8, 1, 3), (1, 7, 7), (2, 6, 4)]:
        Rr, Rc = SH.default_grid(M, N, world, 100, 700)
        seen = np.zeros((M, N), int)
        for r in range(world):
            lay = SH.ShardLayout(100, 700, M, N, Rr, Rc, r)
            seen[lay.blocks_i[0]:lay.blocks_i[1], lay.blocks_j[0]:lay.blocks_j[1]] += 1
            assert rank_in(lay, lay.row_peers()) and rank_in(lay, lay.col_peers())
        assert np.all(seen == 1)
    with pytest.raises(ValueError):
        SH.default_grid(2, 1, 3, 100, 100)


def rank_in(lay, peers):
    return lay.rank in peers and len(set(peers)) == len(peers)
