"""Full-size check of the mixed-precision workload (H 8192 x 131072, 16 row
blocks of 512 rows, FP16 H with per-64-row scales) in the launch configuration
the benchmark times.

The oracle cannot iterate at this size, so the test compares the first
iteration from the zero state, which it can compute block by block: with
v = s = 0 the u-step is u_i = (H_i^H H_i + rho I)^{-1} H_i^H g_i and
v = S_kappa(mean_i u_i).  Every entry of v and of the 16 replicas u_i is
compared (complex64 H against the FP64 oracle on H, FP16 H against the FP64
oracle on the matrix the FP16 copy encodes).
"""

import os

import numpy as np
import pytest
import torch

import synth
from oracle import admm_fp64 as A
from oracle import quantize as Q
from test_gpu_parity import TOL

pytestmark = pytest.mark.gpu

M_ROWS, N_COLS, BLOCKS = synth.CONFIG3["m"], synth.CONFIG3["n"], synth.CONFIG3["row_blocks"]


def _host_memory_gb() -> float:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


@pytest.fixture(scope="module")
def large():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if _host_memory_gb() < 48:
        pytest.skip("needs about 48 GB of free host memory for the FP64 oracle")
    c = synth.CONFIG3
    H, g, u, lam = synth.gaussian_problem_device(c["m"], c["n"], c["nnz"], c["seed"])
    torch.cuda.synchronize()
    return H, g, lam, c["rho"]


def first_iteration_oracle(H_host: np.ndarray, g: np.ndarray, M: int, lam: float, rho: float,
                           encode=None):
    """v and u after one iteration of consensus ADMM from the zero state, FP64."""
    us = []
    for r0, r1 in A.balanced_blocks(H_host.shape[0], M):
        Hb = H_host[r0:r1].astype(np.complex128)
        if encode is not None:
            assert r0 % 64 == 0
            Hb = encode(Hb)
        solver = A.BlockSolver(Hb, rho)
        us.append(solver.solve(A.adjoint(solver.H, g[r0:r1])))
        del solver, Hb
    u = np.stack(us)
    v = A.soft_threshold(u.mean(axis=0), lam / (M * rho))
    return v, u


def _compare(v_gpu, u_gpu, v_ref, u_ref):
    v_gpu = v_gpu.astype(np.complex128)
    u_gpu = u_gpu.astype(np.complex128)
    rv = np.linalg.norm(v_gpu - v_ref) / max(np.linalg.norm(v_ref), 1e-30)
    ru = np.linalg.norm(u_gpu - u_ref) / max(np.linalg.norm(u_ref), 1e-30)
    assert rv <= TOL, f"v relative error {rv:.3e}"
    assert ru <= TOL, f"u relative error {ru:.3e}"
    assert np.max(np.abs(v_gpu - v_ref)) <= TOL * np.max(np.abs(v_ref))


@pytest.mark.parametrize("fp16", [False, True])
def test_mixed_precision_workload_first_iteration_full_size(large, fp16):
    import paper_1811_05571_gb300 as P
    H, g, lam, rho = large
    s = P.Solver(H, g, BLOCKS, 1, lam, rho)
    info = s.info()
    assert info["ctas"] == 152 and info["slab_cols"] >= N_COLS // 152
    if fp16:
        s.use_fp16(True)
    s.iterate(1)
    assert s.status() == 0
    v_gpu = s.v().cpu().numpy()
    u_gpu = s.u().cpu().numpy()
    s.close()
    v_ref, u_ref = first_iteration_oracle(H.cpu().numpy(), g.cpu().numpy().astype(np.complex128),
                                          BLOCKS, lam, rho, Q.dequantized if fp16 else None)
    _compare(v_gpu, u_gpu, v_ref, u_ref)
