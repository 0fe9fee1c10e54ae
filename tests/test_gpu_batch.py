"""GPU parity of the batched shared-H solver (admm_batch_*, tensor-core GEMMs).

Products: Y = Hq X and X = Hq^H Y for every scene against FP64 products of the
matrix the FP16 storage encodes (Hq = oracle.quantize.dequantized(H)), per
scene relative error <= 1e-5.  Iterations: each scene of the batch against the
FP64 oracle run on Hq with that scene's data and lambda, at the 1e-5 bar of
the single-scene path.
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import admm_fp64 as A
from oracle import quantize as Q
from test_gpu_parity import TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_05571_gb300 as P
    P.load()


def _rel_rows(a, b):
    a = np.asarray(a, dtype=np.complex128)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-30)


@pytest.fixture(scope="module")
def cra():
    return synth.cra_problem()


@pytest.mark.parametrize("m,n,M,N,B", [
    (256, 4096, 2, 1, 5),       # batch smaller than one tile of 64 scenes
    (256, 4096, 1, 4, 70),      # two column tiles, sectioning blocks
    (300, 3000, 3, 2, 9),       # ragged row tiles (100 rows), 1500-column blocks
    (1440, 32768, 8, 1, 64),    # CRA-shaped consensus: split-K forward product
    (1440, 32768, 1, 8, 17),
    (1440, 32768, 4, 4, 130),   # three column tiles
])
def test_forward_and_adjoint_products(m, n, M, N, B, cra):
    import paper_1811_05571_gb300 as P
    H = cra.H if (m, n) == (1440, 32768) else synth.gaussian_problem(m, n, 8, seed=1).H
    Hq = Q.dequantized(H)
    bs = P.BatchSolver(torch.from_numpy(H.astype(np.complex64)).cuda(), M, N, [0.1] * B, 1.0)
    rng = np.random.default_rng(m + n + B)
    X = (rng.standard_normal((B, n)) + 1j * rng.standard_normal((B, n))).astype(np.complex64)
    X[0] *= 1e-3                      # scenes of different magnitude get their own scales
    Y = bs.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    err = _rel_rows(Y, (Hq @ X.astype(np.complex128).T).T)
    assert err.max() <= TOL, err.max()
    Yin = (rng.standard_normal((B, m)) + 1j * rng.standard_normal((B, m))).astype(np.complex64)
    Xo = bs.adjoint(torch.from_numpy(Yin).cuda()).cpu().numpy()
    err = _rel_rows(Xo, (Hq.conj().T @ Yin.astype(np.complex128).T).T)
    assert err.max() <= TOL, err.max()
    assert bs.status() == 0
    bs.close()


def _run_batch(H, G, lam, M, N, rho, iters):
    import paper_1811_05571_gb300 as P
    bs = P.BatchSolver(torch.from_numpy(H.astype(np.complex64)).cuda(), M, N, lam, rho)
    bs.set_g(torch.from_numpy(G.astype(np.complex64)).cuda())
    bs.iterate(iters)
    V = bs.v().cpu().numpy()
    res = bs.residuals()
    assert bs.status() == 0
    bs.close()
    return V, res


def _check_scene(V, res, Hq, G, lam, M, N, rho, iters, b):
    ref = oracle.run_split(Hq, G[b], M, N, lam[b], rho, iters)
    v_ref = ref.v
    rel = np.linalg.norm(V[b].astype(np.complex128) - v_ref) / max(np.linalg.norm(v_ref), 1e-30)
    assert rel <= TOL, f"scene {b}: v relative error {rel:.3e}"
    band = TOL * max(np.max(np.abs(ref.a_last)), 1e-30)
    ambiguous = np.abs(np.abs(ref.a_last) - ref.kappa) <= band
    assert not ((V[b] != 0) != (v_ref != 0))[~ambiguous].any(), f"scene {b}: support differs"
    # last residual record, to 1e-4 of the history's maximum (the bar of the single-scene path)
    for q in range(2):
        a, e = np.sqrt(res[b, q]), np.sqrt(ref.hist[-1, q])
        assert abs(a - e) <= 1e-4 * np.sqrt(ref.hist[:, q]).max(), (b, q, a, e)


def test_batch_gaussian_consensus_matches_the_oracle_per_scene():
    p = synth.gaussian_problem(256, 4096, 16, seed=0)
    G, _, lam = synth.shared_h_scenes(p.H, 6, seed0=40, nnz=16)
    V, res = _run_batch(p.H, G, lam, 4, 1, 1.0, 300)
    Hq = Q.dequantized(p.H)
    for b in (0, 3, 5):
        _check_scene(V, res, Hq, G, lam, 4, 1, 1.0, 300, b)


@pytest.mark.parametrize("M,N", [(8, 1), (1, 8), (4, 4)])
def test_batch_cra_splits_match_the_oracle_per_scene(cra, M, N):
    G, _, lam = synth.shared_h_scenes(cra.H, 8, seed0=100, kind="plates")
    V, res = _run_batch(cra.H, G, lam, M, N, cra.rho, 50)
    Hq = Q.dequantized(cra.H)
    for b in (0, 7):
        _check_scene(V, res, Hq, G, lam, M, N, cra.rho, 50, b)


def test_batch_scenes_are_independent():
    """A scene's iterates do not depend on the other scenes of the batch
    (tile position, neighbours' magnitudes)."""
    p = synth.gaussian_problem(256, 4096, 16, seed=0)
    G, _, lam = synth.shared_h_scenes(p.H, 70, seed0=7, nnz=16)
    V70, _ = _run_batch(p.H, G, lam, 2, 2, 2 * max(np.linalg.norm(p.H[:, c0:c1], 2) ** 2
                                                    for c0, c1 in A.balanced_blocks(4096, 2)), 40)
    V3, _ = _run_batch(p.H, G[[0, 65, 69]], [lam[0], lam[65], lam[69]], 2, 2,
                       2 * max(np.linalg.norm(p.H[:, c0:c1], 2) ** 2 for c0, c1 in A.balanced_blocks(4096, 2)), 40)
    # the K split of the forward product depends on the batch size, so the
    # summation order (not the arithmetic of a scene) may differ
    for k, b in enumerate((0, 65, 69)):
        ref = V70[b].astype(np.complex128)
        assert np.linalg.norm(V3[k] - ref) <= 1e-6 * np.linalg.norm(ref)


def test_autotuned_split_keeps_parity():
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(256, 4096, 16, seed=0)
    G, _, lam = synth.shared_h_scenes(p.H, 6, seed0=40, nnz=16)
    bs = P.BatchSolver(torch.from_numpy(p.H_c64()).cuda(), 4, 1, lam, 1.0)
    bs.set_g(torch.from_numpy(G.astype(np.complex64)).cuda())
    sp = bs.tune()
    assert sp >= 1 and (sp & (sp - 1)) == 0
    bs.iterate(300)
    V = bs.v().cpu().numpy()
    res = bs.residuals()
    bs.close()
    _check_scene(V, res, Q.dequantized(p.H), G, lam, 4, 1, 1.0, 300, 2)
