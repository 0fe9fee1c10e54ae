"""GPU parity of the reverse sweep (admm_batch_record / admm_batch_backward):
gradients of L = sum_b ||v_K^b - u_b||^2 with respect to g_b, lambda_b and rho
against the FP64 oracle gradient (oracle/adjoint.py, itself pinned by central
differences) on the matrix the FP16 storage encodes, relative error <= 1e-4.

Scenes whose shrinkage arguments come within 1e-5 (relative) of the threshold
at some iteration are not compared: there the loss has a kink, and an FP32
decision may differ from the FP64 one (measured: one such flip moves the
gradient by about 1e-3; scenes clear of the kink agree to about 1e-6)."""

import numpy as np
import pytest
import torch

import synth
from oracle import adjoint as AD
from oracle import admm_fp64 as A
from oracle import quantize as Q

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_05571_gb300 as P
    P.load()


def _rho(H, N):
    if N == 1:
        return 1.0
    return N * max(np.linalg.norm(H[:, c0:c1], 2) ** 2 for c0, c1 in A.balanced_blocks(H.shape[1], N))


KINK = 1e-5


def _check(H, G, U, lam, M, N, rho, K, scenes, min_checked, stop_after=None):
    import paper_1811_05571_gb300 as P
    Hq = Q.dequantized(H)
    B = G.shape[0]
    bs = P.BatchSolver(torch.from_numpy(H.astype(np.complex64)).cuda(), M, N, lam, rho)
    bs.record(K)
    bs.set_g(torch.from_numpy(G.astype(np.complex64)).cuda())
    bs.iterate(K)
    dV = np.zeros((B, H.shape[1]), np.complex128)
    refs = {}
    clear = 0
    for b in scenes:
        v, rec_a, _, _ = AD.unrolled_forward(Hq, G[b], M, N, lam[b], rho, K)
        kappa = lam[b] / (M * rho)
        margin = min(float(np.min(np.abs(np.abs(a) - kappa))) for a in rec_a) / kappa
        dV[b] = 2.0 * (v - U[b])
        refs[b] = (margin, dV[b].copy())
        clear += margin >= KINK
        if stop_after is not None and clear >= stop_after:
            break
    dG, dl, dr = bs.backward(torch.from_numpy(dV.astype(np.complex64)).cuda())
    dG = dG.cpu().numpy()
    assert bs.status() == 0
    bs.close()
    checked = 0
    for b, (margin, vb) in refs.items():
        if margin < KINK:
            continue
        g_ref, l_ref, r_ref = AD.unrolled_grad(Hq, G[b], M, N, lam[b], rho, K, vb)
        eg = np.linalg.norm(dG[b] - g_ref) / np.linalg.norm(g_ref)
        assert eg <= TOL_GRAD, f"scene {b}: g gradient relative error {eg:.3e}"
        assert abs(dl[b] - l_ref) <= TOL_GRAD * abs(l_ref), (b, dl[b], l_ref)
        assert abs(dr[b] - r_ref) <= TOL_GRAD * abs(r_ref), (b, dr[b], r_ref)
        checked += 1
    assert checked >= min_checked, checked


@pytest.mark.parametrize("M,N,K", [(4, 1, 30), (1, 4, 25), (2, 2, 25)])
def test_gaussian_gradients_match_the_oracle(M, N, K):
    p = synth.gaussian_problem(256, 4096, 16, seed=3)
    G, U, lam = synth.shared_h_scenes(p.H, 6, seed0=60, nnz=16)
    _check(p.H, G, U, lam, M, N, _rho(p.H, N), K, range(6), 3)


def test_cra_consensus_and_sectioning_gradients_match_the_oracle():
    p = synth.cra_problem()
    G, U, lam = synth.shared_h_scenes(p.H, 4, seed0=200, kind="plates")
    _check(p.H, G, U, lam, 4, 4, p.rho, 20, range(4), 1, stop_after=2)


def test_differentiable_workload_full_size():
    """H 2048 x 16384 CN(0,1/2048), 16 scenes of 64 nonzeros (seeds 500-515),
    consensus over 8 row blocks, K = 100; the first scene clear of the kink compared."""
    p = synth.gaussian_problem(2048, 16384, 64, seed=5)
    G, U, lam = synth.shared_h_scenes(p.H, 16, seed0=500, nnz=64)
    _check(p.H, G, U, lam, 8, 1, 1.0, 100, range(16), 1, stop_after=1)


def test_autograd_function_returns_the_library_gradient():
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(256, 4096, 16, seed=3)
    G, U, lam = synth.shared_h_scenes(p.H, 3, seed0=70, nnz=16)
    bs = P.BatchSolver(torch.from_numpy(p.H_c64()).cuda(), 4, 1, lam, 1.0)
    Gt = torch.from_numpy(G.astype(np.complex64)).cuda().requires_grad_(True)
    Ut = torch.from_numpy(U.astype(np.complex64)).cuda()
    V = P.UnrolledADMM.apply(Gt, bs, 20)
    loss = ((V - Ut).abs() ** 2).sum()
    loss.backward()
    dV = (2.0 * (V.detach() - Ut)).contiguous()
    bs.record(20)
    bs.set_g(Gt.detach())
    bs.iterate(20)
    dG, dl, dr = bs.backward(dV)
    assert torch.allclose(Gt.grad, dG, rtol=1e-5, atol=1e-6 * dG.abs().max().item())
    bs.close()


@pytest.mark.parametrize("M,N,K,fp16", [(4, 1, 30, False), (1, 4, 25, False), (2, 2, 25, False), (4, 1, 30, True)])
def test_single_scene_backward_matches_the_oracle(M, N, K, fp16):
    """admm_backward on a single-scene handle (complex64 or FP16 H) against the
    oracle gradient on the matrix that handle streams."""
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(256, 4096, 16, seed=3)
    rho = _rho(p.H, N)
    Hm = Q.dequantized(p.H) if fp16 else p.H
    G, U, lam = synth.shared_h_scenes(p.H, 6, seed0=60, nnz=16)
    checked = 0
    for b in range(6):
        v, rec_a, _, _ = AD.unrolled_forward(Hm, G[b], M, N, lam[b], rho, K)
        kappa = lam[b] / (M * rho)
        if min(float(np.min(np.abs(np.abs(a) - kappa))) for a in rec_a) / kappa < KINK:
            continue
        s = P.Solver(torch.from_numpy(p.H_c64()).cuda(), torch.from_numpy(G[b].astype(np.complex64)).cuda(),
                     M, N, lam[b], rho)
        if fp16:
            s.use_fp16(True)
        s.record(K)
        s.iterate(K)
        vb = 2.0 * (v - U[b])
        gg, gl, gr = s.backward(torch.from_numpy(vb.astype(np.complex64)).cuda())
        g_ref, l_ref, r_ref = AD.unrolled_grad(Hm, G[b], M, N, lam[b], rho, K, vb)
        eg = np.linalg.norm(gg.cpu().numpy() - g_ref) / np.linalg.norm(g_ref)
        assert eg <= TOL_GRAD, f"scene {b}: {eg:.3e}"
        assert abs(gl - l_ref) <= TOL_GRAD * abs(l_ref), (gl, l_ref)
        assert abs(gr - r_ref) <= TOL_GRAD * abs(r_ref), (gr, r_ref)
        # changing the data after recording invalidates the record
        s.set_g(torch.from_numpy(G[b].astype(np.complex64)).cuda())
        with pytest.raises(P.AdmmError):
            s.backward(torch.from_numpy(vb.astype(np.complex64)).cuda())
        s.close()
        checked += 1
        if checked == 2:
            break
    assert checked >= 1
