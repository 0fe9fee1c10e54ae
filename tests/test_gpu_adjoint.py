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


def test_autograd_fills_g_lambda_and_rho_gradients():
    """loss.backward() through UnrolledADMM fills G.grad, lam.grad (one per
    scene) and rho.grad (summed over the scenes, rho being shared) with the
    library's reverse-sweep gradient."""
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(256, 4096, 16, seed=3)
    G, U, lam = synth.shared_h_scenes(p.H, 3, seed0=70, nnz=16)
    bs = P.BatchSolver(torch.from_numpy(p.H_c64()).cuda(), 4, 1, lam, 1.0)
    Gt = torch.from_numpy(G.astype(np.complex64)).cuda().requires_grad_(True)
    lam_t = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    rho_t = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    Ut = torch.from_numpy(U.astype(np.complex64)).cuda()
    V = P.UnrolledADMM.apply(Gt, lam_t, rho_t, bs, 20)
    loss = ((V - Ut).abs() ** 2).sum()
    loss.backward()
    dV = (2.0 * (V.detach() - Ut)).contiguous()
    bs.record(20)
    bs.set_g(Gt.detach())
    bs.iterate(20)
    dG, dl, dr = bs.backward(dV)
    assert torch.allclose(Gt.grad, dG, rtol=1e-5, atol=1e-6 * dG.abs().max().item())
    # a second forward and reverse sweep: the same gradient up to the order of
    # the FP32 partial sums of the split products
    assert np.allclose(lam_t.grad.numpy(), dl, rtol=1e-6, atol=0)
    assert abs(rho_t.grad.item() - float(np.sum(dr))) <= 1e-6 * abs(float(np.sum(dr)))
    bs.close()


def test_autograd_with_new_lambda_and_rho_matches_the_oracle():
    """Values of lam and rho other than the solver's are pushed to it
    (admm_batch_set_lambda, admm_batch_set_rho: refactorisation); the images
    and the gradients then match the FP64 oracle run with the new values on
    the matrix the FP16 storage encodes."""
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(256, 4096, 16, seed=3)
    M, N, K = 2, 2, 20
    G, U, lam = synth.shared_h_scenes(p.H, 4, seed0=90, nnz=16)
    rho0 = _rho(p.H, N)
    bs = P.BatchSolver(torch.from_numpy(p.H_c64()).cuda(), M, N, lam, rho0)
    lam1 = [1.3 * x for x in lam]
    rho1 = 1.5 * rho0
    Gt = torch.from_numpy(G.astype(np.complex64)).cuda().requires_grad_(True)
    lam_t = torch.tensor(lam1, dtype=torch.float64, requires_grad=True)
    rho_t = torch.tensor(rho1, dtype=torch.float64, requires_grad=True)
    V = P.UnrolledADMM.apply(Gt, lam_t, rho_t, bs, K)
    Vn = V.detach().cpu().numpy()
    Ut = torch.from_numpy(U.astype(np.complex64)).cuda()
    ((V - Ut).abs() ** 2).sum().backward()
    Hq = Q.dequantized(p.H)
    rho_ref, checked = 0.0, 0
    for b in range(4):
        v, rec_a, _, _ = AD.unrolled_forward(Hq, G[b], M, N, lam1[b], rho1, K)
        assert np.linalg.norm(Vn[b] - v) <= 1e-5 * np.linalg.norm(v)
        vb = 2.0 * (v - U[b])
        g_ref, l_ref, r_ref = AD.unrolled_grad(Hq, G[b], M, N, lam1[b], rho1, K, vb)
        rho_ref += r_ref
        kappa = lam1[b] / (M * rho1)
        if min(float(np.min(np.abs(np.abs(a) - kappa))) for a in rec_a) / kappa < KINK:
            continue
        eg = np.linalg.norm(Gt.grad[b].cpu().numpy() - g_ref) / np.linalg.norm(g_ref)
        assert eg <= TOL_GRAD, (b, eg)
        assert abs(lam_t.grad[b].item() - l_ref) <= TOL_GRAD * abs(l_ref), (b, lam_t.grad[b].item(), l_ref)
        checked += 1
    assert checked >= 2
    assert abs(rho_t.grad.item() - rho_ref) <= TOL_GRAD * abs(rho_ref), (rho_t.grad.item(), rho_ref)
    bs.close()


# ---------------------------------------------------------------------------
# the differentiable workload with complex64 H: one Solver per scene
# ---------------------------------------------------------------------------

C5 = dict(m=2048, n=16384, nnz=64, seed=5, scenes=16, seed0=500, M=8, K=100)


def _c5_oracle_grad(p, G, U, lam, b: int):
    """Oracle margin of scene b of the differentiable workload on the complex64 H,
    and its FP64 gradient when the scene is clear of the kink (else None)."""
    v, rec_a, _, _ = AD.unrolled_forward(p.H, G[b], C5["M"], 1, lam[b], 1.0, C5["K"])
    kappa = lam[b] / C5["M"]
    margin = min(float(np.min(np.abs(np.abs(a) - kappa))) for a in rec_a) / kappa
    if margin < KINK:
        return margin, None
    return margin, AD.unrolled_grad(p.H, G[b], C5["M"], 1, lam[b], 1.0, C5["K"], 2.0 * (v - U[b]))


@pytest.fixture(scope="module")
def c5_gpu():
    """The differentiable workload through UnrolledADMM over 16 complex64
    single-scene handles: images and the gradients in G, lam and rho."""
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(C5["m"], C5["n"], C5["nnz"], seed=C5["seed"])
    G, U, lam = synth.shared_h_scenes(p.H, C5["scenes"], seed0=C5["seed0"], nnz=C5["nnz"])
    Hd = torch.from_numpy(p.H_c64()).cuda()
    Gd = torch.from_numpy(G.astype(np.complex64)).cuda()
    solvers = [P.Solver(Hd, Gd[b], C5["M"], 1, lam[b], 1.0) for b in range(C5["scenes"])]
    Gt = Gd.clone().requires_grad_(True)
    lam_t = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    rho_t = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    Ut = torch.from_numpy(U.astype(np.complex64)).cuda()
    V = P.UnrolledADMM.apply(Gt, lam_t, rho_t, solvers, C5["K"])
    ((V - Ut).abs() ** 2).sum().backward()
    # per-scene rho gradients (the autograd output is their sum)
    dV = (2.0 * (V.detach() - Ut)).contiguous()
    per_rho = [sv.backward(dV[b])[2] for b, sv in enumerate(solvers)]
    out = dict(p=p, G=G, U=U, lam=lam, V=V.detach().cpu().numpy(), g_bar=Gt.grad.cpu().numpy(),
               lam_bar=lam_t.grad.numpy().copy(), rho_bar=rho_t.grad.item(), per_rho=per_rho)
    for sv in solvers:
        assert sv.status() == 0
        sv.close()
    return out


def test_differentiable_workload_complex64_every_scene(c5_gpu):
    """All 16 scenes of the differentiable workload (H 2048 x 16384 complex64,
    consensus 8 x 1, K = 100) against the FP64 oracle gradient on the same H:
    every scene clear of the kink (no shrinkage argument within 1e-5 of the
    threshold at any of the 100 iterations) is compared, in G, lambda and rho."""
    # rho_bar through autograd is the sum of the per-scene values (a second
    # reverse sweep over the same records: equal up to FP64 atomic order)
    assert abs(c5_gpu["rho_bar"] - sum(c5_gpu["per_rho"])) <= 1e-6 * abs(sum(c5_gpu["per_rho"]))
    p, G, U, lam = c5_gpu["p"], c5_gpu["G"], c5_gpu["U"], c5_gpu["lam"]
    checked = 0
    for b in range(C5["scenes"]):
        margin, ref = _c5_oracle_grad(p, G, U, lam, b)
        if ref is None:
            continue
        g_ref, l_ref, r_ref = ref
        eg = np.linalg.norm(c5_gpu["g_bar"][b] - g_ref) / np.linalg.norm(g_ref)
        assert eg <= TOL_GRAD, f"scene {b}: g gradient relative error {eg:.3e}"
        assert abs(c5_gpu["lam_bar"][b] - l_ref) <= TOL_GRAD * abs(l_ref), (b, c5_gpu["lam_bar"][b], l_ref)
        assert abs(c5_gpu["per_rho"][b] - r_ref) <= TOL_GRAD * abs(r_ref), (b, c5_gpu["per_rho"][b], r_ref)
        checked += 1
    # measured: 4 of the 16 scenes stay clear of the kink over 100 iterations
    assert checked >= 3, checked


def test_differentiable_workload_gradient_matches_central_differences(c5_gpu):
    """The GPU gradient of scene 0 against central differences (h = 1e-6) of the
    FP64 oracle's loss ||v_K - u||^2, along three random unit directions in g
    and in lambda and rho, at the full workload size."""
    p, G, U, lam = c5_gpu["p"], c5_gpu["G"], c5_gpu["U"], c5_gpu["lam"]
    M, K = C5["M"], C5["K"]
    b = 0
    for b in range(C5["scenes"]):
        _, rec_a, _, _ = AD.unrolled_forward(p.H, G[b], M, 1, lam[b], 1.0, K)
        if min(float(np.min(np.abs(np.abs(a) - lam[b] / M))) for a in rec_a) / (lam[b] / M) >= 1e-4:
            break

    def loss(g, lm, rh):
        v = A.run_split(p.H, g, M, 1, lm, rh, K).v
        return float(np.sum(np.abs(v - U[b]) ** 2))

    h = 1e-6
    rng = np.random.default_rng(11)
    gb = c5_gpu["g_bar"][b].astype(np.complex128)
    for _ in range(3):
        d = rng.standard_normal(p.m) + 1j * rng.standard_normal(p.m)
        d /= np.linalg.norm(d)
        fd = (loss(G[b] + h * d, lam[b], 1.0) - loss(G[b] - h * d, lam[b], 1.0)) / (2 * h)
        an = float(np.real(np.vdot(gb, d)))
        assert abs(fd - an) <= TOL_GRAD * max(abs(fd), np.linalg.norm(gb)), (fd, an)
    hl = 1e-6 * lam[b]
    fd_l = (loss(G[b], lam[b] + hl, 1.0) - loss(G[b], lam[b] - hl, 1.0)) / (2 * hl)
    assert abs(fd_l - c5_gpu["lam_bar"][b]) <= TOL_GRAD * abs(fd_l), (fd_l, c5_gpu["lam_bar"][b])
    hr = 1e-6
    fd_r = (loss(G[b], lam[b], 1.0 + hr) - loss(G[b], lam[b], 1.0 - hr)) / (2 * hr)
    assert abs(fd_r - c5_gpu["per_rho"][b]) <= TOL_GRAD * abs(fd_r), (fd_r, c5_gpu["per_rho"][b])


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
