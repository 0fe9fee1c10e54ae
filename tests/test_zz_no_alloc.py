"""The allocation-free entry point, checked against the allocating one.

admm_solve_small_noalloc serves callers that cannot allocate device memory
(a framework whose pool allocator owns the GPU, a real-time loop that must not
allocate).  Through the C ABI it must return the same image as admm_setup +
admm_iterate + admm_get_v, and a second call right after the first must not
see anything the first left in the shared scratch array.  The file is named
to be collected last."""

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _allocating_path(p, M, N, rho, iters):
    import paper_1811_05571_gb300 as P
    H = torch.from_numpy(p.H_c64()).cuda()
    g = torch.from_numpy(p.g_c64()).cuda()
    with P.Solver(H, g, M, N, p.lam, rho) as s:
        s.iterate(iters)
        assert s.status() == 0
        return s.v().cpu().numpy()


def _noalloc_path(p, M, N, rho, iters):
    import paper_1811_05571_gb300 as P
    H = torch.from_numpy(p.H_c64()).cuda()
    g = torch.from_numpy(p.g_c64()).cuda()
    v = torch.full((p.n,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    P.admm_solve_small_noalloc(H, g, p.m, p.n, M, N, p.lam, rho, iters, v)
    torch.cuda.synchronize()
    return v.cpu().numpy()


def _rho(p, N):
    from oracle import admm_fp64 as A
    return 1.0 if N == 1 else N * max(np.linalg.norm(p.H[:, c0:c1], 2) ** 2
                                      for c0, c1 in A.balanced_blocks(p.n, N))


def _check(ref, got):
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= TOL, rel
    assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))
    assert np.array_equal(got != 0, ref != 0)


def test_noalloc_matches_allocating_path_on_two_calls_in_a_row():
    a = synth.gaussian_problem(256, 4096, 16, seed=0)
    b = synth.gaussian_problem(128, 2048, 8, seed=31)
    cases = [(a, 4, 1, 100), (b, 2, 2, 60)]
    refs = [_allocating_path(p, M, N, _rho(p, N), it) for p, M, N, it in cases]
    # two calls in a row, different shapes; then the first again
    for (p, M, N, it), ref in zip(cases + cases[:1], refs + refs[:1]):
        _check(ref, _noalloc_path(p, M, N, _rho(p, N), it))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1811_05571_gb300 as P
    n, m = 65536, 1024
    H = torch.zeros((m, n), dtype=torch.complex64, device="cuda")
    g = torch.zeros(m, dtype=torch.complex64, device="cuda")
    v = torch.zeros(n, dtype=torch.complex64, device="cuda")
    with pytest.raises(P.AdmmError) as e:
        P.admm_solve_small_noalloc(H, g, m, n, 1, 1, 0.1, 1.0, 5, v)
    assert e.value.status == P.ADMM_EINVAL
    assert "8 MiB" in str(e.value)


def test_noalloc_refuses_host_buffers_before_any_kernel():
    """H, g and v_out are used in place, so host memory must be refused: the
    Python binding refuses non-CUDA tensors, and the C ABI itself returns
    ADMM_EINVAL for host pointers (numpy and pinned torch memory)."""
    import ctypes
    import paper_1811_05571_gb300 as P
    from paper_1811_05571_gb300 import _binding as B
    p = synth.gaussian_problem(64, 256, 4, seed=3)
    Hh, gh = p.H_c64(), p.g_c64()
    vh = np.zeros(p.n, dtype=np.complex64)
    with pytest.raises(TypeError):
        P.admm_solve_small_noalloc(Hh, gh, p.m, p.n, 1, 1, p.lam, 1.0, 5, vh)
    lib = B.load()
    pinned = torch.from_numpy(Hh).pin_memory()
    gd = torch.from_numpy(gh).cuda()
    vd = torch.zeros(p.n, dtype=torch.complex64, device="cuda")
    for Hp, gp, vp in ((Hh.ctypes.data, gh.ctypes.data, vh.ctypes.data),
                       (pinned.data_ptr(), gd.data_ptr(), vd.data_ptr()),
                       (ctypes.c_void_p(0), gd.data_ptr(), vd.data_ptr())):
        st = lib.admm_solve_small_noalloc(Hp, gp, p.m, p.n, 1, 1, p.lam, 1.0, 5, vp, None)
        assert st == P.ADMM_EINVAL
    torch.cuda.synchronize()
    assert not torch.any(vd != 0)


def test_noalloc_refuses_non_finite_input():
    import paper_1811_05571_gb300 as P
    p = synth.gaussian_problem(64, 256, 4, seed=3)
    H = torch.from_numpy(p.H_c64()).cuda()
    H[5, 17] = complex(float("nan"), 0.0)
    g = torch.from_numpy(p.g_c64()).cuda()
    v = torch.zeros(p.n, dtype=torch.complex64, device="cuda")
    with pytest.raises(P.AdmmError) as e:
        P.admm_solve_small_noalloc(H, g, p.m, p.n, 1, 1, p.lam, 1.0, 5, v)
    assert e.value.status == P.ADMM_ENONFINITE
    # and the next call with finite data works as before
    H[5, 17] = complex(p.H_c64()[5, 17])
    P.admm_solve_small_noalloc(H, g, p.m, p.n, 1, 1, p.lam, 1.0, 5, v)
