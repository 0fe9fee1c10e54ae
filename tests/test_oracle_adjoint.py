"""Pins of the FP64 unrolled-iteration gradient (oracle/adjoint.py): its forward
sweep against the literal oracle (oracle.run_split), and the gradient against
central finite differences of the literal oracle's loss in FP64, along random
directions in g and in lambda and rho (directions that move a shrinkage
argument across the threshold are not used: the loss has a kink there)."""

import numpy as np
import pytest

import oracle
import synth
from oracle import adjoint as AD


def _problem(m, n, seed):
    p = synth.gaussian_problem(m, n, 6, seed=seed)
    return p


CASES = [
    (64, 256, 2, 1, 25),    # consensus
    (64, 256, 1, 2, 25),    # sectioning
    (64, 256, 2, 2, 20),    # consensus and sectioning
    (48, 160, 1, 1, 30),    # unsplit
]


def _rho(p, N):
    if N == 1:
        return 1.0
    from oracle import admm_fp64 as A
    return N * max(np.linalg.norm(p.H[:, c0:c1], 2) ** 2 for c0, c1 in A.balanced_blocks(p.n, N))


@pytest.mark.parametrize("m,n,M,N,K", CASES)
def test_rearranged_forward_equals_the_literal_oracle(m, n, M, N, K):
    p = _problem(m, n, m + n + M + N)
    rho = _rho(p, N)
    v, rec_a, rec_w, _ = AD.unrolled_forward(p.H, p.g, M, N, p.lam, rho, K)
    ref = oracle.run_split(p.H, p.g, M, N, p.lam, rho, K)
    assert np.linalg.norm(v - ref.v) <= 1e-12 * max(np.linalg.norm(ref.v), 1.0)
    assert np.allclose(rec_a[-1], ref.a_last, rtol=0, atol=1e-12)


def _loss(p, M, N, lam, rho, K, g):
    v = oracle.run_split(p.H, g, M, N, lam, rho, K).v
    return float(np.sum(np.abs(v - p.u_true) ** 2))


def _margin(p, M, N, lam, rho, K, g):
    _, rec_a, _, _ = AD.unrolled_forward(p.H, g, M, N, lam, rho, K)
    kappa = lam / (M * rho)
    return min(float(np.min(np.abs(np.abs(a) - kappa))) for a in rec_a)


@pytest.mark.parametrize("m,n,M,N,K", CASES)
def test_gradient_matches_central_differences(m, n, M, N, K):
    p = _problem(m, n, m + n + M + N)
    rho = _rho(p, N)
    lam = p.lam
    v, _, _, _ = AD.unrolled_forward(p.H, p.g, M, N, lam, rho, K)
    v_bar = 2.0 * (v - p.u_true)                     # dL/dv for L = sum |v - u|^2
    g_bar, lam_bar, rho_bar = AD.unrolled_grad(p.H, p.g, M, N, lam, rho, K, v_bar)
    h = 1e-6
    rng = np.random.default_rng(7)
    checked = 0
    for _ in range(12):
        d = rng.standard_normal(m) + 1j * rng.standard_normal(m)
        d /= np.linalg.norm(d)
        if min(_margin(p, M, N, lam, rho, K, p.g + h * d), _margin(p, M, N, lam, rho, K, p.g - h * d)) < 1e-7:
            continue
        fd = (_loss(p, M, N, lam, rho, K, p.g + h * d) - _loss(p, M, N, lam, rho, K, p.g - h * d)) / (2 * h)
        an = float(np.real(np.vdot(g_bar, d)))
        assert abs(fd - an) <= 1e-5 * max(abs(fd), np.linalg.norm(g_bar)), (fd, an)
        checked += 1
        if checked == 8:
            break
    assert checked >= 6
    for name, val, bar in (("lambda", lam, lam_bar), ("rho", rho, rho_bar)):
        hh = 1e-6 * val
        args = dict(lam=lam, rho=rho)
        plus = dict(args, **{"lam" if name == "lambda" else "rho": val + hh})
        minus = dict(args, **{"lam" if name == "lambda" else "rho": val - hh})
        fd = (_loss(p, M, N, plus["lam"], plus["rho"], K, p.g)
              - _loss(p, M, N, minus["lam"], minus["rho"], K, p.g)) / (2 * hh)
        assert abs(fd - bar) <= 1e-5 * max(abs(fd), 1e-8), (name, fd, bar)


def _mutant(old, new):
    src = open(AD.__file__).read()
    bad = src.replace(old, new)
    assert bad != src
    ns = {"__name__": "oracle.adjoint_mutant", "__package__": "oracle"}
    exec(compile(bad, "adjoint_mutant", "exec"), ns)
    return ns["unrolled_grad"]


@pytest.mark.parametrize("old,new", [
    # sign of the projection term of the soft-threshold Jacobian
    ("t[keep] - (kappa / mag[keep]) * (t[keep] - ahat[keep] * proj[keep])",
     "t[keep] + (kappa / mag[keep]) * (t[keep] - ahat[keep] * proj[keep])"),
    # the d w / d rho term dropped
    ("rho_bar += -float(np.real(np.vdot(w[i][j], r_bar)))", "rho_bar += 0.0"),
    # H instead of H^H in the adjoint of r = gt - H z
    ("z_bar = -adjoint(Hb, r_bar)", "z_bar = -(Hb.T @ r_bar)"),
])
def test_planted_mistakes_in_the_adjoint_fail_the_difference_check(old, new):
    p = _problem(64, 256, 2 + 64 + 256)
    M, N, K = 2, 2, 20
    rho = _rho(p, N)
    grad = _mutant(old, new)
    v, _, _, _ = AD.unrolled_forward(p.H, p.g, M, N, p.lam, rho, K)
    g_bar, lam_bar, rho_bar = grad(p.H, p.g, M, N, p.lam, rho, K, 2.0 * (v - p.u_true))
    h = 1e-6
    d = np.random.default_rng(3).standard_normal(64) + 0j
    d /= np.linalg.norm(d)
    fd_g = (_loss(p, M, N, p.lam, rho, K, p.g + h * d) - _loss(p, M, N, p.lam, rho, K, p.g - h * d)) / (2 * h)
    hr = 1e-6 * rho
    fd_r = (_loss(p, M, N, p.lam, rho + hr, K, p.g) - _loss(p, M, N, p.lam, rho - hr, K, p.g)) / (2 * hr)
    err_g = abs(fd_g - float(np.real(np.vdot(g_bar, d)))) / max(abs(fd_g), 1e-12)
    err_r = abs(fd_r - rho_bar) / max(abs(fd_r), 1e-12)
    assert max(err_g, err_r) > 1e-3, (err_g, err_r)
