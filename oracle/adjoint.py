"""Gradient of a loss of the image after K unrolled iterations, FP64 CPU
restatement (TEST INFRASTRUCTURE ONLY: imported by tests/ and bench.py's CPU
legs, never by the GPU library).

The iteration of Sections III-A..C, written with w_ij = K_ij^{-1} r_ij
(K_ij = rho I + H_ij H_ij^H, the inversion lemma), is

    gt_ij  = g_i - sum_{q != j} ghat_iq                (previous iterate)
    r_ij   = gt_ij - H_ij (v_j - s_j^i)
    w_ij   = K_ij^{-1} r_ij
    u_j^i  = v_j - s_j^i + H_ij^H w_ij
    ghat'  = gt_ij - rho w_ij                          (= H_ij u_j^i)
    a_j    = mean_i (u_j^i + s_j^i)
    v_j'   = S_kappa(a_j),  kappa = lambda / (M rho)   (Eq. softhresholding)
    s_j^i' = s_j^i + u_j^i - v_j'

from v = s = 0, ghat = 0.  Its only non-linear step is the complex
soft-threshold, and rho enters through K_ij, through ghat' and through kappa,
so the reverse sweep needs only the recorded a^k and w^k of every iteration.
Complex adjoints follow the convention x_bar = dL/dRe(x) + i dL/dIm(x) (so that
dL = Re(conj(x_bar) dx)); for |a| > kappa, with a_hat = a/|a|,

    a_bar     = t - (kappa/|a|) (t - a_hat Re(conj(a_hat) t)),
    kappa_bar = -Re(conj(a_hat) t),

and both are zero where |a| <= kappa; dw/drho = -K^{-1} w.
"""

from __future__ import annotations

import numpy as np

from .admm_fp64 import adjoint, balanced_blocks, soft_threshold


def _blocks(H, M, N):
    m, n = H.shape
    return balanced_blocks(m, M), balanced_blocks(n, N)


def unrolled_forward(H, g, M, N, lam, rho, iters):
    """K iterations from the zero state; returns v_K and the records (a^k, w^k)."""
    H = np.asarray(H, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128)
    m, n = H.shape
    rows, cols = _blocks(H, M, N)
    Kinv = [[np.linalg.inv(rho * np.eye(r1 - r0) + H[r0:r1, c0:c1] @ H[r0:r1, c0:c1].conj().T)
             for c0, c1 in cols] for r0, r1 in rows]
    v = np.zeros(n, complex)
    s = np.zeros((M, n), complex)
    gh = [[np.zeros(r1 - r0, complex) for _ in cols] for r0, r1 in rows]
    kappa = lam / (M * rho)
    rec_a, rec_w = [], []
    for _ in range(iters):
        w = [[None] * N for _ in range(M)]
        gh_new = [[None] * N for _ in range(M)]
        sig_sum = np.zeros(n, complex)
        sig = [[None] * N for _ in range(M)]
        for i, (r0, r1) in enumerate(rows):
            for j, (c0, c1) in enumerate(cols):
                Hb = H[r0:r1, c0:c1]
                gt = g[r0:r1] - sum(gh[i][q] for q in range(N) if q != j)
                z = v[c0:c1] - s[i, c0:c1]
                w[i][j] = Kinv[i][j] @ (gt - Hb @ z)
                gh_new[i][j] = gt - rho * w[i][j]
                sig[i][j] = adjoint(Hb, w[i][j])
                sig_sum[c0:c1] += sig[i][j]
        a = v + sig_sum / M
        vn = soft_threshold(a, kappa)
        for i in range(M):
            for j, (c0, c1) in enumerate(cols):
                s[i, c0:c1] = v[c0:c1] + sig[i][j] - vn[c0:c1]
        v, gh = vn, gh_new
        rec_a.append(a)
        rec_w.append(w)
    return v, rec_a, rec_w, Kinv


def unrolled_grad(H, g, M, N, lam, rho, iters, v_bar):
    """(g_bar, lambda_bar, rho_bar) of a real loss L(v_K) with dL/dv_K given as
    v_bar (same convention), by the reverse sweep over the recorded iterations."""
    H = np.asarray(H, dtype=np.complex128)
    m, n = H.shape
    rows, cols = _blocks(H, M, N)
    _, rec_a, rec_w, Kinv = unrolled_forward(H, g, M, N, lam, rho, iters)
    kappa = lam / (M * rho)
    vb = np.asarray(v_bar, dtype=np.complex128).copy()      # adjoint of v after the iteration
    sb = np.zeros((M, n), complex)                          # of s
    ghb = [[np.zeros(r1 - r0, complex) for _ in cols] for r0, r1 in rows]   # of ghat
    g_bar = np.zeros(m, complex)
    kappa_bar = 0.0
    rho_bar = 0.0
    for k in range(iters - 1, -1, -1):
        a, w = rec_a[k], rec_w[k]
        # s' = v + sigma - v'  and  v' = S(a): the adjoint reaching v' in total
        t = vb - sb.sum(axis=0)
        mag = np.abs(a)
        keep = mag > kappa
        ahat = np.zeros_like(a)
        ahat[keep] = a[keep] / mag[keep]
        proj = np.real(np.conj(ahat) * t)
        a_bar = np.zeros_like(a)
        a_bar[keep] = t[keep] - (kappa / mag[keep]) * (t[keep] - ahat[keep] * proj[keep])
        kappa_bar += -float(np.sum(proj[keep]))
        # a = v + mean_i sigma_i, s' = v + sigma - v'
        vb_new = sb.sum(axis=0) + a_bar
        sb_new = np.zeros_like(sb)
        ghb_new = [[np.zeros(r1 - r0, complex) for _ in cols] for r0, r1 in rows]
        gtb = [[None] * N for _ in range(M)]
        for i, (r0, r1) in enumerate(rows):
            for j, (c0, c1) in enumerate(cols):
                Hb = H[r0:r1, c0:c1]
                sig_bar = sb[i, c0:c1] + a_bar[c0:c1] / M
                # sigma = H^H w, ghat' = gt - rho w
                w_bar = Hb @ sig_bar - rho * ghb[i][j]
                rho_bar += -float(np.real(np.vdot(w[i][j], ghb[i][j])))
                # w = K^{-1} r, dw/drho = -K^{-1} w
                r_bar = Kinv[i][j] @ w_bar
                rho_bar += -float(np.real(np.vdot(w[i][j], r_bar)))
                gtb[i][j] = ghb[i][j] + r_bar
                # r = gt - H z, z = v - s
                z_bar = -adjoint(Hb, r_bar)
                vb_new[c0:c1] += z_bar
                sb_new[i, c0:c1] = -z_bar
        # gt_ij = g_i - sum_{q != j} ghat_iq
        for i, (r0, r1) in enumerate(rows):
            tot = sum(gtb[i][j] for j in range(N))
            g_bar[r0:r1] += tot
            for q in range(N):
                ghb_new[i][q] = -(tot - gtb[i][q])
        vb, sb, ghb = vb_new, sb_new, ghb_new
    lam_bar = kappa_bar / (M * rho)
    rho_bar += -kappa_bar * lam / (M * rho * rho)
    return g_bar, lam_bar, rho_bar
