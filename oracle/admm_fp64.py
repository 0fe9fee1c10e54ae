"""FP64 CPU oracle of the paper's three distributed norm-1 ADMM variants.

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; the GPU library neither calls nor
shares code with it.

What it computes (Heredia-Juesas et al., "Consensus and Sectioning-based ADMM
with Norm-1 Regularization for Imaging with a Compressive Reflector Antenna"):

* ``lasso_admm``       -- the unsplit lasso ADMM of Section III, Eq. (original)
                          with the generic iteration of Section II (u-, v- and
                          scaled dual steps) and the residuals of Section II.
* ``consensus_admm``   -- Section III-A, row split into M blocks: Eq.
                          (x_solution), (v_variable), the dual update, and the
                          squared residual norms (Eq. primal_consensus and the
                          dual one beside it).
* ``sectioning_admm``  -- Section III-B, column split into N blocks: Eq.
                          (x_solution_columns), (v_variable_columns), the dual
                          update, the estimated data of Eq. (g_columns) and the
                          residual norms of that section.
* ``cs_admm``          -- Section III-C, M x N blocks: Eq.
                          (x_solution_rows_columns), (v_variable_rows_columns),
                          (s_variable_rows_columns), (g_rows_columns) and the
                          residual norms of that section.

Every u-step solves (H_b^* H_b + rho I) u = q with q formed literally as
H_b^* g_b + rho (v - s).  When the block has fewer rows than columns it uses
the matrix inversion lemma of Eq. (inversion_lemma) / (inversion_lemma2) /
(inversion_lemma3): u = q/rho - H_b^*/rho^2 (I + H_b H_b^*/rho)^{-1} H_b q,
with the small factor (I + H_b H_b^*/rho) Cholesky-factored once in FP64;
otherwise it factors (H_b^* H_b + rho I) directly, the branch Section III-B
recommends when the block is tall.

The estimated data of the column splits is formed from explicit products
H_q u_q of the *previous* iterate (Eq. g_columns, g_rows_columns), never from
an algebraic shortcut.

Readings where the paper is silent:
* initial state v = s = u = 0 (so every estimated datum starts at 0);
* complex sign(a) = a/|a| in the soft-threshold; |a| == kappa maps to 0;
* blocks are contiguous and balanced, the first (total mod parts) blocks one
  row / column larger (the paper assumes exact divisibility);
* the returned image is the consensus variable v (Section III-C: the final
  image is the concatenation of the v_j);
* stopping uses the primal/dual tolerances of Boyd et al. Section 3.3.1, the
  source the paper cites for its residuals.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, textbook solvers (dense solves, least squares, FISTA),
brute-force enumeration and the integers printed in Tables I-III.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


# ----------------------------------------------------------------------------
# elementary pieces
# ----------------------------------------------------------------------------

def soft_threshold(a: np.ndarray, kappa: float) -> np.ndarray:
    """Element-wise soft-thresholding S_kappa(a), Eq. (softhresholding).

    a - kappa*sign(a) where |a| > kappa, and 0 where |a| <= kappa, with the
    complex sign a/|a|."""
    a = np.asarray(a, dtype=np.complex128)
    mag = np.abs(a)
    out = np.zeros_like(a)
    keep = mag > kappa
    out[keep] = a[keep] - kappa * (a[keep] / mag[keep])
    return out


def threshold_margin(a: np.ndarray, kappa: float) -> float:
    """min_k | |a_k| - kappa | / kappa: how close the last shrinkage came to a tie."""
    if kappa <= 0.0:
        return float("inf")
    return float(np.min(np.abs(np.abs(a) - kappa)) / kappa)


def balanced_blocks(total: int, parts: int) -> list[tuple[int, int]]:
    """Contiguous [start, stop) blocks of sizes differing by at most one.

    Sections III-A..C assume N_m/M and N_p/N are integers; for other sizes the
    first (total mod parts) blocks receive one extra element."""
    if parts < 1 or parts > total:
        raise ValueError("need 1 <= parts <= total")
    base, extra = divmod(total, parts)
    out, start = [], 0
    for p in range(parts):
        size = base + (1 if p < extra else 0)
        out.append((start, start + size))
        start += size
    return out


def adjoint(Hb: np.ndarray, x: np.ndarray) -> np.ndarray:
    """H_b^* x (conjugate transpose product) without materialising H_b^*."""
    return np.conj(Hb.T @ np.conj(x))


def lemma_applies(rows: int, cols: int) -> bool:
    """The inversion lemma is used when the block has fewer rows than columns."""
    return rows < cols


class BlockSolver:
    """Solves (H_b^* H_b + rho I) u = q for one block H_b, factor cached once.

    Lemma branch (rows < cols), Eq. (inversion_lemma):
        u = q/rho - H_b^* (I + H_b H_b^*/rho)^{-1} H_b q / rho^2
    Direct branch (rows >= cols): Cholesky of H_b^* H_b + rho I."""

    def __init__(self, Hb: np.ndarray, rho: float):
        self.H = np.ascontiguousarray(Hb, dtype=np.complex128)
        self.rho = float(rho)
        rows, cols = self.H.shape
        self.lemma = lemma_applies(rows, cols)
        if self.lemma:
            small = np.eye(rows, dtype=np.complex128) + (self.H @ self.H.conj().T) / self.rho
            self.factor = sla.cho_factor(small, lower=True)
        else:
            big = self.H.conj().T @ self.H + self.rho * np.eye(cols, dtype=np.complex128)
            self.factor = sla.cho_factor(big, lower=True)

    def solve(self, q: np.ndarray) -> np.ndarray:
        if self.lemma:
            t = sla.cho_solve(self.factor, self.H @ q)
            return q / self.rho - adjoint(self.H, t) / (self.rho * self.rho)
        return sla.cho_solve(self.factor, q)


# ----------------------------------------------------------------------------
# results and stopping
# ----------------------------------------------------------------------------

HIST_FIELDS = ("rp2", "rd2", "u2", "v2", "s2")


@dataclass
class OracleResult:
    """State after the last iteration.

    v      -- consensus variable (the image), shape (n,)
    u      -- replicas, shape (M, n) (M = 1 for the unsplit and column splits)
    s      -- scaled duals, shape (M, n)
    ghat   -- estimated data of the final iterate laid out (N, m): row block i
              of column q holds H_iq u_q^i (zeros for N = 1)
    hist   -- per iteration: ||r_p||^2, ||r_d||^2, ||u||^2 (stacked replicas),
              ||v||^2 (stacked M times), ||s||^2 (stacked), shape (iters, 5)
    a_last -- the soft-threshold argument of the last v-step, shape (n,)
    """

    v: np.ndarray
    u: np.ndarray
    s: np.ndarray
    ghat: np.ndarray
    hist: np.ndarray
    a_last: np.ndarray
    kappa: float
    rows: list
    cols: list
    iters: int = 0
    stopped_at: int | None = None
    extra: dict = field(default_factory=dict)

    @property
    def margin(self) -> float:
        return threshold_margin(self.a_last, self.kappa)


def stop_test(rec: np.ndarray, p: int, rho: float, eps_abs: float, eps_rel: float) -> bool:
    """Boyd et al. Section 3.3.1 tolerances on one history record.

    ||r_p|| <= sqrt(p) eps_abs + eps_rel max(||u||, ||v||)   (c = 0 here)
    ||r_d|| <= sqrt(p) eps_abs + eps_rel rho ||s||
    with p the stacked length (replicas x unknowns)."""
    rp, rd = np.sqrt(rec[0]), np.sqrt(rec[1])
    eps_pri = np.sqrt(p) * eps_abs + eps_rel * max(np.sqrt(rec[2]), np.sqrt(rec[3]))
    eps_dual = np.sqrt(p) * eps_abs + eps_rel * rho * np.sqrt(rec[4])
    return bool(rp <= eps_pri and rd <= eps_dual)


def _sq(x: np.ndarray) -> float:
    return float(np.vdot(x, x).real)


# ----------------------------------------------------------------------------
# the four iterations
# ----------------------------------------------------------------------------

def lasso_admm(H, g, lam, rho, iters, eps=None, on_iter=None) -> OracleResult:
    """Unsplit lasso ADMM: Eq. (original) with P = I, Q = -I, c = 0.

    u <- (H^*H + rho I)^{-1}(H^* g + rho (v - s));  v <- S_{lam/rho}(u + s);
    s <- s + u - v;  r_p = u - v,  r_d = -rho (v - v_old)."""
    H = np.asarray(H, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128)
    m, n = H.shape
    solver = BlockSolver(H, rho)
    Hg = adjoint(solver.H, g)
    v = np.zeros(n, dtype=np.complex128)
    s = np.zeros(n, dtype=np.complex128)
    u = np.zeros(n, dtype=np.complex128)
    kappa = lam / rho
    hist, a, stopped = [], v, None
    for k in range(iters):
        u = solver.solve(Hg + rho * (v - s))
        a = u + s
        v_new = soft_threshold(a, kappa)
        s = s + u - v_new
        hist.append((_sq(u - v_new), rho * rho * _sq(v_new - v), _sq(u), _sq(v_new), _sq(s)))
        v = v_new
        if on_iter is not None:
            on_iter(k)
        if eps is not None and stop_test(np.array(hist[-1]), n, rho, *eps):
            stopped = k + 1
            break
    return OracleResult(v=v, u=u[None, :], s=s[None, :], ghat=np.zeros((1, m), np.complex128),
                        hist=np.array(hist).reshape(-1, 5), a_last=a, kappa=kappa,
                        rows=[(0, m)], cols=[(0, n)], iters=len(hist), stopped_at=stopped)


def consensus_admm(H, g, M, lam, rho, iters, eps=None, on_iter=None) -> OracleResult:
    """Section III-A: H split by rows into M blocks H_i with data g_i.

    u^i <- (H_i^*H_i + rho I)^{-1}(H_i^* g_i + rho (v - s^i))      Eq. (x_solution)
    v   <- S_{lam/(M rho)}(mean_i u^i + mean_i s^i)                 Eq. (v_variable)
    s^i <- s^i + u^i - v
    ||r_p||^2 = sum_i ||u^i - v||^2,  ||r_d||^2 = rho^2 M ||v - v_old||^2."""
    H = np.asarray(H, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128)
    m, n = H.shape
    rows = balanced_blocks(m, M)
    solvers = [BlockSolver(H[r0:r1], rho) for r0, r1 in rows]
    Hg = [adjoint(sv.H, g[r0:r1]) for sv, (r0, r1) in zip(solvers, rows)]
    v = np.zeros(n, dtype=np.complex128)
    s = np.zeros((M, n), dtype=np.complex128)
    u = np.zeros((M, n), dtype=np.complex128)
    kappa = lam / (M * rho)
    hist, a, stopped = [], v, None
    for k in range(iters):
        u = np.stack([solvers[i].solve(Hg[i] + rho * (v - s[i])) for i in range(M)])
        a = u.mean(axis=0) + s.mean(axis=0)
        v_new = soft_threshold(a, kappa)
        s = s + u - v_new
        rp2 = sum(_sq(u[i] - v_new) for i in range(M))
        rd2 = rho * rho * M * _sq(v_new - v)
        hist.append((rp2, rd2, sum(_sq(u[i]) for i in range(M)), M * _sq(v_new),
                     sum(_sq(s[i]) for i in range(M))))
        v = v_new
        if on_iter is not None:
            on_iter(k)
        if eps is not None and stop_test(np.array(hist[-1]), M * n, rho, *eps):
            stopped = k + 1
            break
    return OracleResult(v=v, u=u, s=s, ghat=np.zeros((1, m), np.complex128),
                        hist=np.array(hist).reshape(-1, 5), a_last=a, kappa=kappa,
                        rows=rows, cols=[(0, n)], iters=len(hist), stopped_at=stopped)


def sectioning_admm(H, g, N, lam, rho, iters, eps=None, on_iter=None) -> OracleResult:
    """Section III-B: H split by columns into N blocks H_j, u into segments u_j.

    g_j   = g - sum_{q != j} H_q u_q            (previous iterate)   Eq. (g_columns)
    u_j  <- (H_j^*H_j + rho I)^{-1}(H_j^* g_j + rho (v_j - s_j))      Eq. (x_solution_columns)
    v_j  <- S_{lam/rho}(u_j + s_j)                                    Eq. (v_variable_columns)
    s_j  <- s_j + u_j - v_j
    ||r_p||^2 = sum_j ||u_j - v_j||^2,  ||r_d||^2 = rho^2 sum_j ||v_j - v_j,old||^2."""
    H = np.asarray(H, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128)
    m, n = H.shape
    cols = balanced_blocks(n, N)
    solvers = [BlockSolver(H[:, c0:c1], rho) for c0, c1 in cols]
    u = [np.zeros(c1 - c0, dtype=np.complex128) for c0, c1 in cols]
    v = [np.zeros(c1 - c0, dtype=np.complex128) for c0, c1 in cols]
    s = [np.zeros(c1 - c0, dtype=np.complex128) for c0, c1 in cols]
    kappa = lam / rho
    hist, a_parts, stopped = [], v, None
    ghat = [np.zeros(m, dtype=np.complex128) for _ in range(N)]
    for k in range(iters):
        ghat = [solvers[q].H @ u[q] for q in range(N)]
        u_new = []
        for j in range(N):
            gj = g.copy()
            for q in range(N):
                if q != j:
                    gj = gj - ghat[q]
            u_new.append(solvers[j].solve(adjoint(solvers[j].H, gj) + rho * (v[j] - s[j])))
        a_parts = [u_new[j] + s[j] for j in range(N)]
        v_new = [soft_threshold(a_parts[j], kappa) for j in range(N)]
        s = [s[j] + u_new[j] - v_new[j] for j in range(N)]
        rp2 = sum(_sq(u_new[j] - v_new[j]) for j in range(N))
        rd2 = rho * rho * sum(_sq(v_new[j] - v[j]) for j in range(N))
        hist.append((rp2, rd2, sum(_sq(x) for x in u_new), sum(_sq(x) for x in v_new),
                     sum(_sq(x) for x in s)))
        u, v = u_new, v_new
        if on_iter is not None:
            on_iter(k)
        if eps is not None and stop_test(np.array(hist[-1]), n, rho, *eps):
            stopped = k + 1
            break
    ghat_final = np.stack([solvers[q].H @ u[q] for q in range(N)])
    return OracleResult(v=np.concatenate(v), u=np.concatenate(u)[None, :],
                        s=np.concatenate(s)[None, :], ghat=ghat_final,
                        hist=np.array(hist).reshape(-1, 5), a_last=np.concatenate(a_parts),
                        kappa=kappa, rows=[(0, m)], cols=cols, iters=len(hist),
                        stopped_at=stopped)


def cs_admm(H, g, M, N, lam, rho, iters, eps=None, on_iter=None) -> OracleResult:
    """Section III-C: M x N blocks H_ij; replicas u_j^i of each segment j.

    g_ij   = g_i - sum_{q != j} H_iq u_q^i      (previous iterate)   Eq. (g_rows_columns)
    u_j^i <- (H_ij^*H_ij + rho I)^{-1}(H_ij^* g_ij + rho (v_j - s_j^i))  Eq. (x_solution_rows_columns)
    v_j   <- S_{lam/(M rho)}(mean_i u_j^i + mean_i s_j^i)             Eq. (v_variable_rows_columns)
    s_j^i <- s_j^i + u_j^i - v_j                                      Eq. (s_variable_rows_columns)
    ||r_p||^2 = sum_i sum_j ||u_j^i - v_j||^2,
    ||r_d||^2 = rho^2 M sum_j ||v_j - v_j,old||^2."""
    H = np.asarray(H, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128)
    m, n = H.shape
    rows = balanced_blocks(m, M)
    cols = balanced_blocks(n, N)
    solvers = [[BlockSolver(H[r0:r1, c0:c1], rho) for c0, c1 in cols] for r0, r1 in rows]
    gi = [g[r0:r1] for r0, r1 in rows]
    widths = [c1 - c0 for c0, c1 in cols]
    u = [[np.zeros(w, dtype=np.complex128) for w in widths] for _ in range(M)]
    s = [[np.zeros(w, dtype=np.complex128) for w in widths] for _ in range(M)]
    v = [np.zeros(w, dtype=np.complex128) for w in widths]
    kappa = lam / (M * rho)
    hist, a_parts, stopped = [], v, None
    for k in range(iters):
        ghat = [[solvers[i][q].H @ u[i][q] for q in range(N)] for i in range(M)]
        u_new = [[None] * N for _ in range(M)]
        for i in range(M):
            for j in range(N):
                gij = gi[i].copy()
                for q in range(N):
                    if q != j:
                        gij = gij - ghat[i][q]
                q_rhs = adjoint(solvers[i][j].H, gij) + rho * (v[j] - s[i][j])
                u_new[i][j] = solvers[i][j].solve(q_rhs)
        a_parts = [np.stack([u_new[i][j] for i in range(M)]).mean(axis=0)
                   + np.stack([s[i][j] for i in range(M)]).mean(axis=0) for j in range(N)]
        v_new = [soft_threshold(a_parts[j], kappa) for j in range(N)]
        s = [[s[i][j] + u_new[i][j] - v_new[j] for j in range(N)] for i in range(M)]
        rp2 = sum(_sq(u_new[i][j] - v_new[j]) for i in range(M) for j in range(N))
        rd2 = rho * rho * M * sum(_sq(v_new[j] - v[j]) for j in range(N))
        hist.append((rp2, rd2,
                     sum(_sq(u_new[i][j]) for i in range(M) for j in range(N)),
                     M * sum(_sq(x) for x in v_new),
                     sum(_sq(s[i][j]) for i in range(M) for j in range(N))))
        u, v = u_new, v_new
        if on_iter is not None:
            on_iter(k)
        if eps is not None and stop_test(np.array(hist[-1]), M * n, rho, *eps):
            stopped = k + 1
            break
    ghat_final = np.zeros((N, m), dtype=np.complex128)
    for i, (r0, r1) in enumerate(rows):
        for q in range(N):
            ghat_final[q, r0:r1] = solvers[i][q].H @ u[i][q]
    return OracleResult(v=np.concatenate(v),
                        u=np.stack([np.concatenate(u[i]) for i in range(M)]),
                        s=np.stack([np.concatenate(s[i]) for i in range(M)]),
                        ghat=ghat_final, hist=np.array(hist).reshape(-1, 5),
                        a_last=np.concatenate(a_parts), kappa=kappa, rows=rows, cols=cols,
                        iters=len(hist), stopped_at=stopped)


def run_split(H, g, row_blocks, col_blocks, lam, rho, iters, eps=None, on_iter=None) -> OracleResult:
    """Dispatch on (M, N): (1,1) unsplit, (M,1) consensus, (1,N) sectioning, else C&S.

    ``on_iter(k)``, when given, is called after iteration k (0-based) completes;
    it observes only (the CPU baseline times iterations with it)."""
    if row_blocks == 1 and col_blocks == 1:
        return lasso_admm(H, g, lam, rho, iters, eps, on_iter)
    if col_blocks == 1:
        return consensus_admm(H, g, row_blocks, lam, rho, iters, eps, on_iter)
    if row_blocks == 1:
        return sectioning_admm(H, g, col_blocks, lam, rho, iters, eps, on_iter)
    return cs_admm(H, g, row_blocks, col_blocks, lam, rho, iters, eps, on_iter)


# ----------------------------------------------------------------------------
# Section IV: elements exchanged by one node per iteration (Table I)
# ----------------------------------------------------------------------------

def comm_elements(M: int, N: int, Nm: int, Np: int) -> dict:
    """Table I: 2 N_p (row split), N N_m (column split), N N_m/M + 2 N_p/N (both)."""
    return {
        "consensus": 2 * Np,
        "sectioning": N * Nm,
        "cs": N * Nm / M + 2 * Np / N,
    }
