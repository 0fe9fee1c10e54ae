"""FP64 per-rank engine of the sharded iteration, for tests of the host logic.

TEST INFRASTRUCTURE: the rank's blocks of an M x N split solved with the FP64
oracle's block solver (oracle.admm_fp64.BlockSolver), with the same interface
as paper_1811_05571_gb300.sharded.CudaShardEngine, so that the partitioning
and the exchanges of the sharded driver can run on CPU ranks and be compared
with the single-process oracle.  Per iteration (Section III-C with the other
ranks' blocks folded into the exchanged sums):
  gt_ij = (g_i - T_i + t_i) - sum_{q != j, local} ghat_iq   (T: all column
          blocks' estimated data, t: this rank's; Eq. g_rows_columns)
  u_j^i = (H_ij^* H_ij + rho I)^{-1}(H_ij^* gt_ij + rho (v_j - s_j^i))
  ghat_ij = H_ij u_j^i;  S_j = sum_i (u_j^i + s_j^i) over the local replicas
  v_j = S_kappa(S_j^total / M), s_j^i += u_j^i - v_j.
"""

import numpy as np
import torch

from oracle import admm_fp64 as A


class Fp64ShardEngine:
    def __init__(self, H, g, layout, lam: float, rho: float):
        r0, r1 = layout.rows
        c0, c1 = layout.cols
        self.H = np.ascontiguousarray(np.asarray(H, dtype=np.complex128)[r0:r1, c0:c1])
        self.g0 = np.asarray(g, dtype=np.complex128)[r0:r1].copy()
        self.geff = self.g0.copy()
        self.lay = layout
        self.lam, self.rho = float(lam), float(rho)
        m, n = self.H.shape
        self.rows = A.balanced_blocks(m, layout.M_loc)
        self.cols = A.balanced_blocks(n, layout.N_loc)
        self.solvers = [[A.BlockSolver(self.H[a:b, c:d], rho) for c, d in self.cols] for a, b in self.rows]
        self.v = np.zeros(n, np.complex128)
        self.s = np.zeros((layout.M_loc, n), np.complex128)
        self.u = np.zeros((layout.M_loc, n), np.complex128)
        self.ghat = np.zeros((layout.N_loc, m), np.complex128)
        self.t_loc = np.zeros(m, np.complex128)

    def ghat_sum(self):
        self.t_loc = self.ghat.sum(axis=0)
        return torch.from_numpy(self.t_loc.copy())

    def set_exchange(self, t) -> None:
        self.geff = self.g0 - t.numpy() + self.t_loc

    def ustep(self):
        new_ghat = np.zeros_like(self.ghat)
        for i, (a, b) in enumerate(self.rows):
            for j, (c, d) in enumerate(self.cols):
                gt = self.geff[a:b].copy()
                for q in range(len(self.cols)):
                    if q != j:
                        gt = gt - self.ghat[q, a:b]
                sv = self.solvers[i][j]
                rhs = A.adjoint(sv.H, gt) + self.rho * (self.v[c:d] - self.s[i, c:d])
                self.u[i, c:d] = sv.solve(rhs)
                new_ghat[j, a:b] = sv.H @ self.u[i, c:d]
        self.ghat = new_ghat
        return torch.from_numpy((self.u + self.s).sum(axis=0))

    def vstep(self, S) -> np.ndarray:
        M = self.lay.M
        v_new = A.soft_threshold(S.numpy() / M, self.lam / (M * self.rho))
        self.s = self.s + self.u - v_new[None, :]
        rec = np.array([float(np.sum(np.abs(self.u - v_new[None, :]) ** 2)),
                        float(np.sum(np.abs(v_new - self.v) ** 2)),
                        float(np.sum(np.abs(self.u) ** 2)),
                        float(np.sum(np.abs(v_new) ** 2)),
                        float(np.sum(np.abs(self.s) ** 2))])
        self.v = v_new
        return rec
