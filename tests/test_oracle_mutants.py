"""Planted mistakes in the oracle must be caught by the pins.

Each case rewrites one line of ``oracle/admm_fp64.py`` in memory (a dropped
term, a wrong sign, a wrong index, a transposed operand, a changed update
order), loads the rewritten module, points the pin tests at it and checks
that the named pin now fails.  Everything runs on the CPU.
"""

import importlib.util
import os
import sys
import types

import pytest

import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "admm_fp64.py")


def _mutant(old: str, new: str, count: int = 1) -> types.ModuleType:
    text = open(SRC).read()
    assert text.count(old) >= 1, f"mutation anchor not found: {old!r}"
    text = text.replace(old, new, count)
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = SRC
    sys.modules["oracle_mutant"] = mod
    exec(compile(text, SRC, "exec"), mod.__dict__)
    return mod


MUTANTS = [
    # (id, old, new, pin to run, pin kwargs)
    ("consensus_kappa_drops_M", "kappa = lam / (M * rho)\n    hist, a, stopped",
     "kappa = lam / rho\n    hist, a, stopped",
     pins.test_one_iteration_matches_least_squares_step, dict(M=2, N=1, k=0, mn=(20, 48))),
    ("consensus_dual_sign", "s = s + u - v_new\n        rp2 = sum(_sq(u[i]",
     "s = s - u + v_new\n        rp2 = sum(_sq(u[i]",
     pins.test_one_iteration_matches_least_squares_step, dict(M=2, N=1, k=1, mn=(20, 48))),
    ("lemma_transpose_without_conjugate", "adjoint(self.H, t)", "(self.H.T @ t)",
     pins.test_block_solver_matches_dense_solve, dict(rows=8, cols=64, rho=1.0)),
    ("lemma_rho_power", "/ (self.rho * self.rho)", "/ self.rho",
     pins.test_block_solver_matches_dense_solve, dict(rows=30, cols=200, rho=0.05)),
    ("direct_branch_missing_conjugate", "big = self.H.conj().T @ self.H", "big = self.H.T @ self.H",
     pins.test_block_solver_matches_dense_solve, dict(rows=40, cols=16, rho=0.5)),
    ("direct_branch_drops_rho", "big = self.H.conj().T @ self.H + self.rho * np.eye(cols",
     "big = self.H.conj().T @ self.H + np.eye(cols",
     pins.test_one_iteration_matches_least_squares_step, dict(M=2, N=1, k=1, mn=(60, 12))),
    ("sectioning_wrong_exclusion", "if q != j:\n                    gj = gj - ghat[q]",
     "if q == j:\n                    gj = gj - ghat[q]",
     pins.test_one_iteration_matches_least_squares_step, dict(M=1, N=3, k=1, mn=(20, 48))),
    ("sectioning_gauss_seidel_order", "gj = gj - ghat[q]",
     "gj = gj - solvers[q].H @ (u_new[q] if q < j else u[q])",
     pins.test_one_iteration_matches_least_squares_step, dict(M=1, N=3, k=1, mn=(20, 48))),
    ("cs_wrong_replica_index", "gij = gij - ghat[i][q]", "gij = gij - ghat[0][q]",
     pins.test_one_iteration_matches_least_squares_step, dict(M=3, N=2, k=1, mn=(20, 48))),
    ("consensus_rd_drops_M", "rd2 = rho * rho * M * _sq(v_new - v)", "rd2 = rho * rho * _sq(v_new - v)",
     pins.test_one_iteration_matches_least_squares_step, dict(M=2, N=1, k=1, mn=(20, 48))),
    ("consensus_sum_not_mean", "a = u.mean(axis=0) + s.mean(axis=0)",
     "a = u.sum(axis=0) + s.mean(axis=0)",
     pins.test_one_iteration_matches_least_squares_step, dict(M=2, N=1, k=1, mn=(20, 48))),
    ("threshold_tie_kept", "keep = mag > kappa", "keep = mag >= kappa",
     pins.test_soft_threshold_golden_values, dict()),
    ("threshold_real_sign", "out[keep] = a[keep] - kappa * (a[keep] / mag[keep])",
     "out[keep] = a[keep] - kappa * np.sign(a[keep].real)",
     pins.test_soft_threshold_golden_values, dict()),
    ("cs_kappa_drops_M", "kappa = lam / (M * rho)\n    hist, a_parts, stopped",
     "kappa = lam / rho\n    hist, a_parts, stopped",
     pins.test_every_split_converges_to_the_lasso_minimiser, dict(M=3, N=2)),
    # the stopping rule (Boyd et al. Section 3.3.1)
    ("stop_dual_tolerance_drops_rho",
     "eps_dual = np.sqrt(p) * eps_abs + eps_rel * rho * np.sqrt(rec[4])",
     "eps_dual = np.sqrt(p) * eps_abs + eps_rel * np.sqrt(rec[4])",
     pins.test_stop_rule_hand_worked_records, dict()),
    ("stop_primal_tolerance_ignores_u",
     "eps_rel * max(np.sqrt(rec[2]), np.sqrt(rec[3]))", "eps_rel * np.sqrt(rec[3])",
     pins.test_stop_rule_hand_worked_records, dict()),
    ("consensus_stop_length_is_n", "stop_test(np.array(hist[-1]), M * n, rho, *eps)",
     "stop_test(np.array(hist[-1]), n, rho, *eps)",
     pins.test_stopping_iteration_follows_boyd, dict(M=4, N=1)),
    ("consensus_v_norm_not_stacked", "M * _sq(v_new),\n", "_sq(v_new),\n",
     pins.test_recorded_norms_follow_the_stacked_definitions, dict(M=3, N=1, k=4)),
    ("cs_dual_record_drops_M", "rd2 = rho * rho * M * sum(_sq(v_new[j] - v[j]) for j in range(N))",
     "rd2 = rho * rho * sum(_sq(v_new[j] - v[j]) for j in range(N))",
     pins.test_recorded_norms_follow_the_stacked_definitions, dict(M=2, N=2, k=4)),
]


@pytest.mark.parametrize("mid,old,new,pin,kw", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(monkeypatch, mid, old, new, pin, kw):
    mod = _mutant(old, new)
    monkeypatch.setattr(pins, "A", mod)
    monkeypatch.setattr(pins, "oracle", mod)
    with pytest.raises(Exception):
        pin(**kw)


def test_unmutated_oracle_passes_the_same_pins(monkeypatch):
    mod = _mutant("def soft_threshold(", "def soft_threshold(")
    monkeypatch.setattr(pins, "A", mod)
    monkeypatch.setattr(pins, "oracle", mod)
    seen = set()
    for _, _, _, pin, kw in MUTANTS:
        key = (pin.__name__, tuple(sorted(kw.items())))
        if key in seen:
            continue
        seen.add(key)
        pin(**kw)
