"""``Solver``: an owning wrapper around one libadmm handle.

PyTorch supplies device memory and streams; every computation is a call into
libadmm.so.  Inputs may be torch tensors (CPU or CUDA) or numpy arrays of
complex64 / complex128; outputs are CUDA complex64 tensors unless a
destination buffer is passed.
"""

from __future__ import annotations

import numpy as np

from . import _binding as B


def _dtype_code(x) -> int:
    name = str(getattr(x, "dtype", ""))
    if "complex64" in name:
        return B.ADMM_C64
    if "complex128" in name:
        return B.ADMM_C128
    raise TypeError(f"H and g must be complex64 or complex128, got {name}")


def _contig(x):
    if hasattr(x, "is_contiguous"):
        return x if x.is_contiguous() else x.contiguous()
    return np.ascontiguousarray(x)


class Solver:
    """Norm-1 ADMM for g = Hu + w split into row_blocks x col_blocks (Sections III-A..C).

    form: "lemma" (m_b x m_b factors, every block shape), "direct" (n_b x n_b
    factors of H_b^H H_b + rho I, Section III-B) or "auto" (direct when every
    block has at least as many rows as columns)."""

    def __init__(self, H, g, row_blocks: int = 1, col_blocks: int = 1, lam: float = 0.0,
                 rho: float = 1.0, stream=None, form: str = "lemma"):
        import torch
        self._torch = torch
        H = _contig(H)
        g = _contig(g)
        m, n = int(H.shape[0]), int(H.shape[1])
        if int(g.shape[0]) != m:
            raise ValueError("g must have m entries")
        dt = _dtype_code(H)
        if _dtype_code(g) != dt:
            raise TypeError("H and g must share a dtype")
        self.m, self.n, self.M, self.N = m, n, int(row_blocks), int(col_blocks)
        self.stream = stream
        self._keep = (H, g)   # keep the sources alive until the synchronous setup returns
        codes = {"lemma": B.ADMM_FORM_LEMMA, "direct": B.ADMM_FORM_DIRECT, "auto": B.ADMM_FORM_AUTO}
        if form not in codes:
            raise ValueError("form must be 'lemma', 'direct' or 'auto'")
        self.h = B.admm_setup_form(H, g, m, n, self.M, self.N, float(lam), float(rho), dt, codes[form], stream)
        self._keep = None

    # -- iteration ---------------------------------------------------------
    def iterate(self, iters: int = 1) -> "Solver":
        B.admm_iterate(self.h, int(iters), self.stream)
        return self

    def solve(self, max_iter: int, eps_abs: float = 1e-6, eps_rel: float = 1e-4) -> int:
        return B.admm_solve(self.h, int(max_iter), float(eps_abs), float(eps_rel), self.stream)

    # -- results -----------------------------------------------------------
    def _order_after(self, out) -> None:
        # the copy ran on the handle's stream: later work on torch's current
        # stream (e.g. .cpu() of a device result) must wait for it
        st = self.stream
        if (st is not None and isinstance(st, self._torch.cuda.Stream)
                and isinstance(out, self._torch.Tensor) and out.is_cuda):
            self._torch.cuda.current_stream().wait_stream(st)

    def v(self, out=None):
        out = self._torch.empty(self.n, dtype=self._torch.complex64, device="cuda") if out is None else out
        B.admm_get_v(self.h, out, self.stream)
        self._order_after(out)
        return out

    def u(self, out=None):
        out = (self._torch.empty((self.M, self.n), dtype=self._torch.complex64, device="cuda")
               if out is None else out)
        B.admm_get_u(self.h, out, self.stream)
        self._order_after(out)
        return out

    def residuals(self, cap: int | None = None) -> np.ndarray:
        info = self.info()
        cap = int(info["iterations"]) if cap is None else int(cap)
        return B.admm_get_residuals(self.h, max(cap, 0), self.stream)

    def state(self):
        t = self._torch
        v = t.empty(self.n, dtype=t.complex64)
        s = t.empty((self.M, self.n), dtype=t.complex64)
        gh = t.empty((self.N, self.m), dtype=t.complex64)
        k = B.admm_get_state(self.h, v, s, gh, self.stream)
        return k, v, s, gh

    def set_state(self, k: int, v, s, ghat=None) -> None:
        B.admm_set_state(self.h, int(k), _contig(v), _contig(s),
                         None if ghat is None else _contig(ghat), self.stream)

    # -- parameters ----------------------------------------------------------
    def set_g(self, g) -> None:
        g = _contig(g)
        B.admm_set_g(self.h, g, _dtype_code(g), self.stream)

    def set_lambda(self, lam: float) -> None:
        B.admm_set_lambda(self.h, float(lam))

    def set_rho(self, rho: float) -> None:
        B.admm_set_rho(self.h, float(rho), self.stream)

    def reset(self) -> None:
        B.admm_reset(self.h, self.stream)

    def set_option(self, option: int, value: int) -> None:
        B.admm_set_option(self.h, int(option), int(value))

    def record(self, iters: int) -> None:
        """Record the next `iters` iterations for backward() (resets the state)."""
        B.admm_set_option(self.h, B.ADMM_OPT_RECORD_ITERS, int(iters))

    def backward(self, grad_v):
        """(grad_g, grad_lambda, grad_rho) of a loss of the current image, given dL/dv."""
        t = self._torch
        gg = t.empty(self.m, dtype=t.complex64, device="cuda")
        gl, gr = B.admm_backward(self.h, _contig(grad_v), gg, self.stream)
        return gg, gl, gr

    def tune(self) -> int:
        """Autotune the L2 keep size of the current mode; resets the state. Returns the bytes kept."""
        B.admm_tune(self.h, self.stream)
        return int(self.info()["l2_keep_bytes"])

    def use_fp16(self, on: bool = True) -> None:
        """Stream the FP16 copy of H (built on first use) or the complex64 H."""
        B.admm_set_option(self.h, B.ADMM_OPT_H_FP16, 1 if on else 0)

    def trace(self, cap: int):
        return B.admm_get_trace(self.h, int(cap), self.stream)

    def status(self) -> int:
        return B.admm_status(self.h, self.stream)

    def info(self) -> dict:
        return B.admm_get_info(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            B.admm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BatchSolver:
    """`batch` scenes sharing one H, iterated together on the tensor cores
    (include/admm.h, admm_batch_*).  G is batch x m, images batch x n."""

    def __init__(self, H, row_blocks: int, col_blocks: int, lam, rho: float, stream=None):
        import torch
        self._torch = torch
        H = _contig(H)
        self.m, self.n = int(H.shape[0]), int(H.shape[1])
        lam = [float(x) for x in lam]
        self.batch = len(lam)
        self.M, self.N = int(row_blocks), int(col_blocks)
        self.stream = stream
        self.h = B.admm_batch_setup(H, self.m, self.n, self.M, self.N, self.batch, lam, float(rho),
                                    _dtype_code(H), stream)

    def set_g(self, G) -> None:
        G = _contig(G)
        if _dtype_code(G) != B.ADMM_C64:
            raise TypeError("G must be complex64")
        B.admm_batch_set_g(self.h, G, self.stream)

    def iterate(self, iters: int = 1) -> "BatchSolver":
        B.admm_batch_iterate(self.h, int(iters), self.stream)
        return self

    def v(self, out=None):
        t = self._torch
        out = t.empty((self.batch, self.n), dtype=t.complex64, device="cuda") if out is None else out
        B.admm_batch_get_v(self.h, out, self.stream)
        if self.stream is not None and isinstance(out, t.Tensor) and out.is_cuda:
            t.cuda.current_stream().wait_stream(self.stream)
        return out

    def residuals(self) -> np.ndarray:
        return B.admm_batch_get_residuals(self.h, self.batch, self.stream)

    def reset(self) -> None:
        B.admm_batch_reset(self.h, self.stream)

    def forward(self, X):
        t = self._torch
        Y = t.empty((self.batch, self.m), dtype=t.complex64, device="cuda")
        B.admm_batch_forward(self.h, _contig(X), Y, self.stream)
        return Y

    def adjoint(self, Y):
        t = self._torch
        X = t.empty((self.batch, self.n), dtype=t.complex64, device="cuda")
        B.admm_batch_adjoint(self.h, _contig(Y), X, self.stream)
        return X

    def tune(self) -> int:
        """Pick the fastest K split of the forward product; returns it."""
        B.admm_batch_tune(self.h, self.stream)
        return int(self.info()["splits"])

    def record(self, iters: int) -> None:
        """Record the next `iters` iterations for backward() (resets the state)."""
        B.admm_batch_record(self.h, int(iters))

    def backward(self, dV):
        """(dG, dlambda, drho) of a loss of the current image, given dL/dv (per scene)."""
        t = self._torch
        dG = t.empty((self.batch, self.m), dtype=t.complex64, device="cuda")
        dl, dr = B.admm_batch_backward(self.h, self.batch, _contig(dV), dG, self.stream)
        return dG, dl, dr

    def status(self) -> int:
        return B.admm_batch_status(self.h, self.stream)

    def info(self) -> dict:
        return B.admm_batch_get_info(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            B.admm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _unrolled_function():
    import torch

    class _Unrolled(torch.autograd.Function):
        """v = ADMM_K(G) for every scene of a BatchSolver; backward runs the
        library's reverse sweep and leaves dL/dlambda and dL/drho per scene in
        ``solver.last_param_grads``."""

        @staticmethod
        def forward(ctx, G, solver, iters):
            solver.record(int(iters))
            solver.set_g(G.detach().to(torch.complex64).contiguous())
            solver.iterate(int(iters))
            ctx.solver = solver
            return solver.v()

        @staticmethod
        def backward(ctx, dV):
            dG, dl, dr = ctx.solver.backward(dV.to(torch.complex64).contiguous())
            ctx.solver.last_param_grads = (dl, dr)
            return dG, None, None

    return _Unrolled


class UnrolledADMM:
    """``UnrolledADMM.apply(G, solver, iters)``: the images after `iters`
    iterations from the zero state as a differentiable function of the
    measurements G (batch x m); see BatchSolver.record / backward."""

    _fn = None

    @classmethod
    def apply(cls, G, solver, iters):
        if cls._fn is None:
            cls._fn = _unrolled_function()
        return cls._fn.apply(G, solver, iters)


class Group:
    """Several Solver handles iterated together in one persistent launch per
    wave (include/admm.h, admm_group_*).  The solvers must outlive the group."""

    def __init__(self, solvers, stream=None):
        self.solvers = list(solvers)
        self.stream = stream
        self.g = B.admm_group_setup([s.h for s in self.solvers], stream)

    def iterate(self, iters: int = 1) -> "Group":
        B.admm_group_iterate(self.g, int(iters), self.stream)
        return self

    def info(self):
        waves, ctas = B.admm_group_info(self.g, len(self.solvers))
        return {"waves": waves, "ctas": ctas}

    def close(self) -> None:
        if getattr(self, "g", None):
            B.admm_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

