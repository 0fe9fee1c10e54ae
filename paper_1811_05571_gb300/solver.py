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
        self.lam = list(lam)
        self.rho = float(rho)

    def set_lambda(self, lam) -> None:
        """New per-scene weights (no refactorisation)."""
        lam = [float(x) for x in lam]
        if len(lam) != self.batch:
            raise ValueError("one lambda per scene")
        B.admm_batch_set_lambda(self.h, lam)
        self.lam = lam

    def set_rho(self, rho: float) -> None:
        """New augmented parameter (refactors every block)."""
        B.admm_batch_set_rho(self.h, float(rho), self.stream)
        self.rho = float(rho)

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


def _push_params(solver, lam_v, rho_v) -> None:
    """Bring a solver's lambda (list, one per scene) and rho to the given values."""
    if isinstance(solver, BatchSolver):
        if lam_v != solver.lam:
            solver.set_lambda(lam_v)
        if rho_v != solver.rho:
            solver.set_rho(rho_v)
        return
    info = solver.info()
    if lam_v[0] != info["lambda"]:
        solver.set_lambda(lam_v[0])
    if rho_v != info["rho"]:
        solver.set_rho(rho_v)


def _unrolled_function():
    import torch

    class _Unrolled(torch.autograd.Function):
        """V = ADMM_K(G; lambda, rho) per scene from the zero state.  The forward
        runs K recorded iterations, the backward the library's reverse sweep
        (admm_batch_backward on a BatchSolver, admm_backward on each Solver of
        a list, one per scene)."""

        @staticmethod
        def forward(ctx, G, lam, rho, solver, iters):
            B = G.shape[0]
            lam_v = [float(x) for x in lam.detach().reshape(-1).cpu().tolist()]
            if len(lam_v) == 1:
                lam_v = lam_v * B
            if len(lam_v) != B:
                raise ValueError("lam must hold one value per scene or one shared value")
            rho_v = float(rho.detach().reshape(-1)[0].cpu())
            Gd = G.detach().to(torch.complex64).contiguous()
            if isinstance(solver, BatchSolver):
                _push_params(solver, lam_v, rho_v)
                solver.record(int(iters))
                solver.set_g(Gd)
                solver.iterate(int(iters))
                V = solver.v()
            else:
                if len(solver) != B:
                    raise ValueError("one Solver per scene")
                V = torch.empty((B, solver[0].n), dtype=torch.complex64, device=G.device)
                for b, sv in enumerate(solver):
                    _push_params(sv, [lam_v[b]], rho_v)
                    sv.set_g(Gd[b])
                    sv.record(int(iters))
                    sv.iterate(int(iters))
                    sv.v(out=V[b])
            ctx.solver = solver
            ctx.lam_shape, ctx.lam_dtype, ctx.lam_device = lam.shape, lam.dtype, lam.device
            ctx.rho_shape, ctx.rho_dtype, ctx.rho_device = rho.shape, rho.dtype, rho.device
            return V

        @staticmethod
        def backward(ctx, dV):
            dVc = dV.to(torch.complex64).contiguous()
            if isinstance(ctx.solver, BatchSolver):
                dG, dl, dr = ctx.solver.backward(dVc)
                dl, dr = [float(x) for x in dl], [float(x) for x in dr]
            else:
                dG = torch.empty((len(ctx.solver), ctx.solver[0].m), dtype=torch.complex64, device=dV.device)
                dl, dr = [], []
                for b, sv in enumerate(ctx.solver):
                    gg, gl, gr = sv.backward(dVc[b])
                    dG[b].copy_(gg)
                    dl.append(float(gl))
                    dr.append(float(gr))
            dl_t = torch.tensor(dl, dtype=ctx.lam_dtype)
            if dl_t.numel() != torch.Size(ctx.lam_shape).numel():
                dl_t = dl_t.sum()            # one lambda shared by every scene
            dr_t = torch.tensor(sum(dr), dtype=ctx.rho_dtype)   # rho is shared
            return (dG, dl_t.reshape(ctx.lam_shape).to(ctx.lam_device),
                    dr_t.reshape(ctx.rho_shape).to(ctx.rho_device), None, None)

    return _Unrolled


class UnrolledADMM:
    """``UnrolledADMM.apply(G, lam, rho, solver, iters)``: the images after
    `iters` iterations from the zero state (batch x n complex64) as a
    differentiable function of the measurements G (batch x m complex), the
    regularisation weights `lam` (real tensor, one per scene or one shared)
    and the augmented parameter `rho` (real scalar tensor), so that
    loss.backward() fills G.grad, lam.grad and rho.grad.  `solver` is a
    BatchSolver (all scenes together on the FP16-encoded H) or a list of
    Solver handles, one per scene (complex64 or FP16 H).  New lam or rho values
    are pushed to the solver(s) first (rho refactors)."""

    _fn = None

    @classmethod
    def apply(cls, G, lam, rho, solver, iters):
        if cls._fn is None:
            cls._fn = _unrolled_function()
        return cls._fn.apply(G, lam, rho, solver, iters)


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
        return {"waves": waves, "ctas": ctas, "launches": B.admm_group_launches(self.g),
                "graph": B.admm_group_uses_graph(self.g)}

    def close(self) -> None:
        if getattr(self, "g", None):
            B.admm_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

