"""One iteration-kernel case to profile: a Gaussian m x n problem (device
generator, CN(0, 1/m), m/20 nonzeros, 30 dB, seed 3), split M x N, complex64
or FP16 H; `warmup` single-iteration launches, then one launch of `iters`
iterations timed with CUDA events.

    python -m paper_1811_05571_gb300.profile_case --m 1024 --n 131072 --M 16 --iters 2 [--fp16]
    python -m paper_1811_05571_gb300.profile_case --m 32768 --n 2048 --M 8 --form direct [--factor-pass 1|2]

With the direct factor form (blocks with at least as many rows as columns)
an iteration is the factor pass (and, with several column blocks, the column
and row passes); `--factor-pass` picks the full factor rows (1) or the
lower-triangle tiles (2).

The launches of the iteration kernel are, in order: the warm-up launches, then
the timed one (so ``ncu -k regex:iterate_kernel -s <warmup> -c 1`` captures the
timed launch).
"""

from __future__ import annotations

import argparse
import json


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=1024)
    ap.add_argument("--n", type=int, default=131072)
    ap.add_argument("--M", type=int, default=16)
    ap.add_argument("--N", type=int, default=1)
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--fp16", action="store_true")
    ap.add_argument("--form", choices=("lemma", "direct"), default="lemma")
    ap.add_argument("--factor-pass", type=int, default=0)
    args = ap.parse_args(argv)

    import torch

    import synth
    from . import ADMM_OPT_DIR_FACTOR_PASS, Solver, load

    load()
    dev = torch.device("cuda:0")
    H, g, _, lam = synth.gaussian_problem_device(args.m, args.n, max(1, args.m // 20), 3, device=dev)
    rho = 1.0
    if args.N > 1:
        rho = float(args.N)   # column blocks of a CN(0,1/m) matrix: ||H_j||^2 is about (1 + sqrt(n_j/m))^2
        rho *= (1.0 + (args.n / args.N / args.m) ** 0.5) ** 2
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = Solver(H, g, args.M, args.N, lam, rho, stream=st, form=args.form)
        if args.factor_pass:
            s.set_option(ADMM_OPT_DIR_FACTOR_PASS, args.factor_pass)
    torch.cuda.synchronize()
    del H, g
    if args.fp16:
        s.use_fp16(True)
    for _ in range(args.warmup):
        s.iterate(1)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    s.iterate(args.iters)
    b.record(st)
    torch.cuda.synchronize()
    if s.status() != 0:
        raise RuntimeError("device status after the profiled launch")
    info = s.info()
    hb = info["h16_bytes"] if args.fp16 else info["h_bytes"]
    state = (3 * args.M + 3) * args.n * 8
    if args.form == "direct":   # no pass over H with one column block (H_i^H g_i cached and read)
        alg = (0 if args.N == 1 else 2 * hb) + info["factor_bytes"] + state + (args.M * args.n * 8 if args.N == 1 else 0)
    else:
        alg = 2 * hb + info["factor_bytes"] + state
    us = a.elapsed_time(b) / args.iters * 1e3
    print(json.dumps({"m": args.m, "n": args.n, "M": args.M, "N": args.N, "fp16": args.fp16, "form": args.form, "us_per_iter": us,
                      "alg_bytes_per_iter": alg, "gbs": alg / us / 1e3, "ctas": info["ctas"],
                      "stages": info["stages"], "rows_per_stage": info["rows_per_stage"]}))
    s.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
