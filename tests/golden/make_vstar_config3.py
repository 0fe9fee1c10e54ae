#!/usr/bin/env python3
"""Write the FP64 oracle solution v* of the 8192 x 131072 mixed-precision workload.

Workload (synth.chunked_gaussian_problem): H 8192 x 131072 i.i.d. CN(0, 1/8192)
drawn in row chunks of 64 (chunk c from default_rng([3, c])), 400 planted
unit-magnitude nonzeros of uniform phase, 30 dB, lambda = 0.05 max|H^H g|,
rho = 1, consensus over 16 row blocks of 512 rows.  The oracle runs until its
residuals meet the Boyd tolerances with eps_abs = 1e-14, eps_rel = 1e-12 (at
most 4000 iterations).  The file lists the nonzeros of v* (index, real and
imaginary part in 17 significant digits) after a header with the workload,
lambda, rho, the iteration count and the final residuals.

Only oracle/ computes here (synth only creates the inputs).  Needs about 27 GB
of host memory and, on 8 cores, about half an hour.

    python tests/golden/make_vstar_config3.py
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

C = synth.CONFIG3
EPS, MAX_ITERS = (1e-14, 1e-12), 4000
OUT = os.path.join(HERE, "vstar_gaussian_8192x131072_c16.txt")


def main() -> int:
    t0 = time.time()
    H, g, _, lam = synth.chunked_gaussian_problem(C["m"], C["n"], C["nnz"], C["seed"])
    H = H.astype(np.complex128)
    print(f"inputs ready in {time.time() - t0:.0f} s; lambda {lam!r}", flush=True)
    ref = oracle.run_split(H, g, C["row_blocks"], 1, lam, C["rho"], MAX_ITERS, eps=EPS)
    rp, rd = np.sqrt(ref.hist[-1, 0]), np.sqrt(ref.hist[-1, 1])
    nz = np.flatnonzero(ref.v)
    with open(OUT, "w") as f:
        f.write("# FP64 oracle solution v* of the mixed-precision workload (oracle.run_split)\n")
        f.write(f"# chunked_gaussian_problem(m={C['m']}, n={C['n']}, nnz={C['nnz']}, seed={C['seed']}); "
                f"consensus, {C['row_blocks']} row blocks\n")
        f.write(f"# lambda {lam!r}\n# rho {float(C['rho'])!r}\n# iterations {ref.iters}\n")
        f.write(f"# stopped {ref.stopped_at} eps_abs {EPS[0]!r} eps_rel {EPS[1]!r}\n")
        f.write(f"# final ||r_p|| {float(rp)!r} ||r_d|| {float(rd)!r}\n")
        f.write(f"# norm {float(np.linalg.norm(ref.v))!r}\n# nonzeros {nz.size}\n")
        f.write("# columns: index real imag\n")
        for k in nz:
            f.write(f"{k} {ref.v[k].real:.17g} {ref.v[k].imag:.17g}\n")
    print(OUT, nz.size, "nonzeros;", ref.iters, "iterations; residuals", rp, rd,
          f"; {time.time() - t0:.0f} s", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
