#!/usr/bin/env python3
"""Write the FP64 oracle solution v* of the time-to-tolerance workload.

Workload: H 2048 x 16384 i.i.d. CN(0, 1/2048), 128 planted unit-magnitude
nonzeros, 30 dB, seed 5 (synth.gaussian_problem draw order), lambda = 0.05
max|H^H g|, rho = 1, consensus over 8 row blocks of 256 rows.  The oracle
runs 800 iterations; its primal and dual residuals are then at rounding
level.  The file lists the nonzeros of v* (index, real, imaginary part in
17 significant digits) after a header with the workload, lambda, rho, the
iteration count and the final residuals.

Only oracle/ computes here (synth only creates the inputs).

    python tests/golden/make_vstar.py
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

M_ROWS, N_COLS, NNZ, SEED, BLOCKS, ITERS = 2048, 16384, 128, 5, 8, 800
OUT = os.path.join(HERE, "vstar_gaussian_2048x16384_c8.txt")


def main() -> int:
    p = synth.gaussian_problem(M_ROWS, N_COLS, NNZ, seed=SEED)
    ref = oracle.run_split(p.H, p.g, BLOCKS, 1, p.lam, p.rho, ITERS)
    rp, rd = np.sqrt(ref.hist[-1, 0]), np.sqrt(ref.hist[-1, 1])
    nz = np.flatnonzero(ref.v)
    with open(OUT, "w") as f:
        f.write("# FP64 oracle solution v* of the time-to-tolerance workload (oracle.run_split)\n")
        f.write(f"# gaussian_problem(m={M_ROWS}, n={N_COLS}, nnz={NNZ}, seed={SEED}); consensus, "
                f"{BLOCKS} row blocks\n")
        f.write(f"# lambda {p.lam!r}\n# rho {p.rho!r}\n# iterations {ITERS}\n")
        f.write(f"# final ||r_p|| {float(rp)!r} ||r_d|| {float(rd)!r}\n")
        f.write(f"# norm {float(np.linalg.norm(ref.v))!r}\n# nonzeros {nz.size}\n")
        f.write("# columns: index real imag\n")
        for k in nz:
            f.write(f"{k} {ref.v[k].real:.17g} {ref.v[k].imag:.17g}\n")
    print(OUT, nz.size, "nonzeros; residuals", rp, rd)
    return 0


if __name__ == "__main__":
    sys.exit(main())
