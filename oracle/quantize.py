"""FP16 storage of the sensing matrix, FP64 CPU restatement (TEST
INFRASTRUCTURE ONLY: imported by tests/ and bench.py's CPU legs, never by the
GPU library).

The mixed-precision variant of the iteration streams H in half precision
with one power-of-two scale per group of 64 consecutive rows.  The scale of a
group is 2^(q - 14), where the largest max(|Re|, |Im|) in the group equals
f 2^q with f in [0.5, 1); every entry is stored as the IEEE binary16 number
nearest to H / scale (ties to even).  Because the scale is a power of two the
division and the multiplication back are exact, so the matrix the storage
encodes is binary16(H / scale) * scale, exactly representable in FP32.

The paper runs FP32 throughout; this format is the project's own reading of
the precision row of the hot path (FP16 storage, FP32 arithmetic, then
complex64 polish iterations), and ADMM on the encoded matrix is exact ADMM
on a perturbed problem, so the oracle of the FP16 mode is the FP64 oracle run
on ``dequantized(H)``.
"""

from __future__ import annotations

import numpy as np

GROUP = 64


def group_scales(H: np.ndarray, group: int = GROUP) -> np.ndarray:
    """One scale per row group: 2^(q - 14) with max(|Re|,|Im|) = f 2^q, f in [0.5, 1).

    A group of zeros gets the scale 1.  H is taken as complex64 (the
    device copy), so the maxima are FP32 numbers."""
    H = np.asarray(H).astype(np.complex64)
    m = H.shape[0]
    out = np.empty((m + group - 1) // group, dtype=np.float64)
    for g in range(out.size):
        blk = H[g * group:(g + 1) * group]
        mx = float(max(np.abs(blk.real).max(initial=0.0), np.abs(blk.imag).max(initial=0.0)))
        if mx == 0.0:
            out[g] = 1.0
        else:
            _, q = np.frexp(mx)          # mx = f 2^q, f in [0.5, 1)
            out[g] = 2.0 ** (int(q) - 14)
    return out


def quantize(H: np.ndarray, group: int = GROUP) -> tuple[np.ndarray, np.ndarray]:
    """(H16, scales): H16[r, c] = binary16 nearest to H[r, c] / scale of row r's group."""
    Hc = np.asarray(H).astype(np.complex64)
    sc = group_scales(Hc, group)
    row_scale = np.repeat(sc, group)[: Hc.shape[0]][:, None]
    re = (Hc.real.astype(np.float64) / row_scale).astype(np.float16)
    im = (Hc.imag.astype(np.float64) / row_scale).astype(np.float16)
    return np.stack([re, im], axis=-1), sc


def dequantized(H: np.ndarray, group: int = GROUP) -> np.ndarray:
    """The matrix the FP16 storage encodes, binary16(H / scale) * scale, as complex128."""
    H16, sc = quantize(H, group)
    row_scale = np.repeat(sc, group)[: H16.shape[0]][:, None]
    return H16[..., 0].astype(np.float64) * row_scale + 1j * (H16[..., 1].astype(np.float64) * row_scale)
