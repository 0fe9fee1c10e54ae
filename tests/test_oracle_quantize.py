"""Pins of the FP16 storage format of H (oracle/quantize.py) against facts
that do not come from the oracle: hand-computed values, the binary16 grid
enumerated from its bit patterns, the unit roundoff of binary16, and the
power-of-two property of the scales."""

import numpy as np
import pytest

from oracle import quantize as Q

# every finite binary16 number, from its 65536 bit patterns (not from a conversion)
_GRID = np.arange(1 << 16, dtype=np.uint16).view(np.float16).astype(np.float64)
_GRID_BITS = np.arange(1 << 16, dtype=np.uint16)
_FINITE = np.isfinite(_GRID)
_GRID, _GRID_BITS = _GRID[_FINITE], _GRID_BITS[_FINITE]
_ORDER = np.argsort(_GRID, kind="stable")
_SORTED, _SORTED_BITS = _GRID[_ORDER], _GRID_BITS[_ORDER]


def _nearest_fp16(x: float) -> float:
    """Brute-force nearest binary16 value, ties to the even significand."""
    i = np.searchsorted(_SORTED, x)
    cands = [k for k in (i - 1, i, i + 1) if 0 <= k < _SORTED.size]
    d = [abs(_SORTED[k] - x) for k in cands]
    best = min(d)
    ties = [cands[t] for t in range(len(cands)) if d[t] == best]
    if len(ties) > 1:
        ties = [k for k in ties if (int(_SORTED_BITS[k]) & 1) == 0] or ties
    return float(_SORTED[ties[0]])


def test_worked_example_one_third():
    # group maximum 1 = 0.5 * 2^1 -> scale 2^-13; (1/3) * 8192 = 2730.67, and
    # binary16 numbers in [2048, 4096) are spaced by 2 -> 2730 -> 2730 / 8192
    H = np.zeros((64, 4), dtype=np.complex128)
    H[0, 0] = 1.0
    H[5, 2] = np.float32(1.0 / 3.0)
    sc = Q.group_scales(H)
    assert sc.tolist() == [2.0 ** -13]
    D = Q.dequantized(H)
    assert D[0, 0] == 1.0
    assert D[5, 2] == 2730.0 / 8192.0


def test_scales_are_powers_of_two_and_fill_the_range():
    rng = np.random.default_rng(11)
    H = (rng.standard_normal((300, 40)) + 1j * rng.standard_normal((300, 40))) * 10.0 ** rng.uniform(-6, 3, (300, 1))
    sc = Q.group_scales(H)
    assert sc.size == 5
    for g, s in enumerate(sc):
        mant, _ = np.frexp(s)
        assert mant == 0.5                       # exact power of two
        blk = H[g * 64:(g + 1) * 64].astype(np.complex64)
        mx = max(np.abs(blk.real).max(), np.abs(blk.imag).max())
        assert 2.0 ** 13 <= mx / s < 2.0 ** 14   # largest entry lands in the top binade below 2^14


def test_zero_group_and_ragged_tail():
    H = np.zeros((130, 3), dtype=np.complex128)
    H[128:, :] = 3.0 - 2.0j
    sc = Q.group_scales(H)
    assert sc[0] == 1.0 and sc[1] == 1.0       # all-zero groups
    assert sc[2] == 2.0 ** (2 - 14)            # max 3 = 0.75 * 2^2
    D = Q.dequantized(H)
    assert np.array_equal(D, H)                # 3 and -2 are exact in binary16 after a power-of-two scale


def test_rounding_matches_brute_force_nearest():
    rng = np.random.default_rng(5)
    H = (rng.standard_normal((64, 24)) + 1j * rng.standard_normal((64, 24))) * 1e-3
    H[3, 3] = 0.0
    H[7, 1] = 1e-12 + 0j                         # far below the group maximum: binary16 subnormal / zero
    H16, sc = Q.quantize(H)
    Hc = H.astype(np.complex64)
    for r in range(64):
        for c in range(24):
            for part, got in ((Hc[r, c].real, H16[r, c, 0]), (Hc[r, c].imag, H16[r, c, 1])):
                x = float(part) / sc[0]
                assert float(got) == _nearest_fp16(x), (r, c, x)


def test_ties_round_to_even():
    # in [1024, 2048) binary16 numbers are spaced by 1; with scale 2^0 the group max
    # must lie in [2^13, 2^14): use 10000 = 0.61 * 2^14 -> scale 1
    H = np.zeros((64, 4), dtype=np.complex128)
    H[0, 0] = 10000.0
    H[1, 0] = 1024.5     # tie between 1024 (even) and 1025
    H[1, 1] = 1025.5     # tie between 1025 and 1026 (even)
    H[1, 2] = 8193.0     # spacing 8 above 8192: 8193 -> 8192
    assert Q.group_scales(H)[0] == 1.0
    D = Q.dequantized(H)
    assert D[1, 0] == 1024.0 and D[1, 1] == 1026.0 and D[1, 2] == 8192.0


def test_error_within_unit_roundoff():
    rng = np.random.default_rng(9)
    H = rng.standard_normal((192, 64)) + 1j * rng.standard_normal((192, 64))
    D = Q.dequantized(H)
    Hc = H.astype(np.complex64).astype(np.complex128)
    sc = np.repeat(Q.group_scales(H), 64)[:, None]
    u = 2.0 ** -11                               # unit roundoff of binary16
    sub = 2.0 ** -25 * sc                        # half the subnormal spacing, in H's units
    for part in (np.real, np.imag):
        err = np.abs(part(D) - part(Hc))
        assert np.all(err <= u * np.abs(part(Hc)) + sub)
    # and the relative Frobenius error is about u / sqrt(3) for Gaussian entries
    rel = np.linalg.norm(D - Hc) / np.linalg.norm(Hc)
    assert 1e-4 < rel < 2.0 ** -11


def test_exact_binary16_inputs_are_fixed_points():
    rng = np.random.default_rng(3)
    vals = rng.choice(_GRID[np.abs(_GRID) < 2.0 ** 14], size=(64, 16)).astype(np.float64)
    vals[0, 0] = 16000.0                         # pin the scale to 1
    H = vals * 2.0 ** -20 + 1j * vals[::-1] * 2.0 ** -20
    D = Q.dequantized(H)
    assert np.array_equal(D, H)


@pytest.mark.parametrize("bad", ["shift", "truncate"])
def test_planted_mistakes_fail_a_pin(bad, monkeypatch):
    """A scale off by one binade or truncation instead of rounding is caught."""
    if bad == "shift":
        orig = Q.group_scales
        monkeypatch.setattr(Q, "group_scales", lambda H, group=64: orig(H, group) * 2.0)
        with pytest.raises(AssertionError):
            test_scales_are_powers_of_two_and_fill_the_range()
    else:
        def trunc(H, group=64):
            Hc = np.asarray(H).astype(np.complex64)
            sc = Q.group_scales(Hc, group)
            rs = np.repeat(sc, group)[: Hc.shape[0]][:, None]
            parts = []
            for x in (Hc.real / rs, Hc.imag / rs):
                r = x.astype(np.float16)
                up = np.abs(r.astype(np.float64)) > np.abs(x)
                r[up] = np.nextafter(r[up], np.float16(0))   # round toward zero instead
                parts.append(r)
            return np.stack(parts, axis=-1), sc

        monkeypatch.setattr(Q, "quantize", trunc)
        with pytest.raises(AssertionError):
            test_rounding_matches_brute_force_nearest()
