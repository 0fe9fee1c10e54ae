"""Seeded problem generators for g = Hu + w (paper Eq. 2 and Eq. sensing_eq).

Every generator draws from ``numpy.random.default_rng(seed)`` (PCG64) in a
fixed order, so a (recipe, seed) pair names one instance on every machine.

Two workload families are produced:

* ``gaussian_problem`` -- H with i.i.d. CN(0, 1/m) entries, a sparse scene of
  unit-magnitude random-phase reflectors at uniform random indices, and
  complex Gaussian noise rescaled to an exact SNR.
* ``cra_problem`` -- a synthetic stand-in for the compressive-reflector-antenna
  sensing matrix of Section V (the paper's matrix comes from an EM solver that
  is not available): a stepped-frequency, multi-receiver near-field phase
  model whose columns are coded by one seeded random phase per (measurement,
  reflector facet), a scene of axis-aligned metallic plates, and 30 dB noise.

By default instances are *complex64-representable*: H and g are rounded to
complex64 before being returned (as complex128 arrays), so an FP32 GPU solver
and an FP64 CPU solver start from bit-identical inputs and differ only by the
arithmetic they perform.

The regularisation weight (a fraction of max|H^H g|, the smallest weight for
which the norm-1 solution is zero) and the augmented parameter rule for the
column splits are part of the workload recipe and live here too; they are
scalars handed to both solvers.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SPEED_OF_LIGHT = 299_792_458.0


@dataclass
class Problem:
    """One instance of the norm-1 regularised problem min 1/2||Hu-g||^2 + lam||u||_1."""

    H: np.ndarray          # complex128 (m, n), row-major
    g: np.ndarray          # complex128 (m,)
    u_true: np.ndarray     # complex128 (n,) -- the planted scene
    lam: float
    rho: float
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.H.shape[0])

    @property
    def n(self) -> int:
        return int(self.H.shape[1])

    def H_c64(self) -> np.ndarray:
        return np.ascontiguousarray(self.H.astype(np.complex64))

    def g_c64(self) -> np.ndarray:
        return np.ascontiguousarray(self.g.astype(np.complex64))


def round_to_c64(x: np.ndarray) -> np.ndarray:
    """Return x rounded to complex64 precision, stored as complex128."""
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def _complex_normal(rng: np.random.Generator, shape, var: float) -> np.ndarray:
    """CN(0, var): real and imaginary parts i.i.d. N(0, var/2)."""
    sd = np.sqrt(var / 2.0)
    return rng.standard_normal(shape) * sd + 1j * (rng.standard_normal(shape) * sd)


def noisy_measurements(H: np.ndarray, u: np.ndarray, rng: np.random.Generator,
                       snr_db: float) -> np.ndarray:
    """g = Hu + w with w ~ CN(0,1) rescaled so that ||Hu|| / ||w|| = 10^(snr/20) exactly."""
    clean = H @ u
    w = _complex_normal(rng, clean.shape, 1.0)
    target = np.linalg.norm(clean) / (10.0 ** (snr_db / 20.0))
    w *= target / np.linalg.norm(w)
    return clean + w


def lambda_from_fraction(H: np.ndarray, g: np.ndarray, frac: float) -> float:
    """lam = frac * max_k |(H^H g)_k|, computed in FP64.

    max|H^H g| is the smallest weight for which u = 0 solves the norm-1
    problem, so ``frac`` places lam on a scale-free axis."""
    return float(frac * np.max(np.abs(np.conj(H.T @ np.conj(g)))))


def spectral_norm_sq(A: np.ndarray, iters: int = 50, seed: int = 12345) -> float:
    """||A||_2^2 by ``iters`` power iterations on A^H A (FP64, seeded start)."""
    rng = np.random.default_rng(seed)
    x = _complex_normal(rng, (A.shape[1],), 1.0)
    x /= np.linalg.norm(x)
    est = 0.0
    for _ in range(iters):
        y = A @ x
        est = float(np.vdot(y, y).real)
        x = np.conj(A.T @ np.conj(y))
        nx = np.linalg.norm(x)
        if nx == 0.0:
            return 0.0
        x /= nx
    return est


def _balanced_bounds(total: int, parts: int) -> list[tuple[int, int]]:
    """Contiguous balanced split; the first (total mod parts) blocks get one extra."""
    base, extra = divmod(total, parts)
    out, start = [], 0
    for p in range(parts):
        size = base + (1 if p < extra else 0)
        out.append((start, start + size))
        start += size
    return out


def sectioning_rho(H: np.ndarray, col_blocks: int, iters: int = 50) -> float:
    """rho = N * max_j ||H_j||_2^2 over the column blocks H_j of an N-way column split.

    The estimated-data exchange of the column splits uses the other blocks'
    previous iterate; this proximal weight keeps that parallel update
    contractive."""
    best = 0.0
    for c0, c1 in _balanced_bounds(H.shape[1], col_blocks):
        best = max(best, spectral_norm_sq(np.ascontiguousarray(H[:, c0:c1]), iters))
    return col_blocks * best


# ----------------------------------------------------------------------------
# Gaussian family
# ----------------------------------------------------------------------------

def gaussian_problem(m: int, n: int, nnz: int, seed: int, snr_db: float = 30.0,
                     lam_frac: float = 0.05, rho: float = 1.0,
                     c64: bool = True, name: str = "") -> Problem:
    """H ~ CN(0, 1/m) i.i.d.; u has ``nnz`` unit-magnitude entries with uniform
    phase at distinct uniform indices; w at exactly ``snr_db``.

    Draw order from default_rng(seed): H, support, phases, w."""
    rng = np.random.default_rng(seed)
    H = _complex_normal(rng, (m, n), 1.0 / m)
    if c64:
        H = round_to_c64(H)
    support = rng.choice(n, size=nnz, replace=False)
    phases = rng.uniform(0.0, 2.0 * np.pi, size=nnz)
    u = np.zeros(n, dtype=np.complex128)
    u[support] = np.exp(1j * phases)
    g = noisy_measurements(H, u, rng, snr_db)
    if c64:
        g = round_to_c64(g)
    lam = lambda_from_fraction(H, g, lam_frac)
    return Problem(H=np.ascontiguousarray(H), g=g, u_true=u, lam=lam, rho=float(rho),
                   name=name or f"gaussian_{m}x{n}_s{seed}",
                   meta={"seed": seed, "nnz": nnz, "snr_db": snr_db, "lam_frac": lam_frac})


# ----------------------------------------------------------------------------
# Gaussian family drawn in independently seeded row chunks (large sizes)
# ----------------------------------------------------------------------------

ROWS_PER_DRAW = 64


def chunked_gaussian_rows(m: int, n: int, seed: int, chunk: int) -> np.ndarray:
    """Rows [64 c, min(64 c + 64, m)) of H ~ CN(0, 1/m), c = ``chunk``, drawn from
    default_rng([seed, c]) and rounded to complex64 (returned as complex64)."""
    rng = np.random.default_rng([seed, chunk])
    r0 = chunk * ROWS_PER_DRAW
    r1 = min(m, r0 + ROWS_PER_DRAW)
    return _complex_normal(rng, (r1 - r0, n), 1.0 / m).astype(np.complex64)


def chunked_gaussian_problem(m: int, n: int, nnz: int, seed: int, snr_db: float = 30.0,
                             lam_frac: float = 0.05, sink=None, threads: int | None = None,
                             lam: float | None = None):
    """The Gaussian recipe of ``gaussian_problem`` for matrices too large to draw
    from one generator in reasonable time: H ~ CN(0, 1/m) i.i.d. in row chunks of
    64, chunk c from default_rng([seed, c]) (so chunks can be drawn in parallel);
    the scene from default_rng([seed, 2**30]) in the order support, phases, w;
    g = Hu + w at exactly ``snr_db`` (FP64 from the complex64 H), rounded to
    complex64; lam = lam_frac * max|H^H g| in FP64 unless ``lam`` is given.

    ``sink(r0, rows)`` (optional) receives every chunk as it is drawn (from
    worker threads); otherwise H is kept and returned as one complex64 array.
    lam needs H, so it is computed only when H is kept.  Returns
    (H or None, g as complex128, u_true, lam or None)."""
    from concurrent.futures import ThreadPoolExecutor
    import os
    scene = np.random.default_rng([seed, 1 << 30])
    support = scene.choice(n, size=nnz, replace=False)
    phases = scene.uniform(0.0, 2.0 * np.pi, size=nnz)
    u = np.zeros(n, dtype=np.complex128)
    u[support] = np.exp(1j * phases)
    chunks = (m + ROWS_PER_DRAW - 1) // ROWS_PER_DRAW
    cols = np.empty((m, nnz), dtype=np.complex64)
    H = None if sink is not None else np.empty((m, n), dtype=np.complex64)

    def draw(c):
        rows = chunked_gaussian_rows(m, n, seed, c)
        r0 = c * ROWS_PER_DRAW
        cols[r0:r0 + rows.shape[0]] = rows[:, support]
        if sink is not None:
            sink(r0, rows)
        else:
            H[r0:r0 + rows.shape[0]] = rows

    workers = threads or min(16, os.cpu_count() or 1)
    with ThreadPoolExecutor(workers) as ex:
        list(ex.map(draw, range(chunks)))
    clean = cols.astype(np.complex128) @ u[support]
    w = _complex_normal(scene, (m,), 1.0)
    w *= (np.linalg.norm(clean) / (10.0 ** (snr_db / 20.0))) / np.linalg.norm(w)
    g = round_to_c64(clean + w)
    if lam is None and H is not None:
        def part(c):
            r0, r1 = c * ROWS_PER_DRAW, min(m, (c + 1) * ROWS_PER_DRAW)
            blk = H[r0:r1].astype(np.complex128)
            return np.conj(blk.T @ np.conj(g[r0:r1]))
        acc = np.zeros(n, dtype=np.complex128)
        with ThreadPoolExecutor(workers) as ex:
            for x in ex.map(part, range(chunks)):     # summed in chunk order
                acc += x
        lam = float(lam_frac * np.max(np.abs(acc)))
    return H, g, u, lam


# ----------------------------------------------------------------------------
# CRA-shaped family
# ----------------------------------------------------------------------------

def cra_geometry(n_freq: int = 40, f_lo: float = 70e9, f_hi: float = 77e9,
                 rx_side: int = 6, aperture: float = 0.3, vox_side: int = 32,
                 pitch: float = 0.005, z_centre: float = 0.5):
    """Frequencies, receiver positions and voxel centres of the CRA stand-in.

    Receivers: a rx_side x rx_side grid spanning ``aperture`` metres in the z=0
    plane, centred on the transmitter at the origin, x index fastest.
    Voxels: a vox_side^3 cube of ``pitch`` spacing centred at (0, 0, z_centre);
    flat voxel index v = ix + vox_side*iy + vox_side^2*iz.
    Measurement index i = f_idx * rx_side^2 + rx_idx."""
    freqs = np.linspace(f_lo, f_hi, n_freq)
    ax = np.linspace(-aperture / 2.0, aperture / 2.0, rx_side)
    ry, rx = np.meshgrid(ax, ax, indexing="ij")
    receivers = np.stack([rx.ravel(), ry.ravel(), np.zeros(rx.size)], axis=1)
    c = (np.arange(vox_side) - (vox_side - 1) / 2.0) * pitch
    iz, iy, ix = np.meshgrid(c, c, c, indexing="ij")
    voxels = np.stack([ix.ravel(), iy.ravel(), iz.ravel() + z_centre], axis=1)
    return freqs, receivers, voxels


def cra_matrix(seed: int = 1, n_facets: int = 64, c64: bool = True, **geom) -> np.ndarray:
    """H[i, v] = exp(-j 2 pi f_i (|t - r_v| + |r_v - p_i|)/c) / (|t - r_v| |r_v - p_i|)
                 * exp(j phi[i, v mod n_facets]),
    phi ~ U[0, 2 pi) drawn from default_rng(seed) with shape (m, n_facets);
    then H is scaled by one global constant so that ||H||_F^2 = n."""
    freqs, receivers, voxels = cra_geometry(**geom)
    n_rx = receivers.shape[0]
    m, n = freqs.size * n_rx, voxels.shape[0]
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=(m, n_facets))
    d_t = np.linalg.norm(voxels, axis=1)                                          # (n,)
    d_r = np.linalg.norm(voxels[None, :, :] - receivers[:, None, :], axis=2)      # (n_rx, n)
    path = d_t[None, :] + d_r
    amp = 1.0 / (d_t[None, :] * d_r)
    facet = np.arange(n) % n_facets
    H = np.empty((m, n), dtype=np.complex128)
    for f_idx, f in enumerate(freqs):
        rows = slice(f_idx * n_rx, (f_idx + 1) * n_rx)
        H[rows] = amp * np.exp(-2j * np.pi * f * path / SPEED_OF_LIGHT + 1j * phi[rows][:, facet])
    H *= np.sqrt(n / np.vdot(H.ravel(), H.ravel()).real)
    if c64:
        H = round_to_c64(H)
    return H


def plate_scene(seed: int = 2, vox_side: int = 32, n_plates: int = 3,
                side_lo: int = 6, side_hi: int = 10) -> np.ndarray:
    """Axis-aligned one-voxel-thick metallic plates (reflectivity 1).

    For each plate, in draw order: the normal axis (0=x, 1=y, 2=z), the two
    side lengths in [side_lo, side_hi], the plane index along the normal, and
    the two in-plane offsets so the plate lies fully inside the cube.
    Overlapping voxels count once."""
    rng = np.random.default_rng(seed)
    vol = np.zeros((vox_side, vox_side, vox_side), dtype=np.complex128)   # [iz, iy, ix]
    for _ in range(n_plates):
        axis = int(rng.integers(0, 3))
        a, b = (int(x) for x in rng.integers(side_lo, side_hi + 1, size=2))
        plane = int(rng.integers(0, vox_side))
        o1 = int(rng.integers(0, vox_side - a + 1))
        o2 = int(rng.integers(0, vox_side - b + 1))
        if axis == 0:      # normal along x: plate spans (y, z)
            vol[o2:o2 + b, o1:o1 + a, plane] = 1.0
        elif axis == 1:    # normal along y: plate spans (x, z)
            vol[o2:o2 + b, plane, o1:o1 + a] = 1.0
        else:              # normal along z: plate spans (x, y)
            vol[plane, o2:o2 + b, o1:o1 + a] = 1.0
    return vol.reshape(-1)


def cra_problem(H: np.ndarray | None = None, scene_seed: int = 2, noise_seed: int | None = None,
                snr_db: float = 30.0, lam_frac: float = 0.05, rho: float | None = None,
                rho_col_blocks: int = 8, c64: bool = True, name: str = "") -> Problem:
    """CRA-shaped imaging instance: H from ``cra_matrix`` (seed 1 unless given),
    a three-plate scene (``scene_seed``), and 30 dB noise drawn from
    default_rng([scene_seed, 1]) (or default_rng(noise_seed) when given).

    rho defaults to the column-split rule ``sectioning_rho(H, rho_col_blocks)``."""
    if H is None:
        H = cra_matrix(seed=1, c64=c64)
    u = plate_scene(seed=scene_seed)
    rng = np.random.default_rng([scene_seed, 1] if noise_seed is None else noise_seed)
    g = noisy_measurements(H, u, rng, snr_db)
    if c64:
        g = round_to_c64(g)
    lam = lambda_from_fraction(H, g, lam_frac)
    if rho is None:
        rho = sectioning_rho(H, rho_col_blocks)
    return Problem(H=H, g=g, u_true=u, lam=lam, rho=float(rho),
                   name=name or f"cra_{H.shape[0]}x{H.shape[1]}_scene{scene_seed}",
                   meta={"scene_seed": scene_seed, "snr_db": snr_db, "lam_frac": lam_frac,
                         "rho_rule": None if rho is None else "given"})


# Named recipes (sizes from the two single-matrix workloads the method is measured on).
CONFIG1 = dict(kind="gaussian", m=256, n=4096, nnz=16, seed=0, row_blocks=4, col_blocks=1,
               lam_frac=0.05, rho=1.0, iters=300)
CONFIG2 = dict(kind="cra", m=1440, n=32768, splits=((8, 1), (1, 8), (4, 4)),
               matrix_seed=1, scene_seed=2, lam_frac=0.05, rho_col_blocks=8, iters=300)
CONFIG3 = dict(kind="gaussian_chunked", m=8192, n=131072, nnz=400, seed=3, row_blocks=16,
               col_blocks=1, lam_frac=0.05, rho=1.0, fp16_iters=280, polish_iters=20)

# an overdetermined Gaussian problem whose blocks all have m_b >= n_b in the
# three splits (the direct factor form): 32768 x 2048 complex64 (537 MB, above L2)
TALL = dict(kind="gaussian_device", m=32768, n=2048, nnz=64, seed=7, lam_frac=0.05, rho=1.0,
            splits=((8, 1), (1, 8), (4, 4)))


def gaussian_problem_device(m: int, n: int, nnz: int, seed: int, snr_db: float = 30.0,
                            lam_frac: float = 0.05, device="cuda"):
    """Gaussian instance generated on the GPU (for sizes the host generator is
    too slow for): H ~ CN(0, 1/m) complex64, ``nnz`` unit-magnitude entries of
    uniform phase at distinct uniform indices, complex Gaussian noise scaled to
    exactly ``snr_db``, lambda = lam_frac * max|H^H g| (complex64 products).

    Draws come from one torch.Generator on ``device`` seeded with ``seed``, in
    the order H, support, phases, w.  Returns (H, g, u_true, lam) with the
    tensors on ``device``."""
    import torch
    gen = torch.Generator(device=device).manual_seed(int(seed))
    H = torch.view_as_complex(torch.randn(m, n, 2, generator=gen, device=device).mul_((0.5 / m) ** 0.5))
    u = torch.zeros(n, dtype=torch.complex64, device=device)
    idx = torch.randperm(n, generator=gen, device=device)[:nnz]
    phase = torch.rand(nnz, generator=gen, device=device) * (2.0 * np.pi)
    u[idx] = torch.polar(torch.ones_like(phase), phase)
    clean = H @ u
    w = torch.view_as_complex(torch.randn(m, 2, generator=gen, device=device).contiguous())
    w = w * (clean.norm() / w.norm() / 10.0 ** (snr_db / 20.0))
    g = clean + w
    lam = float(lam_frac * (H.conj().T @ g).abs().max())
    return H, g, u, lam


def shared_h_scenes(H: np.ndarray, count: int, seed0: int, kind: str = "sparse", nnz: int = 16,
                    snr_db: float = 30.0, lam_frac: float = 0.05):
    """``count`` scenes for one sensing matrix H (the batched workload): scene b
    draws from default_rng(seed0 + b) -- for kind "sparse" ``nnz`` unit-magnitude
    entries of uniform phase at distinct indices, for kind "plates" the
    three-plate scene ``plate_scene(seed0 + b)`` with noise from
    default_rng([seed0 + b, 1]) -- then w at exactly ``snr_db``.  Returns
    (G, U, lam): G count x m and U count x n complex128 (G rounded to complex64)
    and lam[b] = lam_frac * max|H^H g_b|."""
    H = np.asarray(H)
    m, n = H.shape
    G = np.empty((count, m), dtype=np.complex128)
    U = np.zeros((count, n), dtype=np.complex128)
    lam = []
    for b in range(count):
        if kind == "plates":
            U[b] = plate_scene(seed=seed0 + b)
            rng = np.random.default_rng([seed0 + b, 1])
        else:
            rng = np.random.default_rng(seed0 + b)
            support = rng.choice(n, size=nnz, replace=False)
            U[b, support] = np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, size=nnz))
        G[b] = round_to_c64(noisy_measurements(H, U[b], rng, snr_db))
        lam.append(lambda_from_fraction(H, G[b], lam_frac))
    return G, U, lam


def uneven_problem_sizes(count: int = 48, seed0: int = 1000):
    """Sizes of the uneven multi-problem workload: problem p draws, from
    default_rng(seed0 + p), m = round(exp U[ln 256, ln 4096]) and
    n = round(exp U[ln 4096, ln 32768]); nnz = max(1, round(m / 16)) and
    ceil(m / 256) row blocks.  Returns a list of (m, n, nnz, row_blocks, seed)."""
    out = []
    for p in range(count):
        rng = np.random.default_rng(seed0 + p)
        m = int(round(np.exp(rng.uniform(np.log(256), np.log(4096)))))
        n = int(round(np.exp(rng.uniform(np.log(4096), np.log(32768)))))
        out.append((m, n, max(1, int(round(m / 16))), int(np.ceil(m / 256)), seed0 + p))
    return out

