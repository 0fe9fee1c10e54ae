"""The seeded generators: determinism, exact SNR, and the CRA phase model."""

import numpy as np

import synth
from synth import workloads as W


def test_gaussian_problem_is_deterministic_and_exact_snr():
    a = synth.gaussian_problem(64, 256, 5, seed=9, c64=False)
    b = synth.gaussian_problem(64, 256, 5, seed=9, c64=False)
    assert np.array_equal(a.H, b.H) and np.array_equal(a.g, b.g)
    clean = a.H @ a.u_true
    snr = np.linalg.norm(clean) / np.linalg.norm(a.g - clean)
    assert abs(snr - 10 ** 1.5) < 1e-9
    assert np.count_nonzero(a.u_true) == 5
    assert np.allclose(np.abs(a.u_true[a.u_true != 0]), 1.0)
    # CN(0, 1/m): E|H_ij|^2 = 1/m
    assert abs(np.mean(np.abs(a.H) ** 2) * 64 - 1.0) < 0.05
    lam = 0.05 * np.max(np.abs(a.H.conj().T @ a.g))
    assert abs(a.lam - lam) < 1e-15


def test_c64_representable_inputs_round_trip():
    p = synth.gaussian_problem(32, 128, 3, seed=1)
    assert np.array_equal(p.H_c64().astype(np.complex128), p.H)
    assert np.array_equal(p.g_c64().astype(np.complex128), p.g)


def test_cra_matrix_follows_phase_model():
    geom = dict(n_freq=3, rx_side=2, vox_side=4)
    H = synth.cra_matrix(seed=1, c64=False, **geom)
    freqs, rx, vox = W.cra_geometry(**geom)
    m, n = freqs.size * rx.shape[0], vox.shape[0]
    assert H.shape == (m, n)
    assert abs(np.vdot(H.ravel(), H.ravel()).real - n) < 1e-9
    phi = np.random.default_rng(1).uniform(0, 2 * np.pi, size=(m, 64))
    raw = np.empty((m, n), complex)
    for i in range(m):
        f, p = freqs[i // rx.shape[0]], rx[i % rx.shape[0]]
        for v in range(n):
            dt = np.linalg.norm(vox[v])
            dr = np.linalg.norm(vox[v] - p)
            raw[i, v] = np.exp(-2j * np.pi * f * (dt + dr) / W.SPEED_OF_LIGHT) / (dt * dr) \
                * np.exp(1j * phi[i, v % 64])
    scale = H[0, 0] / raw[0, 0]
    assert abs(scale.imag) < 1e-12 and scale.real > 0
    assert np.allclose(H, raw * scale.real, rtol=1e-12, atol=0)


def test_cra_geometry_recipe():
    freqs, rx, vox = W.cra_geometry()
    assert freqs.size == 40 and freqs[0] == 70e9 and freqs[-1] == 77e9
    assert rx.shape == (36, 3) and np.allclose(np.diff(np.unique(rx[:, 0])), 0.06)
    assert vox.shape == (32768, 3)
    assert np.allclose(vox.mean(axis=0), [0, 0, 0.5])
    assert np.allclose(vox[1] - vox[0], [0.005, 0, 0])      # x fastest
    assert np.allclose(vox[32] - vox[0], [0, 0.005, 0])
    assert np.allclose(vox[1024] - vox[0], [0, 0, 0.005])


def test_plate_scene_is_axis_aligned_plates():
    u = synth.plate_scene(seed=2).reshape(32, 32, 32)
    assert set(np.unique(u)) <= {0, 1}
    nz = np.count_nonzero(u)
    assert 100 <= nz <= 300
    assert np.array_equal(synth.plate_scene(seed=2), synth.plate_scene(seed=2))


def test_tall_workload_has_only_tall_blocks():
    """The overdetermined workload of the direct-form measurement: every block
    of every one of its splits has at least as many rows as columns, so the
    paper's rule picks the direct branch throughout."""
    from oracle import admm_fp64 as A
    c = synth.TALL
    assert c["m"] > c["n"]
    for M, N in c["splits"]:
        for r0, r1 in A.balanced_blocks(c["m"], M):
            for c0, c1 in A.balanced_blocks(c["n"], N):
                assert not A.lemma_applies(r1 - r0, c1 - c0), (M, N)
