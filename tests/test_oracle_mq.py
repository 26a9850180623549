"""Oracle pins: MQ basis, Helmholtz entries, assembly, manufactured solutions."""
import os

import numpy as np
import pytest

import pins
import workloads as w
from oracle import mq


def test_golden_mq_values(golden_dir):
    rows = np.loadtxt(os.path.join(golden_dir, "mq_values.txt"))
    for r, c, k, Phi, LPhi in rows:
        assert mq.phi(r, c) == pytest.approx(Phi, rel=1e-15, abs=0)
        assert mq.lphi(r, c, k) == pytest.approx(LPhi, rel=1e-14)


def test_diagonal_closed_form():
    rng = np.random.default_rng(0)
    for _ in range(100):
        c, k = rng.uniform(0.05, 1.0), rng.uniform(0, 20)
        assert mq.lphi(0.0, c, k) == pytest.approx(3.0 / c + k * k * c, rel=1e-15)


def test_lphi_matches_fd_laplacian():
    pins.pin_mq_laplacian(mq, np.random.default_rng(1))


@pytest.mark.parametrize("n,ni", [(30, 18), (25, 0), (25, 25), (1, 1), (7, 3)])
def test_assembly_rows_apply_pde_and_bc(n, ni):
    rng = np.random.default_rng(n + ni)
    X = rng.uniform(0, 1, (n, 3))
    pins.pin_assembly_rows(mq, X, ni, 0.3, 4.0, rng)


def test_assembly_brute_force_loops():
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (12, 3))
    c, k, ni = 0.4, 3.0, 7
    A = mq.assemble(X, ni, c, k)
    for i in range(12):
        for j in range(12):
            r = float(np.sqrt(sum((X[i, t] - X[j, t]) ** 2 for t in range(3))))
            s = r * r + c * c
            ref = (2 * r * r + 3 * c * c) / s ** 1.5 + k * k * s ** 0.5 if i < ni else s ** 0.5
            assert A[i, j] == pytest.approx(ref, rel=1e-14)


def test_block_symmetry():
    rng = np.random.default_rng(4)
    X = rng.uniform(0, 1, (40, 3))
    ni = 25
    A = mq.assemble(X, ni, 0.2, 5.0)
    assert np.allclose(A[:ni, :ni], A[:ni, :ni].T, rtol=1e-15, atol=0)
    assert np.allclose(A[ni:, ni:], A[ni:, ni:].T, rtol=1e-15, atol=0)
    assert not np.allclose(A[:ni, ni:], A[ni:, :ni].T)


def test_eps_form_is_scaled_c_form():
    rng = np.random.default_rng(5)
    X = rng.uniform(0, 1, (20, 3))
    c = 0.25
    Ac = mq.assemble(X, 12, c, 2.0)
    Ae = mq.assemble(X, 12, c, 2.0, form="eps")
    # phi(r; eps) = sqrt(1 + eps^2 r^2) with eps = 1/c  (eq. MQ)
    D = mq.distances(X, X)
    assert np.allclose(Ae[12:], np.sqrt(1 + (D[12:] / c) ** 2), rtol=1e-15)
    assert np.allclose(Ae, Ac / c, rtol=1e-15)


def test_plane_wave_solves_helmholtz():
    rng = np.random.default_rng(6)
    P = rng.uniform(0, 1, (50, 3))
    for k in (2.0, 5.0, 10.0):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        lap = pins.fd_laplacian(lambda Q: w.plane_wave(Q, k, d), P, 1e-2)
        res = lap + k * k * w.plane_wave(P, k, d)
        assert np.max(np.abs(res)) < 1e-7 * k * k


def test_gaussian_source_matches_fd():
    rng = np.random.default_rng(7)
    P = rng.uniform(-1, 1, (50, 3))
    for sigma, k, ctr in ((20.0, 3.0, (0, 0, 0)), (20.0, 3.0, (0.25, 0.25, 0)), (10.0, 3.0, (0, 0, 0))):
        lap = pins.fd_laplacian(lambda Q: w.gaussian(Q, sigma, ctr), P, 1e-2)
        ref = lap + k * k * w.gaussian(P, sigma, ctr)
        assert np.allclose(w.gaussian_source(P, sigma, k, ctr), ref, rtol=1e-8, atol=1e-10)
