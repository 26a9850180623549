"""Planted mistakes in the oracle (CPU only) must be caught by the pins.

Each case monkeypatches one plausible slip into an oracle function -- a
dropped term, a wrong sign, a transposed operand, a wrong index -- and shows
that the corresponding pin fails.  This is evidence that the pins constrain
the oracle rather than restate it.
"""
import numpy as np
import pytest

import pins
from oracle import gkb as G
from oracle import mq
from oracle import regularize as R


def _problem():
    rng = np.random.default_rng(0)
    X = rng.uniform(0, 1, (60, 3))
    A = mq.assemble(X, 40, 0.25, 3.0)
    f = rng.normal(size=60)
    return A, f


def test_dropped_k2_term_caught(monkeypatch):
    monkeypatch.setattr(mq, "lphi", lambda r, c, k: mq.laplacian_phi(r, c))
    with pytest.raises(AssertionError):
        pins.pin_mq_laplacian(mq, np.random.default_rng(1))


def test_wrong_laplacian_coefficient_caught(monkeypatch):
    def bad(r, c):
        r = np.asarray(r, dtype=float)
        s = r * r + c * c
        return (2 * r * r + 2 * c * c) / s ** 1.5
    monkeypatch.setattr(mq, "laplacian_phi", bad)
    with pytest.raises(AssertionError):
        pins.pin_mq_laplacian(mq, np.random.default_rng(1))


def test_swapped_row_types_caught(monkeypatch):
    orig = mq.assemble

    def bad(X, ni, c, k, form="c"):
        A = orig(X, ni, c, k, form)
        R_ = mq.distances(X, X)
        A[:ni] = mq.phi(R_[:ni], c)
        return A
    monkeypatch.setattr(mq, "assemble", bad)
    rng = np.random.default_rng(2)
    with pytest.raises(AssertionError):
        pins.pin_assembly_rows(mq, rng.uniform(0, 1, (20, 3)), 12, 0.3, 3.0, rng)


def test_transposed_operand_in_gkb_caught():
    A, f = _problem()
    g = G.gkb(lambda x: A @ x, lambda y: A @ y, f, 20)  # A used where A^T belongs
    with pytest.raises(AssertionError):
        pins.pin_gkb_relations(A, f, g)


def test_missing_reorth_caught(monkeypatch):
    A, f = _problem()
    monkeypatch.setattr(G, "_reorth", lambda v, Q, scheme: v)
    g = G.gkb(A, None, f, 55)
    with pytest.raises(AssertionError):
        pins.pin_gkb_relations(A, f, g)


def test_ftil_from_column_instead_of_row_caught(monkeypatch):
    A, f = _problem()
    g = G.gkb(A, None, f, 20)

    def bad(C, beta1):
        U, s, Vt = np.linalg.svd(C, full_matrices=True)
        return R.ProjectedSVD(s, beta1 * U[:, 0], Vt.T, U, float(beta1))
    ps = bad(g.C(), g.beta1)
    with pytest.raises(AssertionError):
        pins.pin_projected_svd(ps, g.C(), g.beta1)


def test_gcv_denominator_off_by_one_caught(monkeypatch):
    A, f = _problem()
    g = G.gkb(A, None, f, 20)
    ps = R.projected_svd(g.C(), g.beta1)

    def bad(ps_, lam):
        rho2 = R.rho2_proj(ps_, lam)
        L = np.atleast_1d(lam)[0]
        tr = np.sum(ps_.sigma ** 2 / (ps_.sigma ** 2 + L * L))
        return np.array([rho2[0] / (ps_.l - tr) ** 2])
    lam = ps.sigma[0] * 1e-2
    with pytest.raises(AssertionError):
        assert bad(ps, lam)[0] == pytest.approx(pins.gcv_dense(g.C(), g.beta1, lam), rel=1e-9)
    assert R.gcv_proj(ps, lam)[0] == pytest.approx(pins.gcv_dense(g.C(), g.beta1, lam), rel=1e-9)


def test_missing_sigma_factor_in_hkt_caught():
    A, f = _problem()
    g = G.gkb(A, None, f, 20)
    ps = R.projected_svd(g.C(), g.beta1)
    lam = ps.sigma[0] * 1e-3
    bad = ps.V @ (ps.ftil[: ps.l] / (ps.sigma ** 2 + lam * lam))
    b = np.zeros(ps.l + 1)
    b[0] = g.beta1
    ref = pins.tikhonov_lstsq(g.C(), b, lam)
    assert np.linalg.norm(bad - ref) / np.linalg.norm(ref) > 1e-3
    assert np.linalg.norm(R.hkt_solve_proj(ps, lam) - ref) / np.linalg.norm(ref) < 1e-12


def _tsvd_full_mutant(denominator_shift=0, stop_at_r=False):
    """tsvd_full with one planted slip in its GCV rank curve."""
    def bad(A, f, rank=None, fs=None):
        fs = R.full_svd(A, f) if fs is None else fs
        f2 = fs.fhat[: fs.r] ** 2
        if rank is None:
            kmax = fs.r if stop_at_r else min(fs.r, fs.n - 1)
            with np.errstate(divide="ignore", invalid="ignore"):
                curve = np.array([(np.sum(f2[k:]) + fs.s_perp) / (fs.n - k + denominator_shift) ** 2
                                  for k in range(1, kmax + 1)])
            k = int(np.nanargmin(curve)) + 1
        else:
            k, curve = int(rank), None
        coef = fs.V[:, :k] @ (fs.fhat[:k] / fs.sigma[:k])
        return dict(coef=coef, rank=k, fs=fs, curve=curve)
    return bad


def test_tsvd_gcv_denominator_off_by_one_caught():
    with pytest.raises(AssertionError):
        pins.pin_tsvd_gcv_curve(_tsvd_full_mutant(denominator_shift=1), np.random.default_rng(14))


def test_tsvd_gcv_range_ending_at_r_caught():
    with pytest.raises(AssertionError):
        pins.pin_tsvd_gcv_curve(_tsvd_full_mutant(stop_at_r=True), np.random.default_rng(14))


def test_full_rank_threshold_without_n_caught(monkeypatch):
    orig = R.full_svd

    def bad(A, f):
        fs = orig(A, f)
        s = fs.sigma
        fs.r = int(np.sum(s > R.EPS * s[0]))  # planted: drops the factor N
        return fs
    with pytest.raises(AssertionError):
        pins.pin_full_rank(bad, np.random.default_rng(13))
