"""Pins of the oracle's one-sided Jacobi SVD, operator scaling and TSVD.

* Singular values against LAPACK (numpy) and against matrices built with
  known singular values; U, V orthonormal and U diag(s) V^T = B.
* Brute force for n <= 6: roots of the characteristic polynomial of B^T B.
* The spectral identity of Prop. (coro:B-Lambda): the eigenvalues of
  Lambda^nu = diag(nu) A diag(sigma)^{-1} A^T diag(nu) are sigma_i(B)^2, with
  B = diag(nu) A diag(sigma)^{-1/2} (Eq. (Lambda_tilde_nu), (A_r_MC)).
* The r-TSVD solution of Eq. (u1r) against a pseudo-inverse built from
  numpy's SVD, and the Tikhonov filter.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_03686_gb300 import workloads as W


def _orth(rng, n):
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    return Q * np.sign(np.diag(R))[None, :]


@pytest.mark.parametrize("shape", [(40, 12), (12, 40), (33, 33), (200, 64), (1, 5), (5, 1)])
def test_jacobi_against_lapack(shape):
    rng = np.random.default_rng(sum(shape))
    B = rng.standard_normal(shape)
    U, s, V, sweeps, ok = O.jacobi_svd(B)
    assert ok and sweeps < 20
    ref = np.linalg.svd(B, compute_uv=False)
    np.testing.assert_allclose(s, ref, rtol=1e-13, atol=1e-14 * ref[0])
    k = min(shape)
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, B, atol=1e-13 * ref[0])
    assert np.all(np.diff(s) <= 0)
    # sign convention: largest-magnitude entry of every right vector > 0
    for c in range(k):
        assert V[np.argmax(np.abs(V[:, c])), c] > 0


def test_known_singular_values_graded():
    rng = np.random.default_rng(1)
    m, n = 60, 24
    sv = np.logspace(0, -12, n)
    B = _orth(rng, m)[:, :n] @ np.diag(sv) @ _orth(rng, n).T
    U, s, V, sweeps, ok = O.jacobi_svd(B)
    assert ok
    big = sv >= 1e-6
    np.testing.assert_allclose(s[big], sv[big], rtol=1e-10)
    np.testing.assert_allclose(s[~big], sv[~big], atol=1e-10 * sv[0])


def test_rank_deficient_and_zero():
    B = np.zeros((6, 4))
    B[:, 0] = 1.0
    B[:, 2] = 2.0
    U, s, V, sweeps, ok = O.jacobi_svd(B)
    np.testing.assert_allclose(s, [np.sqrt(6 * 5), 0, 0, 0], atol=1e-13)
    np.testing.assert_allclose(U[:, :1] * s[:1] @ V[:, :1].T, B, atol=1e-13)
    U, s, V, sweeps, ok = O.jacobi_svd(np.zeros((3, 3)))
    assert ok and np.all(s == 0)


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_brute_force_characteristic_polynomial(n):
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n + 3, n))
    G = B.T @ B
    # characteristic polynomial by the Faddeev-LeVerrier recursion
    c = [1.0]
    M = np.zeros_like(G)
    for k in range(1, n + 1):
        M = G @ M + c[-1] * np.eye(n)
        c.append(-np.trace(G @ M) / k)
    lam = np.sort(np.roots(c).real)[::-1]
    U, s, V, _, ok = O.jacobi_svd(B)
    np.testing.assert_allclose(s ** 2, lam, rtol=1e-9)


def test_spectral_identity_lambda_nu():
    inst = W.disc_config(N=4000)
    C, U0, _ = O.build_counts(inst)
    nu = inst.nu_vec()
    sig = O.element_measures(inst.domain, inst.partition)
    g1 = inst.partition.gamma1.astype(bool)
    B = O.operator_B(C, inst.N, g1, nu, sig)
    A1 = C[:, g1] / inst.N
    Lam = np.diag(nu) @ A1 @ np.diag(1 / sig[g1]) @ A1.T @ np.diag(nu)
    ev = np.sort(np.linalg.eigvalsh(Lam))[::-1]
    U, s, V, _, ok = O.jacobi_svd(B)
    k = len(s)
    np.testing.assert_allclose(s ** 2, ev[:k], rtol=1e-10, atol=1e-14 * ev[0])
    assert np.all(np.abs(ev[k:]) < 1e-14 * ev[0])
    # B by its definition, entry by entry
    i, j = 3, 5
    jj = np.flatnonzero(g1)[j]
    assert B[i, j] == pytest.approx(nu[i] * C[i, jj] / inst.N / np.sqrt(sig[jj]), rel=1e-15)


def test_tsvd_against_pseudo_inverse():
    inst = W.annulus_config(N=2000, grid=4, m_each=16)
    C, _, _ = O.build_counts(inst)
    nu = inst.nu_vec()
    sig = O.element_measures(inst.domain, inst.partition)
    g1 = inst.partition.gamma1.astype(bool)
    meas = W.measurements(inst, noise=0.01)
    B = O.operator_B(C, inst.N, g1, nu, sig)
    U, s, V, _, ok = O.jacobi_svd(B)
    A = C / inst.N
    b = meas.uD - A[:, ~g1] @ meas.u0
    Ur, sr, Vtr = np.linalg.svd(B, full_matrices=False)
    for r in (1, 3, 7, 12):
        u1, uhat = O.reconstruct(U, s, V, r, C, inst.N, g1, nu, sig, meas.uD, meas.u0)
        Bp = Vtr[:r].T @ np.diag(1 / sr[:r]) @ Ur[:, :r].T
        ref = (Bp @ (nu * b)) / np.sqrt(sig[g1])
        np.testing.assert_allclose(u1, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
        np.testing.assert_allclose(uhat, A[:, g1] @ ref + A[:, ~g1] @ meas.u0, atol=1e-10)
    # Tikhonov filter sigma / (sigma^2 + alpha) with all singular values
    alpha = 1e-4
    u1, _ = O.reconstruct(U, s, V, len(s), C, inst.N, g1, nu, sig, meas.uD, meas.u0,
                          tikhonov=alpha)
    ref = (Vtr.T @ np.diag(sr / (sr ** 2 + alpha)) @ Ur.T @ (nu * b)) / np.sqrt(sig[g1])
    np.testing.assert_allclose(u1, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


# ---------------------------------------------------------------------------
# The Tikhonov branch of the reconstruction, pinned by what the algebra of
# Tikhonov regularisation fixes (not by the filter formula it uses): the
# regularised least-squares problem min |B w - q|^2 + alpha |w|^2 has the
# unique solution w = (B^T B + alpha I)^{-1} B^T q (normal equations), whose
# limits are the pseudo-inverse solution (alpha -> 0) and B^T q / alpha
# (alpha -> infinity).  A filter 1 / (sigma + alpha), or alpha on the wrong
# side of the fraction, fails every one of these.
# ---------------------------------------------------------------------------
def test_tikhonov_hand_worked_diagonal():
    """B = diag(2, 1/2) (counts [[8, 0], [0, 2]] over N = 4 walks, nu = 1,
    sigma = 1, both elements on Gamma_1), u^D = (1, 1), alpha = 1/4:
    w_i = s_i / (s_i^2 + alpha) q_i gives w = (2 / 4.25, 0.5 / 0.5) =
    (8/17, 1) by hand, and the fitted data A w = (16/17, 1/2)."""
    C = np.array([[8, 0], [0, 2]], dtype=np.uint32)
    g1 = np.array([1, 1], np.uint8)
    nu = np.ones(2)
    sig = np.ones(2)
    U = np.eye(2)
    V = np.eye(2)
    s = np.array([2.0, 0.5])
    u1, uhat = O.reconstruct(U, s, V, 2, C, 4, g1, nu, sig, np.ones(2), None,
                             tikhonov=0.25)
    np.testing.assert_allclose(u1, [8.0 / 17.0, 1.0], rtol=1e-15)
    np.testing.assert_allclose(uhat, [16.0 / 17.0, 0.5], rtol=1e-15)


def _tikhonov_case():
    inst = W.annulus_config(N=2000, grid=4, m_each=16)
    C, _, _ = O.build_counts(inst)
    nu = inst.nu_vec()
    sig = O.element_measures(inst.domain, inst.partition)
    g1 = inst.partition.gamma1.astype(bool)
    meas = W.measurements(inst, noise=0.01)
    B = O.operator_B(C, inst.N, g1, nu, sig)
    U, s, V, _, ok = O.jacobi_svd(B)
    assert ok
    b = meas.uD - (C / inst.N)[:, ~g1] @ meas.u0
    return inst, C, nu, sig, g1, meas, B, U, s, V, nu * b


@pytest.mark.parametrize("alpha", [1e-8, 1e-5, 1e-2, 10.0])
def test_tikhonov_matches_normal_equations(alpha):
    """u_Gamma1 = diag(sigma)^{-1/2} (B^T B + alpha I)^{-1} B^T diag(nu) b, the
    solution of the regularised least-squares problem, for every alpha."""
    inst, C, nu, sig, g1, meas, B, U, s, V, q = _tikhonov_case()
    n = B.shape[1]
    w = np.linalg.solve(B.T @ B + alpha * np.eye(n), B.T @ q)
    ref = w / np.sqrt(sig[g1])
    u1, _ = O.reconstruct(U, s, V, len(s), C, inst.N, g1, nu, sig, meas.uD, meas.u0,
                          tikhonov=alpha)
    # the normal equations square the condition number: their own error is
    # eps kappa(B^T B + alpha I) relative
    kappa = (s[0] ** 2 + alpha) / (s[-1] ** 2 + alpha)
    tol = max(1e-12, 50 * np.finfo(float).eps * kappa)
    assert np.linalg.norm(u1 - ref) <= tol * np.linalg.norm(ref)


def test_tikhonov_limits():
    """alpha -> infinity: alpha u_Gamma1 -> diag(sigma)^{-1/2} B^T diag(nu) b
    (first order in 1 / alpha); alpha -> 0: the full-rank TSVD solution, which
    refits u^D exactly when M_D <= M_1 and B has full row rank."""
    inst, C, nu, sig, g1, meas, B, U, s, V, q = _tikhonov_case()
    lim = (B.T @ q) / np.sqrt(sig[g1])
    for alpha in (1e4, 1e6):
        u1, _ = O.reconstruct(U, s, V, len(s), C, inst.N, g1, nu, sig, meas.uD,
                              meas.u0, tikhonov=alpha)
        # alpha w = B^T q - B^T B B^T q / alpha + ...: relative gap <= s_1^2 / alpha
        assert np.linalg.norm(alpha * u1 - lim) <= 2 * s[0] ** 2 / alpha * np.linalg.norm(lim)
    # alpha -> 0 on a problem with M_D <= M_1 (fewer points than Gamma_1 cells)
    small = W.annulus_config(N=4000, grid=3, m_each=16)
    C2, _, _ = O.build_counts(small)
    nu2 = small.nu_vec()
    sig2 = O.element_measures(small.domain, small.partition)
    h1 = small.partition.gamma1.astype(bool)
    assert small.M_D <= int(h1.sum())
    meas2 = W.measurements(small, noise=0.01)
    U2, s2, V2, _, _ = O.jacobi_svd(O.operator_B(C2, small.N, h1, nu2, sig2))
    k = len(s2)
    t1, that = O.reconstruct(U2, s2, V2, k, C2, small.N, h1, nu2, sig2, meas2.uD,
                             meas2.u0, tikhonov=1e-14 * s2[-1] ** 2)
    p1, phat = O.reconstruct(U2, s2, V2, k, C2, small.N, h1, nu2, sig2, meas2.uD,
                             meas2.u0)
    np.testing.assert_allclose(t1, p1, rtol=1e-9, atol=1e-12 * np.abs(p1).max())
    np.testing.assert_allclose(phat, meas2.uD, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(that, meas2.uD, rtol=1e-9, atol=1e-12)
