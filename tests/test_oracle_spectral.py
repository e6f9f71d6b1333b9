"""Pins of the oracle's spectral diagnostics (Sec. 5.2 items (i)-(iv)):

* eigenvalues of Lambda^nu, computed by numpy's eigvalsh of the matrix the
  paper defines (Eq. (Lambda_tilde_nu)), equal the squared singular values of
  B from the C Jacobi SVD (Prop. coro:B-Lambda);
* the eigenfunction estimators (Eq. (eigenfunctions_MC)) equal
  diag(sigma)^{-1/2} v_j (from B^T u_j = s_j v_j) and are orthonormal in the
  sigma-weighted inner product;
* the TSVD family at full rank equals the pseudo-inverse solution from
  numpy's SVD, and with M_D <= M_1 its fitted interior data reproduce u^D
  exactly (B B^+ = I);
* the averaged density on the disc with K = I matches the mean of the
  closed-form Poisson-kernel arc measures over the poles, within the
  statistical band.
"""
import numpy as np
import pytest

from oracle import closed_forms as CF
from oracle import oracle as O
from paper_2409_03686_gb300 import workloads as W
from stats_util import beta_eps, check_band


def _operator(inst):
    C, _, _ = O.build_counts(inst)
    nu = inst.nu_vec()
    sig = O.element_measures(inst.domain, inst.partition)
    g1 = inst.partition.gamma1.astype(bool)
    B = O.operator_B(C, inst.N, g1, nu, sig)
    U, s, V, _, ok = O.jacobi_svd(B)
    assert ok
    return C, nu, sig, g1, U, s, V


@pytest.fixture(scope="module")
def annulus():
    inst = W.annulus_config(N=2000, grid=4, m_each=16)
    return inst, _operator(inst)


def test_eigenvalues_are_squared_singular_values(annulus):
    inst, (C, nu, sig, g1, U, s, V) = annulus
    out = O.spectral(U, s, V, C, inst.N, g1, nu, sig)
    big = out["lam"] >= 1e-12 * out["lam"][0]
    np.testing.assert_allclose(out["lam"][big], (s ** 2)[big], rtol=1e-9)
    assert np.all(np.abs(out["lam"] - s ** 2) <= 1e-14 * out["lam"][0])


def test_eigenfunctions_identity_and_orthonormality(annulus):
    inst, (C, nu, sig, g1, U, s, V) = annulus
    out = O.spectral(U, s, V, C, inst.N, g1, nu, sig)
    ef = out["eigfun"]
    ref = V / np.sqrt(sig[g1])[:, None]
    np.testing.assert_allclose(ef, ref, atol=1e-10 * np.abs(ref).max())
    G = ef.T @ (sig[g1][:, None] * ef)
    np.testing.assert_allclose(G, np.eye(len(s)), atol=1e-9)


def test_sweep_is_the_pseudo_inverse_and_refits_exactly(annulus):
    inst, (C, nu, sig, g1, U, s, V) = annulus
    meas = W.measurements(inst, noise=0.01)
    k = len(s)
    assert inst.M_D <= int(g1.sum())  # B has full row rank: B B^+ = I
    out = O.spectral(U, s, V, C, inst.N, g1, nu, sig, meas.uD, meas.u0, r_max=k)
    A = C / inst.N
    b = meas.uD - A[:, ~g1] @ meas.u0
    B = O.operator_B(C, inst.N, g1, nu, sig)
    ref = (np.linalg.pinv(B, rcond=1e-300) @ (nu * b)) / np.sqrt(sig[g1])
    u = out["u_sweep"][k - 1]
    assert np.linalg.norm(u - ref) <= 1e-6 * np.linalg.norm(ref)
    np.testing.assert_allclose(out["uD_sweep"][k - 1], meas.uD, atol=1e-8)
    # every r agrees with the TSVD reconstruction
    for r in (1, 2, 5, k):
        u1, uhat = O.reconstruct(U, s, V, r, C, inst.N, g1, nu, sig, meas.uD, meas.u0)
        np.testing.assert_allclose(out["u_sweep"][r - 1], u1, rtol=1e-12,
                                   atol=1e-12 * np.abs(u1).max())
        np.testing.assert_allclose(out["uD_sweep"][r - 1], uhat, atol=1e-12)


def test_averaged_density_on_the_disc_against_the_poisson_kernel():
    inst = W.disc_config(N=20_000)
    C, nu, sig, g1, U, s, V = _operator(inst)
    out = O.spectral(U, s, V, C, inst.N, g1, nu, sig)
    m = inst.partition.outer_m
    P = np.array([CF.disc_row(x, m, inst.partition.outer_theta0) for x in inst.points])
    want = P[:, g1].mean(axis=0)  # mean arc measure over the poles
    got = out["density"] * sig[g1]
    # the mean of M_D independent binomial proportions: N M_D walks per arc
    ok, info = check_band(got, want, inst.N * inst.M_D, beta=beta_eps(inst.eps, 1.0))
    assert ok, info
