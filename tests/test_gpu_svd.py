"""Parity of the CUDA FP64 Jacobi SVD (wos_op_svd) and the TSVD
reconstruction (wos_reconstruct) with the oracle, on the same counts.

Singular values: |s - s_ref| <= 1e-10 s_ref for s_ref >= 1e-6 s_1, else
<= 1e-10 s_1 (two different FP64 Jacobi orders cannot agree relatively on
the tiny singular values of a severely ill-posed operator).  Singular
vectors are compared through the projector U_r U_r^T at spectral gaps (they
are defined only up to sign / rotation inside clusters).  Reconstructions
agree to 1e-8 relative in the 2-norm for r at a gap."""
import numpy as np
import pytest
import torch

from gpu_util import ctx
from oracle import oracle as O
from paper_2409_03686_gb300 import workloads as W
from paper_2409_03686_gb300 import wos

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(params=[wos.SVD_AUTO, wos.SVD_GRID], ids=["cluster", "grid"])
def svd_path(request):
    """Both factorisation kernels: the cluster kernel (taken by every problem
    here that fits it: at most 256 columns) and the grid-wide kernels."""
    wos.wos_set_svd_path(ctx(), request.param)
    yield request.param
    wos.wos_set_svd_path(ctx(), wos.SVD_AUTO)


def _svd_pair(C, N, gamma1, sigma, nu, sigma_lib=None):
    """The library's SVD (element measures sigma_lib, default sigma) and the
    oracle's (sigma) of the same counts."""
    Ct = torch.as_tensor(C.astype(np.int32), device=DEV)
    sg = torch.as_tensor(sigma if sigma_lib is None else sigma_lib, device=DEV)
    nut = torch.as_tensor(nu, device=DEV)
    U, S, V, sweeps = wos.wos_op_svd(ctx(), Ct, N, gamma1, sg, nu=nut)
    B = O.operator_B(C, N, gamma1, nu, sigma)
    Uo, so, Vo, sw_o, ok = O.jacobi_svd(B)
    return (U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy(), sweeps), (Uo, so, Vo), (Ct, sg, nut)


def _check_sv(s, so):
    big = so >= 1e-6 * so[0]
    assert np.all(np.abs(s - so)[big] <= 1e-10 * so[big]), np.max(np.abs(s - so)[big] / so[big])
    assert np.all(np.abs(s - so)[~big] <= 1e-10 * so[0])


def _gaps(so, max_r):
    return [r for r in range(1, min(max_r, len(so) - 1) + 1)
            if so[r] > 0 and so[r - 1] / so[r] >= 1.5 and so[r - 1] > 1e-6 * so[0]]


@pytest.mark.parametrize("make", [
    lambda: W.disc_config(N=4000, fp64=True),
    lambda: W.annulus_config(N=1000, grid=6, m_each=32),
    lambda: W.perforated_disc_config(N=1000, eps=1e-6, n_points=20, m_outer=20, m_hole=8),
])
def test_svd_matches_oracle_on_oracle_counts(make, svd_path):
    inst = make()
    C, _, _ = O.build_counts(inst)
    # each side takes the element measures from its own implementation
    sigma = O.element_measures(inst.domain, inst.partition)
    sigma_lib = wos.wos_element_measures(inst.domain, inst.partition)
    g1 = inst.partition.gamma1
    (U, s, V, sweeps), (Uo, so, Vo), _ = _svd_pair(C, inst.N, g1, sigma, inst.nu_vec(),
                                                   sigma_lib)
    _check_sv(s, so)
    k = len(so)
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-12)
    B = O.operator_B(C, inst.N, g1, inst.nu_vec(), sigma)
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, B, atol=1e-13 * so[0])
    for r in _gaps(so, 12):
        np.testing.assert_allclose(U[:, :r] @ U[:, :r].T, Uo[:, :r] @ Uo[:, :r].T, atol=1e-8)
    # spectral identity eig(Lambda^nu) = s^2 (Prop. coro:B-Lambda)
    ev = np.sort(np.linalg.eigvalsh(B @ B.T))[::-1][:k]
    np.testing.assert_allclose(s ** 2, ev, rtol=1e-9, atol=1e-14 * ev[0])


def _orth_tol(s):
    """Elementwise bound of |U^T U - I| for singular vectors recovered as
    W v / sigma (the grid-wide path above 256 columns, which does not
    accumulate V): the rounding error of column i is about eps |W| / s_i
    relative, so entry (i, j) may reach c eps s_1 / min(s_i, s_j), c = 64;
    plus 1e-12 for the norms, W v_j and sigma_j (from the preconditioned
    factor) agreeing to ~1e-12 relative."""
    eps = np.finfo(float).eps
    sm = np.minimum.outer(s, s)
    return 64 * eps * s[0] / np.maximum(sm, 1e-300) + 1e-12


@pytest.mark.parametrize("shape", [(256, 256, 128), (96, 300, 200), (1024, 1536, 768),
                                   (600, 900, 300), (300, 900, 600)])
def test_svd_matches_oracle_at_benchmark_shapes(shape, svd_path):
    """Operator-shaped counts at the benchmark sizes (1024 x 768 is the 3-D
    configuration's Gamma_1 block) and beyond the cluster kernel in both
    orientations (300 and 600 columns of the worked matrix): singular values
    as the oracle's, both sets of singular vectors orthonormal (to 1e-12, or
    to the bound of _orth_tol for vectors formed as W v / sigma), B
    reproduced to 1e-13 s_1, and the leading subspaces at gaps as the
    oracle's."""
    M_D, M_tot, M_1 = shape
    N = 100_000
    C = W.synthetic_counts(M_D, M_tot, N, seed=M_D)
    g1 = np.zeros(M_tot, np.uint8)
    g1[:M_1] = 1
    sigma = np.full(M_tot, 2 * np.pi / M_tot)
    nu = np.full(M_D, 1 / np.sqrt(M_D))
    (U, s, V, sweeps), (Uo, so, Vo), _ = _svd_pair(C, N, g1, sigma, nu)
    _check_sv(s, so)
    assert sweeps < 40
    k = len(s)
    tol = _orth_tol(so) if max(M_D, M_1) > 256 and min(M_D, M_1) > 256 else 1e-12
    assert np.all(np.abs(U.T @ U - np.eye(k)) <= tol)
    assert np.all(np.abs(V.T @ V - np.eye(k)) <= tol)
    B = O.operator_B(C, N, g1, nu, sigma)
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, B, atol=1e-13 * so[0])
    for r in _gaps(so, 12):
        np.testing.assert_allclose(U[:, :r] @ U[:, :r].T, Uo[:, :r] @ Uo[:, :r].T, atol=1e-8)
        np.testing.assert_allclose(V[:, :r] @ V[:, :r].T, Vo[:, :r] @ Vo[:, :r].T, atol=1e-8)


def test_reconstruction_matches_oracle():
    inst = W.annulus_config(N=2000, grid=6, m_each=32)
    C, _, _ = O.build_counts(inst)
    sigma = O.element_measures(inst.domain, inst.partition)
    sigma_lib = wos.wos_element_measures(inst.domain, inst.partition)
    g1 = inst.partition.gamma1
    nu = inst.nu_vec()
    meas = W.measurements(inst, noise=0.01)
    (U, s, V, _), (Uo, so, Vo), (Ct, sg, nut) = _svd_pair(C, inst.N, g1, sigma, nu,
                                                          sigma_lib)
    Ut, St, Vt = (torch.as_tensor(x, device=DEV) for x in (U, s, V))
    uD = torch.as_tensor(meas.uD, device=DEV)
    u0 = torch.as_tensor(meas.u0, device=DEV)
    gaps = _gaps(so, 20)
    assert gaps
    for r in gaps:
        u1, uhat = wos.wos_reconstruct(ctx(), Ut, St, Vt, Ct, inst.N, g1, sg, uD, r,
                                       u0=u0, nu=nut)
        ro, rhat = O.reconstruct(Uo, so, Vo, r, C, inst.N, g1, nu, sigma, meas.uD, meas.u0)
        u1 = u1.cpu().numpy()
        assert np.linalg.norm(u1 - ro) <= 1e-8 * np.linalg.norm(ro), r
        assert np.linalg.norm(uhat.cpu().numpy() - rhat) <= 1e-8 * np.linalg.norm(rhat)
    u1, _ = wos.wos_reconstruct(ctx(), Ut, St, Vt, Ct, inst.N, g1, sg, uD, len(s), u0=u0,
                                nu=nut, tikhonov_alpha=1e-6)
    ro, _ = O.reconstruct(Uo, so, Vo, len(so), C, inst.N, g1, nu, sigma, meas.uD, meas.u0,
                          tikhonov=1e-6)
    assert np.linalg.norm(u1.cpu().numpy() - ro) <= 1e-8 * np.linalg.norm(ro)


@pytest.mark.parametrize("transposed", [False, True])
def test_rank_deficient_operator(transposed, svd_path):
    """Zero Gamma_1 columns and repeated rows (rank deficiency) on the
    preconditioned path (n >= 32): singular values as the oracle's, B
    reproduced, singular vectors of the non-zero singular values
    orthonormal."""
    M_D, M_1 = (64, 48) if not transposed else (48, 64)
    M_tot = M_1 + 16
    N = 50_000
    C = W.synthetic_counts(M_D, M_tot, N, seed=5)
    g1 = np.zeros(M_tot, np.uint8)
    g1[:M_1] = 1
    C[:, [3, 7, 20]] = 0               # elements no walk reached
    C[10] = C[11] = C[12]              # repeated rows
    sigma = np.full(M_tot, 2 * np.pi / M_tot)
    nu = np.full(M_D, 1 / np.sqrt(M_D))
    (U, s, V, sweeps), (Uo, so, Vo), _ = _svd_pair(C, N, g1, sigma, nu)
    _check_sv(s, so)
    B = O.operator_B(C, N, g1, nu, sigma)
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, B, atol=1e-13 * so[0])
    nz = s > 1e-12 * s[0]
    np.testing.assert_allclose(U[:, nz].T @ U[:, nz], np.eye(nz.sum()), atol=1e-12)
    np.testing.assert_allclose(V[:, nz].T @ V[:, nz], np.eye(nz.sum()), atol=1e-12)


@pytest.mark.parametrize("shape", [(256, 256, 128), (300, 1536, 768)])
def test_svd_is_deterministic(shape, svd_path):
    """Repeated SVDs of the same counts are bit-identical (the preconditioned
    path's cooperative QR and the Jacobi dataflow take the same decisions
    whatever the CTA timing)."""
    M_D, M_tot, M_1 = shape
    C = W.synthetic_counts(M_D, M_tot, 100_000, seed=M_D + 1)
    g1 = np.zeros(M_tot, np.uint8)
    g1[:M_1] = 1
    Ct = torch.as_tensor(C.astype(np.int32), device=DEV)
    sg = torch.full((M_tot,), 2 * np.pi / M_tot, dtype=torch.float64, device=DEV)
    ref = wos.wos_op_svd(ctx(), Ct, 100_000, g1, sg)
    side = torch.cuda.Stream()
    for rep in range(4):
        with torch.cuda.stream(side):  # another stream and a busy GPU
            busy = torch.randn(4096, 4096, device=DEV) @ torch.randn(4096, 4096, device=DEV)
        got = wos.wos_op_svd(ctx(), Ct, 100_000, g1, sg)
        torch.cuda.synchronize()
        for a, b in zip(ref[:3], got[:3]):
            assert torch.equal(a, b), rep


@pytest.mark.parametrize("large", [False, True, "fp64", "dense"],
                         ids=["mixed", "without-V", "fp64-sweeps", "dense"])
def test_batched_svd_equals_single_calls(svd_path, large):
    """wos_op_svd_batched: problems of different shapes and orientations
    (direct path n < 32 and preconditioned n >= 32), and a batch larger than
    the co-resident CTAs of one launch, give each problem's single-call
    results bit for bit.  Problems of more than 256 columns (sweeps without
    V): with the FP32 preconditioning (a CTA per pair alone and in the
    batch), and with FP64 sweeps alone in a batch large enough for four
    pairs per CTA against single calls with a CTA per pair (the two kernels'
    canonical summation order); and four 1024 x 768 problems, whose FP64
    sweeps take the twelve-CTAs-an-SM variant of the kernel."""
    if large == "fp64":
        wos.wos_set_svd_path(ctx(), wos.SVD_FP64_SWEEPS)
    if large == "dense":
        shapes = [(1024, 1536, 768)] * 4
    elif large:
        shapes = [(600, 900, 300), (300, 900, 600), (520, 800, 400), (700, 1000, 350)]
    else:
        shapes = [(256, 256, 128), (96, 300, 200), (40, 60, 20), (64, 96, 48),
                  (300, 400, 150)]
        shapes += [(128, 200, 96)] * 24
    items, refs = [], []
    for q, (M_D, M_tot, M_1) in enumerate(shapes):
        C = W.synthetic_counts(M_D, M_tot, 50_000, seed=q + 11)
        g1 = np.zeros(M_tot, np.uint8)
        g1[:M_1] = 1
        Ct = torch.as_tensor(C.astype(np.int32), device=DEV)
        sg = torch.full((M_tot,), 2 * np.pi / M_tot, dtype=torch.float64, device=DEV)
        items.append((Ct, 50_000, g1, sg))
        refs.append(wos.wos_op_svd(ctx(), Ct, 50_000, g1, sg))
    got = wos.wos_op_svd_batched(ctx(), items)
    torch.cuda.synchronize()
    wos.wos_set_svd_path(ctx(), svd_path)
    for q, (r, g) in enumerate(zip(refs, got)):
        for a, b in zip(r[:3], g[:3]):
            assert torch.equal(a, b), q
        assert r[3] == g[3]


@pytest.mark.parametrize("shape", [(32, 48, 16), (20, 48, 30), (256, 256, 128), (96, 300, 200),
                                   (300, 400, 256), (33, 40, 33)])
def test_cluster_and_grid_kernels_agree(shape):
    """The cluster kernel and the grid-wide kernels factor the same problems
    (direct path n < 32, preconditioned path, transposed orientation, odd n,
    the largest n the cluster takes): the same singular values to rounding,
    B reproduced by both, the same singular subspaces at gaps; on the
    preconditioned path the cluster kernel is the one taken (fewer launches:
    no separate QR, X and Jacobi launches)."""
    M_D, M_tot, M_1 = shape
    N = 80_000
    C = W.synthetic_counts(M_D, M_tot, N, seed=M_D + M_1)
    g1 = np.zeros(M_tot, np.uint8)
    g1[:M_1] = 1
    Ct = torch.as_tensor(C.astype(np.int32), device=DEV)
    sg = torch.full((M_tot,), 2 * np.pi / M_tot, dtype=torch.float64, device=DEV)
    c = ctx()
    out = {}
    launches = {}
    for path in (wos.SVD_AUTO, wos.SVD_GRID):
        wos.wos_set_svd_path(c, path)
        torch.cuda.synchronize()
        l0 = c.kernel_launches()
        U, S, V, sw = wos.wos_op_svd(c, Ct, N, g1, sg)
        torch.cuda.synchronize()
        launches[path] = c.kernel_launches() - l0
        out[path] = (U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy(), sw)
    wos.wos_set_svd_path(c, wos.SVD_AUTO)
    if min(M_D, M_1) >= 32:  # preconditioned: QR, X and Jacobi are one launch
        assert launches[wos.SVD_AUTO] < launches[wos.SVD_GRID]
    Ua, sa, Va, swa = out[wos.SVD_AUTO]
    Ug, sg_, Vg, swg = out[wos.SVD_GRID]
    _check_sv(sa, sg_)
    B = O.operator_B(C, N, g1, np.full(M_D, 1 / np.sqrt(M_D)), np.full(M_tot, 2 * np.pi / M_tot))
    for U, s, V in ((Ua, sa, Va), (Ug, sg_, Vg)):
        np.testing.assert_allclose(U @ np.diag(s) @ V.T, B, atol=1e-13 * s[0])
        k = len(s)
        np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-12)
        np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-12)
    for r in _gaps(sg_, 16):
        np.testing.assert_allclose(Ua[:, :r] @ Ua[:, :r].T, Ug[:, :r] @ Ug[:, :r].T, atol=1e-8)
    assert abs(swa - swg) <= 2


@pytest.mark.parametrize("shape", [(1, 3, 1), (2, 3, 1), (1, 4, 3), (3, 5, 2), (5, 7, 5),
                                   (31, 40, 31), (2, 40, 33)])
def test_degenerate_shapes(shape, svd_path):
    """One row, one column, square, n just below and above the QR threshold
    (31, 33), a wide operator with two points: singular values as LAPACK's,
    B reproduced, orthonormal vectors."""
    M_D, M_tot, M_1 = shape
    N = 5000
    C = W.synthetic_counts(M_D, M_tot, N, seed=sum(shape))
    g1 = np.zeros(M_tot, np.uint8)
    g1[:M_1] = 1
    sigma = np.full(M_tot, 2 * np.pi / M_tot)
    nu = np.full(M_D, 1 / np.sqrt(M_D))
    (U, s, V, sweeps), (Uo, so, Vo), _ = _svd_pair(C, N, g1, sigma, nu)
    B = O.operator_B(C, N, g1, nu, sigma)
    ref = np.linalg.svd(B, compute_uv=False)
    np.testing.assert_allclose(s, ref, rtol=1e-12, atol=1e-15 * ref[0])
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, B, atol=1e-13 * ref[0])
    k = len(s)
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-12)


@pytest.mark.parametrize("shape", [(1024, 1536, 768), (300, 900, 600), (600, 900, 300),
                                   (520, 800, 257)])
def test_fp32_preconditioned_sweeps_agree_with_fp64_sweeps(shape):
    """Problems of more than 256 columns: the default path (FP32 sweeps on X
    in a thread-block cluster, their rotations replayed into J, two
    Newton-Schulz steps in FP64, then FP64 sweeps from X Q) and FP64 sweeps
    alone both match LAPACK's singular values of the same FP64 matrix (the
    default path to 1e-13 relative, every value; FP64 sweeps alone, whose
    ten-odd sweeps of scaled rotations round more, to 1e-12), give the same
    singular subspaces at gaps and orthonormal vectors; the preconditioned
    FP64 sweeps are at most half as many."""
    M_D, M_tot, M_1 = shape
    N = 100_000
    C = W.synthetic_counts(M_D, M_tot, N, seed=M_D + 3 * M_1)
    g1 = np.zeros(M_tot, np.uint8)
    g1[:M_1] = 1
    Ct = torch.as_tensor(C.astype(np.int32), device=DEV)
    sg = torch.full((M_tot,), 2 * np.pi / M_tot, dtype=torch.float64, device=DEV)
    c = ctx()
    out = {}
    for path in (wos.SVD_FP64_SWEEPS, wos.SVD_AUTO):
        wos.wos_set_svd_path(c, path)
        U, S, V, sw = wos.wos_op_svd(c, Ct, N, g1, sg)
        out[path] = (U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy(), sw)
    wos.wos_set_svd_path(c, wos.SVD_AUTO)
    (U0, s0, V0, sw0), (U1, s1, V1, sw1) = out[wos.SVD_FP64_SWEEPS], out[wos.SVD_AUTO]
    B = O.operator_B(C, N, g1, np.full(M_D, 1 / np.sqrt(M_D)), np.full(M_tot, 2 * np.pi / M_tot))
    s_lapack = np.linalg.svd(B, compute_uv=False)
    assert np.max(np.abs(s1 / s_lapack - 1)) <= 1e-13, np.max(np.abs(s1 / s_lapack - 1))
    assert np.max(np.abs(s0 / s_lapack - 1)) <= 1e-12, np.max(np.abs(s0 / s_lapack - 1))
    assert 2 * sw1 <= sw0, (sw0, sw1)
    k = len(s1)
    for U in (U1, V1):
        G = U.T @ U
        tol = _orth_tol(s1)
        assert np.all(np.abs(G - np.eye(k)) <= tol), np.max(np.abs(G - np.eye(k)) / tol)
    for r in _gaps(s0, 40):
        for A, B2 in ((U0, U1), (V0, V1)):
            P0, P1 = A[:, :r] @ A[:, :r].T, B2[:, :r] @ B2[:, :r].T
            assert np.abs(P0 - P1).max() <= 1e-9, r


def test_svd_above_768_columns_runs_fp64_sweeps_alone():
    """A worked matrix of more than 768 columns (more than the FP32 sweeps'
    columns hold in a lane's registers) takes the FP64-only path by default:
    the same sweep count as with WOS_SVD_FP64_SWEEPS, bit-identical results,
    and singular values within 1e-12 of LAPACK's."""
    M_D, M_tot, M_1 = 800, 1200, 780
    N = 100_000
    C = W.synthetic_counts(M_D, M_tot, N, seed=7)
    g1 = np.zeros(M_tot, np.uint8)
    g1[:M_1] = 1
    Ct = torch.as_tensor(C.astype(np.int32), device=DEV)
    sg = torch.full((M_tot,), 2 * np.pi / M_tot, dtype=torch.float64, device=DEV)
    c = ctx()
    U, S, V, sw = wos.wos_op_svd(c, Ct, N, g1, sg)
    wos.wos_set_svd_path(c, wos.SVD_FP64_SWEEPS)
    U0, S0, V0, sw0 = wos.wos_op_svd(c, Ct, N, g1, sg)
    wos.wos_set_svd_path(c, wos.SVD_AUTO)
    assert sw == sw0 and sw >= 5, (sw, sw0)
    assert torch.equal(S, S0) and torch.equal(U, U0) and torch.equal(V, V0)
    B = O.operator_B(C, N, g1, np.full(M_D, 1 / np.sqrt(M_D)), np.full(M_tot, 2 * np.pi / M_tot))
    s_lapack = np.linalg.svd(B, compute_uv=False)
    assert np.max(np.abs(S.cpu().numpy() / s_lapack - 1)) <= 1e-12


def test_svd_path_setting_is_checked():
    for bad in (-1, 4, 100):
        with pytest.raises(wos.WosError) as e:
            wos.wos_set_svd_path(ctx(), bad)
        assert e.value.code == 1
    wos.wos_set_svd_path(ctx(), wos.SVD_AUTO)


def test_bauer_spiral_shell_end_to_end_with_library_measures():
    """The paper's own discretisation of Ex. 5.6 (unit ball minus the ball of
    radius 1/2; extrinsic Voronoi cells of 1000 + 100 Bauer-spiral sites;
    100 points on the spiral of radius 0.95) through the library alone:
    build, cell measures sigma(omega_j) from wos_element_measures (no caller
    measures), SVD and TSVD.  Against the oracle on the same counts (with the
    oracle's own measures): singular values to 1e-10, the reconstruction at
    the gaps to 1e-8."""
    from gpu_util import gpu_build
    inst = W.shell_config(N=20_000, n_points=100, voronoi=(1000, 100))
    r = gpu_build(inst, trace=False)
    C = r["counts"]
    assert (C.sum(1) + r["unterm"] == inst.N).all()
    sigma = O.voronoi_measures(inst.domain, inst.partition)
    sigma_lib = wos.wos_element_measures(inst.domain, inst.partition)
    g1 = inst.partition.gamma1
    nu = inst.nu_vec()
    meas = W.measurements(inst, noise=0.01)
    (U, s, V, _), (Uo, so, Vo), (Ct, sg, nut) = _svd_pair(C, inst.N, g1, sigma, nu, sigma_lib)
    _check_sv(s, so)
    Ut, St, Vt = (torch.as_tensor(x, device=DEV) for x in (U, s, V))
    uD = torch.as_tensor(meas.uD, device=DEV)
    u0 = torch.as_tensor(meas.u0, device=DEV)
    gaps = _gaps(so, 40)   # clusters of 1, 3, 5, 7, ... (Sec. 5.3): gaps at 16, 25
    assert gaps
    for rr in gaps:
        u1, _ = wos.wos_reconstruct(ctx(), Ut, St, Vt, Ct, inst.N, g1, sg, uD, rr, u0=u0,
                                    nu=nut)
        ro, _ = O.reconstruct(Uo, so, Vo, rr, C, inst.N, g1, nu, sigma, meas.uD, meas.u0)
        assert np.linalg.norm(u1.cpu().numpy() - ro) <= 1e-8 * np.linalg.norm(ro), rr
