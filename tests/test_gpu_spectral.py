"""wos_spectral (Sec. 5.2 items (i)-(iv)) against the oracle's definitions on
the same counts and the same SVD factors, and its TSVD family against
wos_reconstruct at every truncation (bit for bit: same arithmetic, same
order)."""
import numpy as np
import pytest
import torch

from gpu_util import ctx, gpu_build
from oracle import oracle as O
from paper_2409_03686_gb300 import workloads as W
from paper_2409_03686_gb300 import wos

pytestmark = pytest.mark.gpu

CASES = {
    "annulus": lambda: W.annulus_config(N=3000, grid=6, m_each=40),
    "square": lambda: W.square_config(N=3000, grid=6),
    "ball": lambda: W.ball_config(N=2000, n_points=48, nb=8, ns=12),
}


@pytest.mark.parametrize("name", list(CASES))
def test_spectral_matches_oracle_definitions(name):
    inst = CASES[name]()
    dev = torch.device("cuda:0")
    g = gpu_build(inst, trace=False)
    C = g["counts_t"]
    g1 = inst.partition.gamma1
    sig = wos.wos_element_measures(inst.domain, inst.partition)
    sig_t = torch.as_tensor(sig, device=dev)
    meas = W.measurements(inst, noise=0.01)
    uD = torch.as_tensor(meas.uD, device=dev)
    u0 = torch.as_tensor(meas.u0, device=dev)
    U, S, V, _ = wos.wos_op_svd(ctx(), C, inst.N, g1, sig_t)
    k = int(S.shape[0])
    r_max = min(k, 24)
    out = wos.wos_spectral(ctx(), U, S, V, C, inst.N, g1, sig_t, uD=uD, u0=u0, r_max=r_max)
    torch.cuda.synchronize()
    Un, Sn, Vn = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    Cn = g["counts"]
    ref = O.spectral(Un, Sn, Vn, Cn, inst.N, g1, inst.nu_vec(), sig, meas.uD, meas.u0,
                     r_max=r_max)
    lam = out["lambda_"].cpu().numpy()
    big = ref["lam"] >= 1e-6 * ref["lam"][0]
    np.testing.assert_allclose(lam[big], ref["lam"][big], rtol=1e-9)
    assert np.all(np.abs(lam - ref["lam"]) <= 1e-12 * ref["lam"][0])
    ef = out["eigfun"].cpu().numpy()
    np.testing.assert_allclose(ef, ref["eigfun"], rtol=1e-10,
                               atol=1e-12 * np.abs(ref["eigfun"]).max())
    np.testing.assert_allclose(out["density"].cpu().numpy(), ref["density"], rtol=1e-13)
    us, ys = out["u_sweep"].cpu().numpy(), out["uD_sweep"].cpu().numpy()
    for r in range(r_max):
        np.testing.assert_allclose(us[r], ref["u_sweep"][r], rtol=1e-9,
                                   atol=1e-11 * np.abs(ref["u_sweep"][r]).max())
        np.testing.assert_allclose(ys[r], ref["uD_sweep"][r], rtol=1e-9, atol=1e-11)
    # the family equals single reconstructions, bit for bit
    for r in (1, r_max // 2, r_max):
        u1, uhat = wos.wos_reconstruct(ctx(), U, S, V, C, inst.N, g1, sig_t, uD, r, u0=u0)
        assert torch.equal(out["u_sweep"][r - 1], u1), r
        assert torch.equal(out["uD_sweep"][r - 1], uhat), r


def test_spectral_options_and_errors():
    inst = W.disc_config(N=500)
    dev = torch.device("cuda:0")
    g = gpu_build(inst, trace=False)
    C = g["counts_t"]
    g1 = inst.partition.gamma1
    sig_t = torch.as_tensor(wos.wos_element_measures(inst.domain, inst.partition),
                            device=dev)
    U, S, V, _ = wos.wos_op_svd(ctx(), C, inst.N, g1, sig_t)
    out = wos.wos_spectral(ctx(), U, S, V, C, inst.N, g1, sig_t, want_eigfun=False)
    torch.cuda.synchronize()
    assert out["eigfun"] is None and "u_sweep" not in out
    assert torch.allclose(out["lambda_"], S * S)
    with pytest.raises(wos.WosError) as e:  # a sweep needs the measurements
        wos.wos_spectral(ctx(), U, S, V, C, inst.N, g1, sig_t, r_max=2)
    assert e.value.code == 1
    with pytest.raises(wos.WosError):  # r_max beyond k
        wos.wos_spectral(ctx(), U, S, V, C, inst.N, g1, sig_t,
                         uD=torch.zeros(inst.M_D, dtype=torch.float64, device=dev),
                         r_max=int(S.shape[0]) + 1)
