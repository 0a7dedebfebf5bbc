"""The degree options of the density kernel on the GPU (sq3_kernel_from_hs_ex):
the Paterson-Stockmeyer evaluation against the plain recurrence and the
oracle's Fermi-operator expansion (Sec. 4) at the same degree, and the
degree chosen from a tolerance against the library's rule and the oracle
at that degree.  FP64 throughout: the two evaluations are the same
polynomial, so they agree to rounding (1e-12 of the largest entry)."""
import numpy as np
import pytest
import torch

from oracle import chebyshev, fermi
from paper_2112_08639_gb300 import inputs

from gpu_common import need_gpu, sq3

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _ctx():
    c = sq3().Context(0)
    c.setup_grid(8, 8, 8, 4.0, 4.0, 4.0, 12)
    return c


def _hs(Ns, seed, lo=-0.6, hi=2.4):
    rng = np.random.default_rng(seed)
    lam = np.sort(rng.uniform(lo, hi, Ns))
    Q, _ = np.linalg.qr(rng.normal(size=(Ns, Ns)))
    H = (Q * lam) @ Q.T
    return 0.5 * (H + H.T), lam


@pytest.mark.parametrize("npl,Ns", [(5, 40), (16, 90), (60, 150), (120, 200), (121, 131)])
def test_paterson_stockmeyer_equals_the_recurrence_and_the_oracle(npl, Ns):
    m = sq3()
    ctx = _ctx()
    Hs, lam = _hs(Ns, npl)
    chi, xi = 0.5 * (lam[0] + lam[-1]), 0.5 * (lam[-1] - lam[0]) * 1.001
    sigma, Ne = inputs.ev_to_ha(10.0), 0.3 * Ns
    Hg = torch.from_numpy(Hs).cuda()
    Dr, outr, nr = ctx.kernel_from_hs_ex(Hg, npl, sigma, Ne, bounds=(chi, xi))
    Dp, outp, npp = ctx.kernel_from_hs_ex(Hg, npl, sigma, Ne, bounds=(chi, xi),
                                          eval_mode=m.EVAL_PATERSON_STOCKMEYER)
    assert nr == npp == npl
    Dr, Dp = Dr.cpu().numpy(), Dp.cpu().numpy()
    assert np.max(np.abs(Dp - Dr)) < 1e-12 * np.max(np.abs(Dr))
    for k in ("mu", "e_band", "e_ent", "two_tr_D"):
        assert abs(outp[k] - outr[k]) < 1e-11 * max(1.0, abs(outr[k])), k
    ref = chebyshev.foe_density_kernel(Hs, npl, sigma, Ne, chi, xi)
    assert np.max(np.abs(Dp - ref["D"])) < 1e-11 * np.max(np.abs(ref["D"]))
    assert abs(outp["mu"] - ref["mu"]) < 1e-11


def test_paterson_stockmeyer_rejects_the_mixed_path():
    m = sq3()
    ctx = _ctx()
    Hs, _ = _hs(40, 1)
    with pytest.raises(m.SQ3Error) as e:
        ctx.kernel_from_hs_ex(torch.from_numpy(Hs).cuda(), 20, 0.3, 10.0, prec=m.MIXED,
                              eval_mode=m.EVAL_PATERSON_STOCKMEYER)
    assert e.value.code == m.EINVAL


@pytest.mark.parametrize("kT_ev,tol", [(10.0, 1e-8), (50.0, 1e-10), (250.0, 1e-12)])
def test_adaptive_degree_meets_its_tolerance(kT_ev, tol):
    """npl < 1: the degree is the library's rule at the Lanczos bounds; the
    kernel at that degree equals the oracle's expansion at the same degree,
    and the occupations are within the tolerance of the exact Fermi
    function (Ds against g(Hs) by diagonalisation)."""
    m = sq3()
    ctx = _ctx()
    Ns = 160
    Hs, lam = _hs(Ns, int(kT_ev))
    sigma, Ne = inputs.ev_to_ha(kT_ev), 0.25 * Ns
    D, out, used = ctx.kernel_from_hs_ex(torch.from_numpy(Hs).cuda(), 0, sigma, Ne,
                                         fermi_tol=tol,
                                         eval_mode=m.EVAL_PATERSON_STOCKMEYER)
    assert used == m.fermi_degree(sigma, out["xi"], tol)
    ref = chebyshev.foe_density_kernel(Hs, used, sigma, Ne, out["chi"], out["xi"])
    D = D.cpu().numpy()
    assert np.max(np.abs(D - ref["D"])) < 1e-11
    w, U = np.linalg.eigh(Hs)
    g = fermi.fermi(w, out["mu"], sigma)
    assert np.max(np.abs(D - (U * g) @ U.T)) < 10 * tol


def test_scf_driver_with_paterson_stockmeyer_matches_the_dense_oracle_scf():
    from oracle import scf
    from gpu_common import to_gpu_block
    n, L, Ns, Ne = 12, inputs.A0_FCC, 57, 12.0
    pos = inputs.fcc_positions(1, disp_sigma=0.05, seed=0)
    sigma, Z, rc = inputs.ev_to_ha(10.0), inputs.Z_VALENCE, inputs.RC_LOCAL
    dV = (L / n) ** 3
    ref = scf.scf(n, L, pos, Ns=Ns, sigma=sigma, Z=Z, rc=rc, tol=1e-11)
    m = sq3()
    ctx = m.Context(0)
    ctx.setup_grid(n, n, n, L, L, L, 12)
    b, _ = ctx.pseudocharge(pos, Z, rc)
    rho = torch.full((n ** 3,), Ne / (n ** 3 * dV), dtype=torch.float64, device="cuda:0")
    X = to_gpu_block(inputs.random_block(n ** 3, Ns, seed=0).T)
    res, hist = ctx.scf_solve(b, rho, X, degree=16, npl=80, kT=sigma, Ne=Ne,
                              e_self=scf.self_energy(4, Z, rc), tol=1e-10, first_passes=12,
                              passes=3, max_iter=80, cut_shift=0.07,
                              kernel_eval=m.EVAL_PATERSON_STOCKMEYER)
    assert res["converged"] == 1
    assert np.sum(np.abs(rho.cpu().numpy() - ref["rho"])) * dV / Ne < 1e-8
    assert abs(res["F"] - ref["F"]) / 4 < 1e-8
