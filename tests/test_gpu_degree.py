"""The degree options of the density kernel on the GPU (sq3_kernel_from_hs_ex):
the Paterson-Stockmeyer evaluation against the plain recurrence and the
oracle's Fermi-operator expansion (Sec. 4) at the same degree, and the
degree chosen from a tolerance against the library's rule and the oracle
at that degree.  In FP64 the two evaluations are the same polynomial, so
they agree to rounding (1e-12 of the largest entry); the mixed path's
Paterson-Stockmeyer form is held to the mixed recurrence's bar."""
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


@pytest.mark.parametrize("npl,Ns", [(5, 40), (60, 150), (120, 200), (121, 131), (120, 2200)])
def test_mixed_paterson_stockmeyer_matches_the_oracle_and_the_mixed_recurrence(npl, Ns):
    """The mixed path's Paterson-Stockmeyer form (FP32 matrices, BF16-split
    tensor-core products, Clenshaw in T_s) against the FP64 oracle expansion
    at the same degree and bounds, with the mixed recurrence's bar (D within
    2e-5, mu within 1e-5), and against the mixed recurrence itself; Ns = 2200, n_pl = 120 is the 108-atom workload's
    expansion (s = 16 baby steps, 7 giant steps, 28 products)."""
    m = sq3()
    ctx = _ctx()
    Hs, lam = _hs(Ns, npl + Ns)
    chi, xi = 0.5 * (lam[0] + lam[-1]), 0.5 * (lam[-1] - lam[0]) * 1.001
    sigma, Ne = inputs.ev_to_ha(10.0), 0.3 * Ns
    Hg = torch.from_numpy(Hs).cuda()
    Dp, outp, npp = ctx.kernel_from_hs_ex(Hg, npl, sigma, Ne, bounds=(chi, xi), prec=m.MIXED,
                                          eval_mode=m.EVAL_PATERSON_STOCKMEYER)
    Dr, outr, _ = ctx.kernel_from_hs_ex(Hg, npl, sigma, Ne, bounds=(chi, xi), prec=m.MIXED)
    assert npp == npl
    Dp, Dr = Dp.cpu().numpy(), Dr.cpu().numpy()
    ref = chebyshev.foe_density_kernel(Hs, npl, sigma, Ne, chi, xi)
    assert np.max(np.abs(Dp - ref["D"])) < 2e-5
    assert np.max(np.abs(Dp - Dr)) < 2e-5
    assert abs(outp["mu"] - ref["mu"]) < 1e-5
    # the energies are sums over Ns states: 1e-4 absolute or 1e-5 relative
    # (the FP32 moments' rounding grows with Ns), and no worse than the
    # mixed recurrence's own error
    for k in ("e_band", "e_ent"):
        err_p, err_r = abs(outp[k] - ref[k]), abs(outr[k] - ref[k])
        assert err_p < max(1e-4, 1e-5 * abs(ref[k])), k
        assert err_p < 2.0 * err_r + 1e-4, k
    assert abs(outp["two_tr_D"] - Ne) < 1e-9


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
