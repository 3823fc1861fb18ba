"""Real flavor (real coefficients under inversion and time reversal) on the
GPU against the FP64 oracle.  Bars as for the complex flavor: 1e-12 relative
Frobenius on the plain FP64 path, 1e-5 for FP32 M, 1e-5/1e-6 (FP16 split)
and 3e-5/1e-5 (BF16 split) on chi/eps~^-1 of the mixed path."""
import numpy as np
import pytest

import oracle
from paper_1111_4429_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4429_gb300 import bgw
    return bgw.Context(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _real_c0(**kw):
    p = dict(synth.CONFIGS["c0"])
    p.update(kw)
    return synth.make_system("c0r", **p, real=True)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_real_flavor_mtxel_and_chi(ctx, prec):
    from paper_1111_4429_gb300 import bgw
    s = _real_c0()
    cell = bgw.system_cell(s)
    rdt = torch.float64 if prec == 0 else torch.float32
    M = torch.empty((s.npairs, s.ng), dtype=rdt, device="cuda")
    ctx.mtxel(cell, s.gv, _dev(s.cv), s.gc, _dev(s.cc), s.geps, prec | bgw.BGW_FLAVOR_REAL, M)
    chi = torch.zeros((1, s.ng, s.ng), dtype=torch.float64, device="cuda")
    ctx.chi_sum(cell, s.nv, s.nc, s.ng, M, s.ev, s.ec, None, prec | bgw.BGW_FLAVOR_REAL, False, chi)
    ctx.sync()
    mref = oracle.mtxel_direct(s.gv, s.cv, s.gc, s.cc, s.geps).real
    xref = oracle.chi(mref, oracle.chi_weights(s.ev, s.ec), s.omega).real
    m, x = M.cpu().numpy().astype(np.float64), chi[0].cpu().numpy()
    assert _rel(m, mref) <= (TOL64 if prec == 0 else 1e-5)
    assert _rel(x, xref) <= {0: TOL64, 1: 1e-5, 2: 3e-5}[prec]
    assert np.array_equal(x, x.T)


@pytest.mark.parametrize("tc", [0, 1])
def test_real_flavor_inverse(ctx, tc):
    from paper_1111_4429_gb300 import bgw
    s = _real_c0()
    r = oracle.solve(s)
    x = _dev(r["chi"].real)
    inv = torch.zeros_like(x)
    eps = torch.zeros_like(x)
    try:
        ctx.set_option(bgw.BGW_OPT_INVERSE, tc)
        ctx.epsinv_rflavor([bgw.system_cell(s)], [s.geps], [x], [eps], [inv])
        ctx.sync()
    finally:
        ctx.set_option(bgw.BGW_OPT_INVERSE, -1)
    assert _rel(eps.cpu().numpy(), r["eps"].real) <= TOL64
    assert _rel(inv.cpu().numpy(), r["epsinv"].real) <= TOL64
    g = inv.cpu().numpy()
    assert np.array_equal(g, g.T)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_real_flavor_whole_path_vs_complex_flavor(ctx, prec):
    """bgw_epsilon with the flavor flag (host buffers, conduction chunks,
    imaginary frequencies) against the oracle, and against the complex path
    on the same coefficients held as complex numbers."""
    from paper_1111_4429_gb300 import bgw
    s = synth.make_system("rr", a=14.0, fft=24, ecut_wfn=6.0, ecut_eps=2.5, nv=5, nc=37, seed=97, real=True)
    om = np.concatenate([[0.0], synth.gauss_legendre_frequencies(2)])
    cell = bgw.system_cell(s)
    chi = np.zeros((3, s.ng, s.ng))
    inv = np.zeros((3, s.ng, s.ng))
    ctx.epsilon(cell, s.gv, s.cv, s.ev, s.gc, s.cc, s.ec, s.geps, om, prec | bgw.BGW_FLAVOR_REAL, 10, chi, inv)
    chic = np.zeros((3, s.ng, s.ng), dtype=np.complex128)
    invc = np.zeros_like(chic)
    ctx.epsilon(cell, s.gv, s.cv.astype(np.complex128), s.ev, s.gc, s.cc.astype(np.complex128), s.ec, s.geps, om,
                prec, 10, chic, invc)
    m = oracle.mtxel_direct(s.gv, s.cv, s.gc, s.cc, s.geps).real
    v = oracle.coulomb(s.bvec, s.q_frac, s.geps)
    tol = {0: TOL64, 1: 1e-6, 2: 1e-5}[prec]
    for f, w in enumerate(om):
        x = oracle.chi(m, oracle.chi_weights(s.ev, s.ec, w), s.omega)
        _, ei = oracle.epsinv_sym(x, v)
        assert _rel(inv[f], ei.real) <= tol
        assert _rel(inv[f], invc[f].real) <= (1e-13 if prec == 0 else 2 * tol)
        assert np.abs(invc[f].imag).max() <= 1e-13 * np.abs(invc[f]).max() or prec != 0


def test_real_flavor_unsupported_combinations(ctx):
    from paper_1111_4429_gb300 import bgw
    s = _real_c0()
    chi = torch.zeros((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    inv = torch.zeros_like(chi)
    with pytest.raises(bgw.BgwError) as e:
        ctx.epsilon_real(bgw.system_cell(s), s.gv, _dev(s.cv), s.ev, s.gc, _dev(s.cc), s.ec, s.geps,
                         np.array([0.2]), 0.05, False, bgw.BGW_FLAVOR_REAL, 0, chi, inv)
    assert e.value.code == 8
    with pytest.raises(bgw.BgwError) as e:
        ctx.epsilon_batch([s], [_dev(s.cv)], [_dev(s.cc)], None, bgw.BGW_FLAVOR_REAL, [inv])
    assert e.value.code == 8
