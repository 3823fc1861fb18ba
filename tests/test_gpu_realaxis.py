"""Real-axis (full-frequency) response on the GPU against the FP64 oracle.

Eq. retarded_advanced_epsilon with broadening delta: complex pair weights, a
non-Hermitian chi and eps~, and an inverse with partial pivoting.  Bars: the
plain FP64 path within 1e-12 relative Frobenius; the mixed precisions (X = M
and Y = w M split into FP16 or BF16 hi/lo on the tensor cores) within 1e-6
(FP16) or 1e-5 (BF16) on eps~^-1, as for the imaginary axis.
"""
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


def _real(ctx, s, energies, delta, advanced=False, prec=0, nc_chunk=0, cell=None):
    from paper_1111_4429_gb300 import bgw
    nf = len(energies)
    chi = torch.zeros((nf, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    inv = torch.zeros_like(chi)
    ctx.epsilon_real(cell or bgw.system_cell(s), s.gv, _dev(s.cv), s.ev, s.gc, _dev(s.cc), s.ec, s.geps,
                     np.asarray(energies, dtype=np.float64), delta, advanced, prec, nc_chunk, chi, inv)
    ctx.sync()
    return chi.cpu().numpy(), inv.cpu().numpy()


E_C0 = [0.0, 0.35, 0.8, 1.6]


@pytest.mark.parametrize("advanced", [False, True])
def test_real_axis_fp64_c0_vs_oracle(ctx, advanced):
    s = synth.config_system("c0")
    r = oracle.solve_real(s, E_C0, 0.05, advanced=advanced)
    chi, inv = _real(ctx, s, E_C0, 0.05, advanced=advanced)
    for f in range(len(E_C0)):
        assert _rel(chi[f], r["chi"][f]) <= TOL64
        assert _rel(inv[f], r["epsinv"][f]) <= TOL64


def test_real_axis_adjoint_chunks_and_static_limit(ctx):
    s = synth.make_system("r", a=14.0, fft=24, ecut_wfn=6.0, ecut_eps=2.5, nv=5, nc=37, seed=83)
    e = [0.0, 0.5, 1.2]
    chi_r, inv_r = _real(ctx, s, e, 0.03, nc_chunk=10)          # conduction in 4 chunks
    chi_a, inv_a = _real(ctx, s, e, 0.03, advanced=True)
    r = oracle.solve_real(s, e, 0.03)
    for f in range(3):
        assert _rel(inv_r[f], r["epsinv"][f]) <= TOL64
        assert _rel(inv_a[f], np.conj(inv_r[f]).T) <= TOL64
    # E = 0 on the real axis is the imaginary axis at omega = delta
    from paper_1111_4429_gb300 import bgw
    inv_i = torch.zeros((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    ctx.epsilon(bgw.system_cell(s), s.gv, _dev(s.cv), s.ev, s.gc, _dev(s.cc), s.ec, s.geps, np.array([0.03]), 0, 0,
                None, inv_i)
    ctx.sync()
    assert _rel(inv_r[0], inv_i[0].cpu().numpy()) <= TOL64


@pytest.mark.parametrize("tc", [0, 1, 5])
@pytest.mark.parametrize("ng,seed", [(85, 1), (300, 2), (700, 3), (2311, 4)])
def test_general_inverse_pivoting_vs_library(ctx, ng, seed, tc):
    """bgw_epsinv_general on random complex chi of several sizes: one leaf,
    two leaves and a merge, three leaves, ten leaves and two merge rounds;
    trailing updates in FP64 FMA (tc = 0) or on the tensor cores (tc = 1,
    exact 8-bit slices, FP64-level accuracy).  The first diagonal entries of
    eps~ are made to vanish, so elimination without row interchanges would
    divide by zero."""
    from paper_1111_4429_gb300 import bgw
    gen = np.random.default_rng(seed)
    bvec, _ = synth.cubic_cell(30.0)
    geps = synth.gsphere(bvec, (0.1, 0.0, 0.0), 40.0)[:ng]
    assert geps.shape[0] == ng
    cell = bgw.make_cell(bvec, 27000.0, (0.1, 0.0, 0.0), 64)
    v = oracle.coulomb(bvec, (0.1, 0.0, 0.0), geps)
    sv = np.sqrt(v)
    x = (gen.standard_normal((ng, ng)) + 1j * gen.standard_normal((ng, ng))) / (np.sqrt(ng) * sv[:, None] * sv[None, :])
    for i in range(3):
        x[i, i] = 1.0 / v[i]                                   # eps~_ii = 1 - v_i chi_ii = 0 (up to rounding)
    e = np.eye(ng) - sv[:, None] * x * sv[None, :]
    assert np.abs(np.diag(e)[:3]).max() < 1e-12
    ref = np.linalg.inv(e)
    inv = torch.zeros((ng, ng), dtype=torch.complex128, device="cuda")
    eps = torch.zeros_like(inv)
    try:
        # tc: 0 FP64 FMA, 1 tensor cores (7 slices), 5 tensor cores with 5 slices
        ctx.set_option(bgw.BGW_OPT_INVERSE, 1 if tc else 0)
        ctx.set_option(bgw.BGW_OPT_UPDATE_SLICES, 5 if tc == 5 else 0)
        ctx.epsinv_general([cell], [geps], [_dev(x)], [eps], [inv])
        ctx.sync()
    finally:
        ctx.set_option(bgw.BGW_OPT_INVERSE, -1)
        ctx.set_option(bgw.BGW_OPT_UPDATE_SLICES, 0)
    assert _rel(eps.cpu().numpy(), e) <= 1e-15
    got = inv.cpu().numpy()
    cond = np.linalg.cond(e)
    # the tensor-core update is accurate to about 2^-48 of the update's scale
    # with 7 slices, 2^-34 with 5 (FP64 FMA: 2^-53): bars 32 and 2^19 times
    # the FP64 ones
    k = {0: 1, 1: 32, 5: 2 ** 19}[tc]
    assert _rel(got, ref) <= 1e-15 * cond * ng ** 0.5 * max(1, k // 32)
    assert np.linalg.norm(e @ got - np.eye(ng)) / np.sqrt(ng) <= 1e-12 * k


@pytest.mark.parametrize("prec", [1, 2])
def test_real_axis_mixed_c0(ctx, prec):
    s = synth.config_system("c0")
    r = oracle.solve_real(s, E_C0, 0.05)
    chi, inv = _real(ctx, s, E_C0, 0.05, prec=prec)
    tchi, tinv = {1: (1e-5, 1e-6), 2: (3e-5, 1e-5)}[prec]
    for f in range(len(E_C0)):
        ec, ei = _rel(chi[f], r["chi"][f]), _rel(inv[f], r["epsinv"][f])
        print(f"prec {prec} E {E_C0[f]}: chi {ec:.2e} epsinv {ei:.2e}")
        assert ec <= tchi and ei <= tinv


def test_real_axis_mixed_ragged_chunks(ctx):
    from paper_1111_4429_gb300 import bgw
    s = synth.make_system("r", a=14.0, fft=24, ecut_wfn=6.0, ecut_eps=2.5, nv=5, nc=37, seed=85)
    e = [0.2, 0.9]
    r = oracle.solve_real(s, e, 0.04)
    try:
        ctx.set_option(bgw.BGW_OPT_CHI_CHUNK_PAIRS, 64)           # several operand chunks
        chi, inv = _real(ctx, s, e, 0.04, prec=1, nc_chunk=13)
    finally:
        ctx.set_option(bgw.BGW_OPT_CHI_CHUNK_PAIRS, 0)
    for f in range(2):
        assert _rel(chi[f], r["chi"][f]) <= 1e-5
        assert _rel(inv[f], r["epsinv"][f]) <= 1e-6


def test_real_axis_argument_errors(ctx):
    from paper_1111_4429_gb300 import bgw
    s = synth.config_system("c0")
    for e, d, adv in (([0.1], 0.0, False), ([0.1], -1.0, False), ([float("nan")], 0.1, False),
                      ([0.1], float("inf"), False)):
        with pytest.raises(bgw.BgwError) as ex:
            _real(ctx, s, e, d, advanced=adv)
        assert ex.value.code == 1
    M = torch.zeros((s.npairs, s.ng), dtype=torch.complex128, device="cuda")
    chi = torch.zeros((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    with pytest.raises(bgw.BgwError) as ex:
        ctx.chi_sum_real(bgw.system_cell(s), s.nv, s.nc, s.ng, M, s.ev, s.ec, np.zeros(0), 0.1, False, 0, False, chi)
    assert ex.value.code == 1
    big = 14337
    with pytest.raises(bgw.BgwError) as ex:
        ctx.epsinv_general([bgw.system_cell(s)], [np.zeros((big, 3), np.int32)], [chi], None, [chi])
    assert ex.value.code == 8
