"""Argument checks of the C ABI: invalid inputs are refused before any launch."""
import numpy as np
import pytest

from paper_1111_4429_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4429_gb300 import bgw
    return bgw.Context(0)


def _sys():
    return synth.make_system("e", a=8.0, fft=12, ecut_wfn=4.0, ecut_eps=1.5, nv=3, nc=5, seed=3)


def _run(ctx, s, n=None, gv=None, prec=0):
    from paper_1111_4429_gb300 import bgw
    cell = bgw.make_cell(s.bvec, s.omega, s.q_frac, n or s.fft)
    M = torch.zeros((s.nv * s.nc, s.ng), dtype=torch.complex128, device="cuda")
    cv = torch.from_numpy(s.cv).cuda()
    cc = torch.from_numpy(s.cc).cuda()
    ctx.mtxel(cell, s.gv if gv is None else gv, cv, s.gc, cc, s.geps, prec, M)
    return M


def test_aliasing_grid_is_rejected(ctx):
    from paper_1111_4429_gb300 import bgw
    s = synth.config_system("c0")        # max|Gv| + max|Gc| + max|Geps| = 5 + 5 + 2
    with pytest.raises(bgw.BgwError) as e:
        _run(ctx, s, n=12)               # components fit [-6, 6) but 12 <= 12 aliases
    assert e.value.code == bgw.BGW_EINVAL
    assert "aliases" in str(e.value)
    _run(ctx, s, n=20)                   # the configured grid is accepted
    ctx.sync()


def test_g_outside_half_open_range_is_rejected(ctx):
    from paper_1111_4429_gb300 import bgw
    s = _sys()
    gv = s.gv.copy()
    gv[0] = (6, 0, 0)       # n/2 is outside [-n/2, n/2)
    with pytest.raises(bgw.BgwError) as e:
        _run(ctx, s, gv=gv)
    assert e.value.code == bgw.BGW_EINVAL


def test_duplicate_g_is_rejected(ctx):
    from paper_1111_4429_gb300 import bgw
    s = _sys()
    gv = s.gv.copy()
    gv[1] = gv[0]
    with pytest.raises(bgw.BgwError):
        _run(ctx, s, gv=gv)


def test_unsupported_grid_is_reported(ctx):
    from paper_1111_4429_gb300 import bgw
    s = _sys()
    with pytest.raises(bgw.BgwError) as e:
        _run(ctx, s, n=14)
    assert e.value.code == bgw.BGW_EUNSUPPORTED


def test_energy_order_and_gap_are_checked(ctx):
    from paper_1111_4429_gb300 import bgw
    s = _sys()
    M = _run(ctx, s)
    chi = torch.zeros((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    cell = bgw.system_cell(s)
    with pytest.raises(bgw.BgwError):
        ctx.chi_sum(cell, s.nv, s.nc, s.ng, M, s.ev[::-1].copy(), s.ec, None, 0, False, chi)
    ec = s.ec.copy()
    ec[0] = s.ev[-1]        # Delta = 0
    with pytest.raises(bgw.BgwError):
        ctx.chi_sum(cell, s.nv, s.nc, s.ng, M, s.ev, ec, None, 0, False, chi)
    ctx.sync()


def test_q_plus_g_zero_is_rejected(ctx):
    from paper_1111_4429_gb300 import bgw
    s = _sys()
    cell = bgw.make_cell(s.bvec, s.omega, (0.0, 0.0, 0.0), s.fft)
    geps = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.int32)
    chi = torch.zeros((2, 2), dtype=torch.complex128, device="cuda")
    inv = torch.zeros_like(chi)
    with pytest.raises(bgw.BgwError) as e:
        ctx.epsinv([cell], [geps], [chi], None, [inv])
    assert e.value.code == bgw.BGW_EINVAL


def test_zero_pivot_sets_numeric_status(ctx):
    # chi chosen so that eps~ = 0 on the diagonal block: the inversion must
    # report BGW_ENUMERIC through bgw_sync (no fault, no hang).
    from paper_1111_4429_gb300 import bgw, synth as sy
    s = _sys()
    cell = bgw.system_cell(s)
    geps = s.geps[:2]
    import oracle
    v = oracle.coulomb(s.bvec, s.q_frac, geps)
    chi = torch.from_numpy(np.diag(1.0 / v).astype(np.complex128)).cuda()   # eps~ = I - I = 0
    inv = torch.zeros_like(chi)
    ctx.epsinv([cell], [geps], [chi], None, [inv])
    with pytest.raises(bgw.BgwError) as e:
        ctx.sync()
    assert e.value.code == bgw.BGW_ENUMERIC
    ctx.sync()   # status was cleared


def test_chi_wait_limit_reports_timeout_and_context_recovers(ctx):
    """With a wait limit of 0, every wait of the tensor-core chi kernels that
    is not already complete gives up (a TMA copy cannot land before the MMA
    issuer's first look): each CTA lets its copies and MMAs in flight finish,
    frees its tensor memory and returns, and bgw_sync reports BGW_ETIMEOUT.
    The context and the GPU stay usable: the same call with the default
    limit then gives the oracle's chi."""
    from paper_1111_4429_gb300 import bgw
    import oracle
    # K = 5400 pairs: several 512-pair segments per CTA
    s = synth.make_system("k", a=14.0, fft=24, ecut_wfn=8.0, ecut_eps=2.0, nv=6, nc=900, seed=55)
    cell = bgw.system_cell(s)
    M = torch.empty((s.npairs, s.ng), dtype=torch.complex64, device="cuda")
    ctx.mtxel(cell, s.gv, torch.from_numpy(s.cv).cuda(), s.gc, torch.from_numpy(s.cc).cuda(), s.geps,
              bgw.BGW_PREC_MIX_FP16, M)
    chi = torch.zeros((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    ctx.sync()
    ctx.set_option(bgw.BGW_OPT_WAIT_LIMIT_NS, 0)
    try:
        ctx.chi_sum(cell, s.nv, s.nc, s.ng, M, s.ev, s.ec, None, bgw.BGW_PREC_MIX_FP16, False, chi)
        with pytest.raises(bgw.BgwError) as e:
            ctx.sync()
        assert e.value.code == bgw.BGW_ETIMEOUT
    finally:
        ctx.set_option(bgw.BGW_OPT_WAIT_LIMIT_NS, 10 ** 9)
    ctx.sync()   # status was cleared
    ctx.chi_sum(cell, s.nv, s.nc, s.ng, M, s.ev, s.ec, None, bgw.BGW_PREC_MIX_FP16, False, chi)
    ctx.sync()
    m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    want = oracle.chi(m, oracle.chi_weights(s.ev, s.ec), s.omega)
    got = chi[0].cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-5


@pytest.mark.parametrize("option,bad,good", [("BGW_OPT_WAIT_LIMIT_NS", [-1, 10 ** 10 + 1], [10 ** 9, 0, 10 ** 10]),
                                             ("BGW_OPT_UPDATE_SLICES", [1, 6, 8, -1], [0, 5, 7]),
                                             ("BGW_OPT_DOUBLE_FP32", [2, -2], [-1, 0, 1]),
                                             ("BGW_OPT_SIGMA_DENSITY", [2, -2], [-1, 0, 1]),
                                             ("BGW_OPT_INVERSE", [2, -2], [-1, 0, 1]),
                                             ("BGW_OPT_PAIR_KERNEL", [-2, 2, 11], [-1, 0, 1]),
                                             ("BGW_OPT_UPDATE_ITEMS", [-2, 2, 4], [-1, 0, 1])])
def test_option_values(ctx, option, bad, good):
    """Values outside an option's documented set are refused (code 1) and
    leave the context usable; the documented ones are accepted."""
    from paper_1111_4429_gb300 import bgw
    opt = getattr(bgw, option)
    for v in bad:
        with pytest.raises(bgw.BgwError) as ex:
            ctx.set_option(opt, v)
        assert ex.value.code == 1
    for v in good:
        ctx.set_option(opt, v)
    ctx.set_option(opt, good[0])   # back to the default (first listed)
