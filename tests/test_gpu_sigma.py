"""Diagonal static COHSEX and bare exchange (bgw_sigma_cohsex) on the GPU
against the FP64 oracle.  Bar: 1e-12 of the largest magnitude of each
quantity (FP64 throughout).

Mixed precisions: m comes from FP32 FFTs (relative error a few 2^-24 of the
largest |m|) and W m from hi/lo split operands on the tensor cores (FP16
hi/lo keep 22 bits, BF16 hi/lo 16 bits, of each operand's largest
element).  The quadratic forms then carry about 1e-6 (FP16) or 1e-5 (BF16)
of max|W| max|m|^2 per term; the bars are 2e-6 and 2e-5 of each quantity's
largest magnitude.  The bare exchange uses no tensor cores: its bar is the
FP32 m's, 1e-6."""
import math

import numpy as np
import pytest

import oracle
from paper_1111_4429_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("X", "SX", "CH", "CH_exact")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4429_gb300 import bgw
    return bgw.Context(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(got, ref, tol=1e-12):
    for k, key in enumerate(KEYS):
        r = np.real(ref[key])
        assert np.abs(got[k] - r).max() <= tol * max(np.abs(r).max(), 1e-300), key


@pytest.mark.parametrize("no,ni,nocc", [(3, 40, 4), (5, 70, 9), (1, 1, 1)])
def test_sigma_c0_vs_oracle(ctx, no, ni, nocc):
    from paper_1111_4429_gb300 import bgw
    s = synth.config_system("c0")
    r = oracle.solve(s)
    sb = synth.sigma_bands(s, no, ni, nocc, seed=11 + ni)
    got = ctx.sigma_cohsex(bgw.system_cell(s), sb.go, _dev(sb.co), sb.gi, _dev(sb.ci), nocc, s.geps,
                           _dev(r["epsinv"]))
    ref = oracle.sigma_cohsex(sb.gi, sb.ci, nocc, sb.go, sb.co, s.geps, r["epsinv"], r["v"], s.omega)
    _check(got, ref)


def test_sigma_from_gpu_epsinv_and_unscreened_limit(ctx):
    from paper_1111_4429_gb300 import bgw
    s = synth.make_system("r", a=14.0, fft=24, ecut_wfn=6.0, ecut_eps=2.5, nv=5, nc=37, seed=61)
    cell = bgw.system_cell(s)
    inv = torch.zeros((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    ctx.epsilon(cell, s.gv, _dev(s.cv), s.ev, s.gc, _dev(s.cc), s.ec, s.geps, None, 0, 0, None, inv)
    ctx.sync()
    sb = synth.sigma_bands(s, 4, 90, 5, seed=3)       # ng = 231: four column tiles, ragged
    got = ctx.sigma_cohsex(cell, sb.go, _dev(sb.co), sb.gi, _dev(sb.ci), 5, s.geps, inv[0])
    r = oracle.solve(s)
    ref = oracle.sigma_cohsex(sb.gi, sb.ci, 5, sb.go, sb.co, s.geps, r["epsinv"], r["v"], s.omega)
    _check(got, ref, 1e-11)
    eye = torch.eye(s.ng, dtype=torch.complex128, device="cuda")
    got = ctx.sigma_cohsex(cell, sb.go, _dev(sb.co), sb.gi, _dev(sb.ci), 5, s.geps, eye)
    assert np.allclose(got[1], got[0], rtol=1e-13, atol=0)          # W = V: SX is the bare exchange
    assert np.abs(got[2:]).max() <= 1e-15


def test_sigma_closed_form_is_the_sum_over_a_complete_inner_basis(ctx):
    from paper_1111_4429_gb300 import bgw
    s = synth.make_system("sg", a=8.0, fft=16, ecut_wfn=2.0, ecut_eps=1.0, nv=2, nc=4, seed=3)
    gen = np.random.default_rng(3)
    go = s.gc
    co = synth.orthonormal_bands(gen, go.shape[0], 3)
    gi = synth.gsphere(s.bvec, -np.asarray(s.q_frac), (math.sqrt(2.0) + 1.0) ** 2 + 1e-9)
    ci = np.eye(gi.shape[0], dtype=np.complex128)
    z = gen.standard_normal((s.ng, s.ng)) + 1j * gen.standard_normal((s.ng, s.ng))
    ei = np.eye(s.ng) + 0.1 * (z + np.conj(z).T)
    got = ctx.sigma_cohsex(bgw.system_cell(s), go, _dev(co), gi, _dev(ci), 0, s.geps, _dev(ei))
    assert np.abs(got[2] - got[3]).max() <= 1e-12 * np.abs(got[3]).max()


@pytest.mark.parametrize("prec,tol", [(1, 2e-6), (2, 2e-5)])
@pytest.mark.parametrize("no,ni,nocc", [(3, 40, 4), (4, 150, 9)])
def test_sigma_mixed_vs_oracle(ctx, prec, tol, no, ni, nocc):
    from paper_1111_4429_gb300 import bgw
    s = synth.make_system("r", a=14.0, fft=24, ecut_wfn=6.0, ecut_eps=2.5, nv=5, nc=37, seed=61)
    r = oracle.solve(s)
    sb = synth.sigma_bands(s, no, ni, nocc, seed=5 + ni)   # K = ni no pairs: several row tiles at ni = 150
    got = ctx.sigma_cohsex(bgw.system_cell(s), sb.go, _dev(sb.co), sb.gi, _dev(sb.ci), nocc, s.geps,
                           _dev(r["epsinv"]), prec=prec)
    ref = oracle.sigma_cohsex(sb.gi, sb.ci, nocc, sb.go, sb.co, s.geps, r["epsinv"], r["v"], s.omega)
    for k, key in enumerate(KEYS):
        rr = np.real(ref[key])
        bar = (1e-6 if key == "X" else tol) * np.abs(rr).max()
        assert np.abs(got[k] - rr).max() <= bar, (key, np.abs(got[k] - rr).max() / np.abs(rr).max())


def test_sigma_mixed_matches_fp64_path(ctx):
    """The mixed and plain paths on a GPU-made eps~^-1 agree to the FP16 bar."""
    from paper_1111_4429_gb300 import bgw
    s = synth.config_system("c0")
    cell = bgw.system_cell(s)
    inv = torch.zeros((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    ctx.epsilon(cell, s.gv, _dev(s.cv), s.ev, s.gc, _dev(s.cc), s.ec, s.geps, None, 0, 0, None, inv)
    ctx.sync()
    sb = synth.sigma_bands(s, 2, 33, 3, seed=9)   # K = 66: one ragged row tile
    a = ctx.sigma_cohsex(cell, sb.go, _dev(sb.co), sb.gi, _dev(sb.ci), 3, s.geps, inv[0])
    b = ctx.sigma_cohsex(cell, sb.go, _dev(sb.co), sb.gi, _dev(sb.ci), 3, s.geps, inv[0], prec=1)
    for k in range(4):
        assert np.abs(a[k] - b[k]).max() <= 2e-6 * np.abs(a[k]).max()


def test_sigma_density_routes_agree(ctx):
    """The band densities of the closed form by the product transform (default)
    and by the direct sum over the sphere give the same CH_exact."""
    from paper_1111_4429_gb300 import bgw
    s = synth.config_system("c0")
    r = oracle.solve(s)
    sb = synth.sigma_bands(s, 11, 30, 4, seed=21)       # two chunks of bands
    args = (bgw.system_cell(s), sb.go, _dev(sb.co), sb.gi, _dev(sb.ci), 4, s.geps, _dev(r["epsinv"]))
    a = ctx.sigma_cohsex(*args)
    ctx.set_option(bgw.BGW_OPT_SIGMA_DENSITY, 0)
    try:
        b = ctx.sigma_cohsex(*args)
    finally:
        ctx.set_option(bgw.BGW_OPT_SIGMA_DENSITY, -1)
    assert np.array_equal(a[:3], b[:3])
    assert np.abs(a[3] - b[3]).max() <= 1e-12 * np.abs(b[3]).max()
    ref = oracle.sigma_cohsex(sb.gi, sb.ci, 4, sb.go, sb.co, s.geps, r["epsinv"], r["v"], s.omega)
    assert np.abs(a[3] - np.real(ref["CH_exact"])).max() <= 1e-12 * np.abs(np.real(ref["CH_exact"])).max()


def test_sigma_density_routes_agree_c1_box(ctx):
    """c1 geometry (N_G = 2120): the difference box holds 33^3 points, more
    than a shared-memory row of the product transform, so its z pass writes
    straight to memory.  The two density routes agree on CH_exact."""
    from paper_1111_4429_gb300 import bgw
    s = synth.config_system("c1")
    gen = np.random.default_rng(4)
    z = gen.standard_normal((s.ng, s.ng)) + 1j * gen.standard_normal((s.ng, s.ng))
    ei = _dev(np.eye(s.ng) + 0.01 * (z + np.conj(z).T))
    sb = synth.sigma_bands(s, 3, 4, 2, seed=8)
    args = (bgw.system_cell(s), sb.go, _dev(sb.co), sb.gi, _dev(sb.ci), 2, s.geps, ei)
    a = ctx.sigma_cohsex(*args)
    ctx.set_option(bgw.BGW_OPT_SIGMA_DENSITY, 0)
    try:
        b = ctx.sigma_cohsex(*args)
    finally:
        ctx.set_option(bgw.BGW_OPT_SIGMA_DENSITY, -1)
    assert np.abs(a[3] - b[3]).max() <= 1e-12 * np.abs(b[3]).max()


def test_sigma_argument_errors(ctx):
    from paper_1111_4429_gb300 import bgw
    s = synth.config_system("c0")
    sb = synth.sigma_bands(s, 2, 10, 2, seed=1)
    e = torch.eye(s.ng, dtype=torch.complex128, device="cuda")
    with pytest.raises(bgw.BgwError) as ex:
        ctx.sigma_cohsex(bgw.system_cell(s), sb.go, _dev(sb.co), sb.gi, _dev(sb.ci), 11, s.geps, e)
    assert ex.value.code == 1
    with pytest.raises(bgw.BgwError) as ex:
        ctx.sigma_cohsex(bgw.system_cell(s), sb.go, sb.co, sb.gi, _dev(sb.ci), 2, s.geps, e)
    assert ex.value.code == 1 and "device" in str(ex.value)
