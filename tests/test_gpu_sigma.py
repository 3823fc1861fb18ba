"""Diagonal static COHSEX and bare exchange (bgw_sigma_cohsex) on the GPU
against the FP64 oracle.  Bar: 1e-12 of the largest magnitude of each
quantity (FP64 throughout)."""
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
