"""Mixed-precision path against the FP64 oracle.

M in complex64 (FP32 FFTs); chi from split-precision products on the tensor
cores (FP16 hi/lo with a power-of-two scale, or BF16 hi/lo) accumulated in
FP32 per segment of pairs and summed in FP64; eps~ and its inverse in FP64.
Bar: eps~^-1 within 1e-6 relative Frobenius of the oracle (FP16 split).  The
chi error is reported and held to 1e-5: single-precision FFTs leave M with a
relative error near 1e-6, which chi carries twice.  BF16 splits carry about
16 significant bits per value, so their bars are 3e-5 on chi and 1e-5 on
eps~^-1.
"""
import numpy as np
import pytest

import oracle
from paper_1111_4429_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {1: (1e-5, 1e-6), 2: (3e-5, 1e-5)}   # prec -> (chi, epsinv)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4429_gb300 import bgw
    return bgw.Context(0)


def _run(ctx, s, prec, omega=None, chunks=None):
    from paper_1111_4429_gb300 import bgw
    cell = bgw.system_cell(s)
    nrow = 1 if omega is None else len(omega)
    M = torch.empty((s.nv * s.nc, s.ng), dtype=torch.complex64, device="cuda")
    ctx.mtxel(cell, s.gv, torch.from_numpy(s.cv).cuda(), s.gc, torch.from_numpy(s.cc).cuda(), s.geps, prec, M)
    chi = torch.zeros((nrow, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    if chunks is None:
        ctx.chi_sum(cell, s.nv, s.nc, s.ng, M, s.ev, s.ec, omega, prec, False, chi)
    else:
        Mv = M.view(s.nv, s.nc, s.ng)
        for k, (c0, c1) in enumerate(chunks):
            Mc = Mv[:, c0:c1].contiguous().view(-1, s.ng)
            ctx.chi_sum(cell, s.nv, c1 - c0, s.ng, Mc, s.ev, s.ec[c0:c1], omega, prec, k > 0, chi)
    inv = torch.empty_like(chi)
    ctx.epsinv([cell] * nrow, [s.geps] * nrow, [chi[f] for f in range(nrow)], None, [inv[f] for f in range(nrow)])
    ctx.sync()
    _run.last_M = M
    return chi.cpu().numpy(), inv.cpu().numpy()


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_c0_vs_oracle(ctx, prec):
    s = synth.config_system("c0")
    r = oracle.solve(s)
    chi, inv = _run(ctx, s, prec)
    tchi, tinv = TOL[prec]
    assert _rel(chi[0], r["chi"]) <= tchi
    assert _rel(inv[0], r["epsinv"]) <= tinv
    assert np.array_equal(chi[0], np.conj(chi[0]).T)


def test_mixed_ragged_tiles_chunks_and_frequencies(ctx):
    # ng = 231: two 128-row tiles, ragged; conduction streamed in three chunks
    s = synth.make_system("r", a=14.0, fft=24, ecut_wfn=6.0, ecut_eps=2.5, nv=5, nc=37, seed=77)
    om = np.concatenate([[0.0], synth.gauss_legendre_frequencies(2)])
    chi, inv = _run(ctx, s, 1, omega=om, chunks=[(0, 10), (10, 11), (11, 37)])
    m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    v = oracle.coulomb(s.bvec, s.q_frac, s.geps)
    for f, w in enumerate(om):
        x = oracle.chi(m, oracle.chi_weights(s.ev, s.ec, w), s.omega)
        _, ei = oracle.epsinv_sym(x, v)
        assert _rel(chi[f], x) <= 1e-5
        assert _rel(inv[f], ei) <= 1e-6


def test_mixed_multi_segment_k(ctx):
    # K = 6 x 900 = 5400 pairs > one 4096-pair segment: FP32 partials of two
    # segments summed in FP64
    s = synth.make_system("k", a=14.0, fft=24, ecut_wfn=8.0, ecut_eps=2.0, nv=6, nc=900, seed=55)
    r = oracle.solve(s)
    chi, inv = _run(ctx, s, 1)
    assert s.npairs > 4096
    assert _rel(chi[0], r["chi"]) <= 1e-5
    assert _rel(inv[0], r["epsinv"]) <= 1e-6


@pytest.mark.parametrize("seg", [32, 4096])
def test_mixed_segment_option(ctx, seg):
    from paper_1111_4429_gb300 import bgw
    s = synth.make_system("k", a=14.0, fft=24, ecut_wfn=8.0, ecut_eps=2.0, nv=6, nc=900, seed=56)
    r = oracle.solve(s)
    ctx.set_option(bgw.BGW_OPT_CHI_SEGMENT_PAIRS, seg)
    try:
        chi, inv = _run(ctx, s, 1)
    finally:
        ctx.set_option(bgw.BGW_OPT_CHI_SEGMENT_PAIRS, 0)
    e_chi, e_inv = _rel(chi[0], r["chi"]), _rel(inv[0], r["epsinv"])
    print(f"segment {seg}: chi {e_chi:.3e} epsinv {e_inv:.3e}")
    assert e_chi <= 1e-4 and e_inv <= 1e-5


@pytest.mark.parametrize("chunk", [1000, 3000])
def test_mixed_pair_chunks(ctx, chunk):
    # K = 5400 pairs summed in chunks of 992 / 2976 pairs (ragged last chunk)
    from paper_1111_4429_gb300 import bgw
    s = synth.make_system("k", a=14.0, fft=24, ecut_wfn=8.0, ecut_eps=2.0, nv=6, nc=900, seed=57)
    r = oracle.solve(s)
    ctx.set_option(bgw.BGW_OPT_CHI_CHUNK_PAIRS, chunk)
    try:
        chi, inv = _run(ctx, s, 1, omega=np.array([0.0, 0.5]))
    finally:
        ctx.set_option(bgw.BGW_OPT_CHI_CHUNK_PAIRS, 0)
    m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    v = oracle.coulomb(s.bvec, s.q_frac, s.geps)
    for f, w in enumerate([0.0, 0.5]):
        x = oracle.chi(m, oracle.chi_weights(s.ev, s.ec, w), s.omega)
        assert _rel(chi[f], x) <= 1e-5
        assert _rel(inv[f], oracle.epsinv_sym(x, v)[1]) <= 1e-6


def test_mixed_c1_full_size_vs_oracle(ctx):
    """c1 at full size (N_G = 2120, K = 25,600) in mixed precision against the
    full FP64 oracle solve."""
    s = synth.config_system("c1")
    r = oracle.solve(s)
    chi, inv = _run(ctx, s, 1)
    e_chi, e_inv = _rel(chi[0], r["chi"]), _rel(inv[0], r["epsinv"])
    e_m = _rel(_run.last_M.cpu().numpy().astype(np.complex128), r["M"])
    print(f"c1 mixed: M rel err {e_m:.3e}, chi rel err {e_chi:.3e}, epsinv rel err {e_inv:.3e}")
    assert e_chi <= 1e-5
    assert e_inv <= 1e-6
