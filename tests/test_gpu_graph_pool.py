"""Scratch blocks of a captured CUDA graph and the context's cached uploads.

A graph captured by bgw_epsinv keeps writing the pool blocks it used at every
replay.  Those blocks go back to the pool's free list after the capture, where
a later call's scratch may take them (stream order puts that use after the
replays), but an input cached for the context's life must never land in one:
the next replay would overwrite it and every later call that hits the cache
would read garbage.  The test captures an inverse, uploads new energies
through bgw_chi_sum, replays the inverse, and repeats the chi call, which now
reads the cached energies: chi must still equal the oracle's."""
import numpy as np
import pytest

import oracle
from paper_1111_4429_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_cached_upload_survives_graph_replay():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4429_gb300 import bgw
    s = synth.config_system("c0")
    cell = bgw.system_cell(s)
    ctx = bgw.Context(0)
    m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    ev2 = s.ev - 0.125                      # new energies: a new upload
    want = oracle.chi(m, oracle.chi_weights(ev2, s.ec), s.omega)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        M = torch.from_numpy(m).cuda()
        chi = torch.zeros((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
        inv = torch.empty_like(chi)
        ctx.chi_sum(cell, s.nv, s.nc, s.ng, M, s.ev, s.ec, None, bgw.BGW_PREC_FP64, False, chi)
        ctx.epsinv([cell], [s.geps], [chi[0]], None, [inv[0]])   # direct run, then captured
        g0, r0 = ctx.graph_stats()
        chi2 = torch.zeros_like(chi)
        ctx.chi_sum(cell, s.nv, s.nc, s.ng, M, ev2, s.ec, None, bgw.BGW_PREC_FP64, False, chi2)
        ctx.epsinv([cell], [s.geps], [chi[0]], None, [inv[0]])   # replay
        g1, r1 = ctx.graph_stats()
        chi3 = torch.zeros_like(chi)
        ctx.chi_sum(cell, s.nv, s.nc, s.ng, M, ev2, s.ec, None, bgw.BGW_PREC_FP64, False, chi3)  # cached ev2
        ctx.sync(st)
    assert g0 >= 1 and r1 == r0 + 1, "the second inverse must replay the captured graph"
    assert _rel(chi2[0].cpu().numpy(), want) <= 1e-12
    assert _rel(chi3[0].cpu().numpy(), want) <= 1e-12
