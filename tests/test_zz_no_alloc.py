"""bgw_epsinv_noalloc: the inverse for callers that cannot allocate device
memory (their own allocator already holds the GPU's memory, or an allocation's
synchronization is not acceptable).  Its scratch is a fixed array inside the
library.  Checked through the C ABI against bgw_epsinv and against the FP64
oracle on two calls in a row with different sizes, so a stale scratch from
the first call would show; a size above the array's limit must be refused
before anything is written.  Collected last on purpose: it must pass alone in
a fresh process and after every other test.
"""
import numpy as np
import pytest

import oracle
from paper_1111_4429_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
MAX_NG = 4096


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_inverse_matches_epsinv_and_oracle_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4429_gb300 import bgw
    systems = [synth.make_system("na1", a=14.0, fft=24, ecut_wfn=6.0, ecut_eps=2.5, nv=5, nc=37, seed=91),
               synth.config_system("c0")]
    ctx = bgw.Context(0)
    for s in systems:
        cell = bgw.system_cell(s)
        ref = oracle.solve(s)
        chi = torch.from_numpy(ref["chi"]).cuda()
        ref_inv = torch.empty_like(chi)
        ref_eps = torch.empty_like(chi)
        ctx.epsinv([cell], [s.geps], [chi], [ref_eps], [ref_inv])
        ctx.sync()
        inv = torch.full_like(chi, float("nan"))
        eps = torch.full_like(chi, float("nan"))
        bgw.epsinv_noalloc(cell, s.geps, chi, eps, inv)
        torch.cuda.synchronize()
        got_inv, got_eps = inv.cpu().numpy(), eps.cpu().numpy()
        assert _rel(got_inv, ref_inv.cpu().numpy()) <= TOL64
        assert _rel(got_eps, ref_eps.cpu().numpy()) <= TOL64
        assert _rel(got_inv, ref["epsinv"]) <= TOL64
        assert _rel(got_eps, ref["eps"]) <= TOL64
    assert systems[0].ng != systems[1].ng


def test_noalloc_refuses_ng_above_its_scratch_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4429_gb300 import bgw
    s = synth.config_system("c1")
    geps = synth.gsphere(s.bvec, s.q_frac, 10.0)[:MAX_NG + 1]
    assert geps.shape[0] == MAX_NG + 1
    ng = geps.shape[0]
    chi = torch.zeros((ng, ng), dtype=torch.complex128, device="cuda")
    inv = torch.full_like(chi, float("nan"))
    with pytest.raises(bgw.BgwError) as e:
        bgw.epsinv_noalloc(bgw.system_cell(s), geps, chi, None, inv)
    assert e.value.code == bgw.BGW_EINVAL
    torch.cuda.synchronize()
    assert bool(torch.isnan(inv).all())    # nothing was written
