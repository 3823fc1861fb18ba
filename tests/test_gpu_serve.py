"""Serving (bgw_serve_*): requests of different sizes in flight together give
the same eps~^-1 as each request run alone, within the mixed-precision
tolerance; admission by budget, cancellation and polling time-outs."""
import time

import numpy as np
import pytest

import oracle
from paper_1111_4429_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _requests():
    out = []
    for k, (a, n, ew, ee, nv, nc) in enumerate([(10.26, 20, 10.0, 3.0, 4, 60), (14.0, 24, 6.0, 2.5, 5, 37),
                                                 (10.26, 20, 10.0, 4.0, 4, 120), (20.52, 40, 10.0, 3.0, 8, 200),
                                                 (12.0, 20, 5.0, 3.3, 3, 20), (14.0, 24, 8.0, 2.0, 6, 300)]):
        out.append(synth.make_system(f"r{k}", a=a, fft=n, ecut_wfn=ew, ecut_eps=ee, nv=nv, nc=nc, seed=500 + k))
    return out


def _alone(s, prec):
    from paper_1111_4429_gb300 import bgw
    ctx = bgw.Context(0)
    inv = np.zeros((1, s.ng, s.ng), dtype=np.complex128)
    ctx.epsilon(bgw.system_cell(s), s.gv, s.cv, s.ev, s.gc, s.cc, s.ec, s.geps, None, prec, 0, None, inv)
    ctx.close()
    return inv[0]


def test_served_mix_matches_alone_and_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4429_gb300 import bgw
    reqs = _requests()
    srv = bgw.Server(bgw.Context(0), hbm_budget_bytes=64 << 30, max_slots=3, prec=bgw.BGW_PREC_MIX_FP16)
    outs = [np.zeros((s.ng, s.ng), dtype=np.complex128) for s in reqs]
    pinned = [torch.zeros((s.ng, s.ng), dtype=torch.complex128).pin_memory() for s in reqs[:2]]
    tickets = []
    for k, s in enumerate(reqs):
        tickets.append(srv.submit(s, pinned[k] if k < 2 else outs[k]))
        time.sleep(0.002 * (k % 3))
    results = [srv.poll(t, timeout_ms=120000) for t in tickets]
    srv.close()
    for k, (s, r) in enumerate(zip(reqs, results)):
        assert r is not None and r["status"] == 0, r
        assert r["latency_ms"] >= r["queue_ms"] >= 0.0
        got = pinned[k].numpy() if k < 2 else outs[k]
        alone = _alone(s, bgw.BGW_PREC_MIX_FP16)
        assert _rel(got, alone) <= 1e-6
        if s.npairs <= 2000:
            assert _rel(got, oracle.solve(s)["epsinv"]) <= 1e-6


def test_over_budget_request_is_refused_and_queue_cancel():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4429_gb300 import bgw
    small = synth.config_system("c0")
    big = synth.make_system("big", a=20.52, fft=40, ecut_wfn=10.0, ecut_eps=3.0, nv=8, nc=400, seed=9)
    srv = bgw.Server(bgw.Context(0), hbm_budget_bytes=256 << 20, max_slots=1, prec=bgw.BGW_PREC_MIX_FP16)
    o1 = np.zeros((big.ng, big.ng), dtype=np.complex128)
    t_big = srv.submit(big, o1)                 # estimate far above 256 MiB
    r = srv.poll(t_big, timeout_ms=60000)
    assert r["status"] == bgw.BGW_ENOMEM
    srv.close()

    srv = bgw.Server(bgw.Context(0), hbm_budget_bytes=0, max_slots=1, prec=bgw.BGW_PREC_MIX_FP16)
    outs = [np.zeros((small.ng, small.ng), dtype=np.complex128) for _ in range(4)]
    o_big = np.zeros((big.ng, big.ng), dtype=np.complex128)
    t0 = srv.submit(big, o_big)                 # occupies the only slot
    ts = [srv.submit(small, o) for o in outs]
    rc = srv.cancel(ts[-1])                     # still queued behind the big request
    assert rc in (bgw.BGW_OK, bgw.BGW_EBUSY)
    first = srv.poll(t0, timeout_ms=0)          # pending (None) or already done
    done = {t0: first} if first is not None else {}
    for t in [t0] + ts:
        if t not in done:
            done[t] = srv.poll(t, timeout_ms=120000)
    srv.close()
    assert done[t0]["status"] == 0
    for t in ts[:-1]:
        assert done[t]["status"] == 0
    if rc == bgw.BGW_OK:
        assert done[ts[-1]]["status"] == bgw.BGW_ECANCELED
    ref = _alone(small, bgw.BGW_PREC_MIX_FP16)
    assert _rel(outs[1], ref) <= 1e-6
