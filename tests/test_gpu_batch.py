"""Batched q-points x imaginary frequencies (bgw_epsilon_batch): uneven
epsilon spheres, matrix elements computed once per q-point, batched inverses,
and the CUDA-graph replay of a repeated argument set."""
import numpy as np
import pytest

import oracle
from paper_1111_4429_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4429_gb300 import bgw
    return bgw.Context(0)


def _systems():
    # three q-points of one cell: different q shifts give different N_G
    return [synth.make_system(f"b{j}", a=14.0, fft=24, ecut_wfn=6.0, ecut_eps=2.5, nv=5, nc=37, seed=300 + j,
                              q_frac=(0.1 * j, 0.05 * j, 0.0)) for j in (1, 2, 3)]


def _oracle(s, om):
    m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    v = oracle.coulomb(s.bvec, s.q_frac, s.geps)
    out = []
    for w in (om if om is not None else [None]):
        x = oracle.chi(m, oracle.chi_weights(s.ev, s.ec, w), s.omega)
        out.append(oracle.epsinv_sym(x, v)[1])
    return out


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_batch_vs_oracle_uneven_spheres(ctx, prec, tol):
    systems = _systems()
    assert len({s.ng for s in systems}) > 1
    om = synth.gauss_legendre_frequencies(3)
    cvs = [torch.from_numpy(s.cv).cuda() for s in systems]
    ccs = [torch.from_numpy(s.cc).cuda() for s in systems]
    outs = [torch.zeros((3, s.ng, s.ng), dtype=torch.complex128, device="cuda") for s in systems]
    ctx.epsilon_batch(systems, cvs, ccs, om, prec, outs)
    ctx.sync()
    for s, o in zip(systems, outs):
        ref = _oracle(s, om)
        for f in range(3):
            assert _rel(o[f].cpu().numpy(), ref[f]) <= tol


def test_batch_graph_replay_and_fresh_inputs(ctx):
    systems = _systems()
    st = torch.cuda.Stream()
    cvs = [torch.from_numpy(s.cv).cuda() for s in systems]
    ccs = [torch.from_numpy(s.cc).cuda() for s in systems]
    outs = [torch.zeros((2, s.ng, s.ng), dtype=torch.complex128, device="cuda") for s in systems]
    om = np.array([0.0, 0.7])
    with torch.cuda.stream(st):
        l0 = ctx.launch_count()
        ctx.epsilon_batch(systems, cvs, ccs, om, 1, outs, stream=st)   # direct run + capture
        st.synchronize()
        direct = ctx.launch_count() - l0
        first = [o.clone() for o in outs]
        for o in outs:
            o.zero_()
        l0 = ctx.launch_count()
        ctx.epsilon_batch(systems, cvs, ccs, om, 1, outs, stream=st)   # graph replay
        st.synchronize()
        # a replay counts the kernels its graph holds: those of one direct pass
        # (less the autotuner's trial launches of the first call)
        assert 0 < ctx.launch_count() - l0 <= direct
        for a, b in zip(first, outs):
            assert torch.equal(a, b)
        # new device contents under the same graph: swap in other coefficients
        other = [synth.make_system("o", a=14.0, fft=24, ecut_wfn=6.0, ecut_eps=2.5, nv=5, nc=37, seed=400 + j,
                                   q_frac=s.q_frac) for j, s in enumerate(systems)]
        for k, o in enumerate(other):
            cvs[k].copy_(torch.from_numpy(o.cv))
            ccs[k].copy_(torch.from_numpy(o.cc))
        ctx.epsilon_batch(systems, cvs, ccs, om, 1, outs, stream=st)
        st.synchronize()
    ctx.sync(st)
    for s, o, out in zip(systems, other, outs):
        o.ev, o.ec = s.ev, s.ec      # the graph keeps the first call's energies
        ref = _oracle(o, om)
        for f in range(2):
            assert _rel(out[f].cpu().numpy(), ref[f]) <= 1e-6


@pytest.mark.parametrize("nc_chunk", [0, 25])
def test_epsilon_host_buffers_graph_replay(ctx, nc_chunk):
    """bgw_epsilon with page-locked host buffers on a capturable stream: the
    second call replays a graph of the whole path (copies included); new
    host coefficients in the same buffers give the direct result bit for bit.
    With conduction chunks (25 of 60 bands) the chunk copies run on the
    context's copy stream, one chunk ahead, inside the graph as well."""
    from paper_1111_4429_gb300 import bgw
    s = synth.config_system("c0")
    cell = bgw.system_cell(s)
    cvh = torch.from_numpy(s.cv).pin_memory()
    cch = torch.from_numpy(s.cc).pin_memory()
    out = torch.empty((1, s.ng, s.ng), dtype=torch.complex128).pin_memory()
    st = torch.cuda.Stream()
    res = []
    g0 = ctx.graph_stats()
    with torch.cuda.stream(st):
        for k in range(3):
            if k == 2:   # new contents, same buffers: scrambled phases of the same bands
                cvh.mul_(torch.exp(1j * torch.arange(cvh.shape[0], dtype=torch.float64))[:, None])
            l0 = ctx.launch_count()
            ctx.epsilon(cell, s.gv, cvh, s.ev, s.gc, cch, s.ec, s.geps, None, 1, nc_chunk, None, out)
            res.append((out.clone(), ctx.launch_count() - l0))
    ctx.set_option(bgw.BGW_OPT_TIMING, 1)   # timing on: direct runs
    try:
        with torch.cuda.stream(st):
            ctx.epsilon(cell, s.gv, cvh, s.ev, s.gc, cch, s.ec, s.geps, None, 1, nc_chunk, None, out)
            direct = out.clone()
    finally:
        ctx.set_option(bgw.BGW_OPT_TIMING, 0)
    g1 = ctx.graph_stats()
    assert g1[0] == g0[0] + 1 and g1[1] == g0[1] + 2   # one graph, replayed by the second and third calls
    assert torch.equal(res[0][0], res[1][0])
    assert torch.equal(res[2][0], direct)
    assert res[1][1] > 0
    # a band phase does not change chi: the result stays that of the first inputs up to rounding
    assert float((res[2][0] - res[0][0]).abs().max()) <= 1e-6 * float(res[0][0].abs().max())
