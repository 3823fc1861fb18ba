"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Bar (plain FP64 path): relative Frobenius error <= 1e-12 for M, chi, eps~ and
eps~^-1 against the oracle on the same seeded inputs.  The FP32 matrix
elements of the mixed path are held to 1e-5 (single-precision FFTs of
length <= 64: a few units of 2^-24 per stage, times the data's dynamic range).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1111_4429_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_M = 1e-5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_4429_gb300 import bgw
    return bgw.Context(0)


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _mtxel(ctx, s, prec=0):
    from paper_1111_4429_gb300 import bgw
    cdt = torch.complex128 if prec == 0 else torch.complex64
    M = torch.empty((s.nv * s.nc, s.ng), dtype=cdt, device="cuda")
    ctx.mtxel(bgw.system_cell(s), s.gv, _dev(s.cv), s.gc, _dev(s.cc), s.geps, prec, M)
    ctx.sync()
    return M


def _tiny(seed, n=12, a=8.0, ew=4.0, ee=1.5, nv=3, nc=5, q=(0.1, 0.0, 0.0)):
    return synth.make_system("t", a=a, fft=n, ecut_wfn=ew, ecut_eps=ee, nv=nv, nc=nc, seed=seed, q_frac=q)


# ------------------------------------------------------------------ M

@pytest.mark.parametrize("n,a,ew,ee,nv,nc", [
    (12, 8.0, 4.0, 1.5, 3, 5),
    (16, 9.0, 5.0, 2.0, 2, 7),
    (20, 10.26, 10.0, 3.0, 4, 60),   # c0
    (24, 14.0, 6.0, 2.5, 5, 37),     # ragged: several tiles, odd counts
])
def test_mtxel_fp64_vs_oracle(ctx, n, a, ew, ee, nv, nc):
    s = synth.make_system("m", a=a, fft=n, ecut_wfn=ew, ecut_eps=ee, nv=nv, nc=nc, seed=100 + n)
    ref = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    got = _mtxel(ctx, s).cpu().numpy()
    assert _rel(got, ref) <= TOL64


def test_mtxel_fp64_plane_wave_closed_form(ctx):
    s = _tiny(31, nv=4, nc=6)
    gen = np.random.default_rng(31)
    iv = gen.choice(s.gv.shape[0], s.nv, replace=False)
    ic = gen.choice(s.gc.shape[0], s.nc, replace=False)
    s.cv = np.zeros_like(s.cv)
    s.cc = np.zeros_like(s.cc)
    s.cv[np.arange(s.nv), iv] = 1.0
    s.cc[np.arange(s.nc), ic] = 1.0
    got = _mtxel(ctx, s).cpu().numpy()
    expect = np.zeros_like(got)
    gidx = {tuple(g): i for i, g in enumerate(s.geps.tolist())}
    for v in range(s.nv):
        for c in range(s.nc):
            d = tuple((s.gv[iv[v]] - s.gc[ic[c]]).tolist())
            if d in gidx:
                expect[v * s.nc + c, gidx[d]] = 1.0
    assert np.abs(got - expect).max() < 1e-14


def test_mtxel_q0_head_is_delta(ctx):
    bvec, _ = synth.cubic_cell(8.0)
    g = synth.gsphere(bvec, (0, 0, 0), 4.0)
    c = synth.orthonormal_bands(np.random.default_rng(5), g.shape[0], 6)
    geps = synth.gsphere(bvec, (0, 0, 0), 1.5)
    s = synth.System("q0", 8.0, bvec, 512.0, np.zeros(3), 12, g, g, geps, c, c, np.zeros(6), np.ones(6))
    m = _mtxel(ctx, s).cpu().numpy().reshape(6, 6, -1)
    assert np.abs(m[:, :, 0] - np.eye(6)).max() < 1e-13


@pytest.mark.parametrize("n", [12, 20, 40])
def test_mtxel_fp32_vs_oracle(ctx, n):
    p = {12: (8.0, 4.0, 1.5, 3, 5), 20: (10.26, 10.0, 3.0, 4, 60), 40: (20.52, 12.0, 6.0, 2, 9)}[n]
    s = synth.make_system("m32", a=p[0], fft=n, ecut_wfn=p[1], ecut_eps=p[2], nv=p[3], nc=p[4], seed=200 + n)
    ref = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    got = _mtxel(ctx, s, prec=1).cpu().numpy().astype(np.complex128)
    assert _rel(got, ref) <= TOL32_M


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [30, 36, 48, 50, 60, 64])
def test_mtxel_large_grids_vs_oracle(ctx, n, prec):
    # the grids of the larger cells (60: the 30.78 bohr cell's grid; radices
    # 2, 3, 4, 5 in every mix), a 12 Ry wavefunction and 6 Ry epsilon sphere
    # in a cell of n / 2 bohr (alias-free: 2 sqrt(12) + sqrt(6) < 2 pi n / a)
    s = synth.make_system("mL", a=0.5 * n, fft=n, ecut_wfn=12.0, ecut_eps=6.0, nv=3, nc=7, seed=400 + n)
    ref = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    got = _mtxel(ctx, s, prec=prec).cpu().numpy().astype(np.complex128)
    assert _rel(got, ref) <= (TOL64 if prec == 0 else TOL32_M)
    # element by element: every entry within the bar of its row's largest
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - ref) <= (TOL64 if prec == 0 else TOL32_M) * scale)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("n,prec", [(40, 1), (60, 1), (60, 0), (24, 1)])
def test_mtxel_pair_kernels_vs_oracle(ctx, n, prec, kernel):
    # both y,x kernels of the pair transform (block, warp per pair) on
    # low-band grids, against the oracle element by element; ragged pair
    # counts (nv nc = 3 x 7 = 21 is no multiple of the 4 pairs of a warp
    # kernel's block), pairs of a block across two bands v
    from paper_1111_4429_gb300 import bgw
    a, ew, ee = {40: (20.52, 12.0, 6.0), 60: (30.0, 12.0, 6.0), 24: (12.0, 12.0, 6.0)}[n]
    s = synth.make_system("mk", a=a, fft=n, ecut_wfn=ew, ecut_eps=ee, nv=3, nc=7, seed=460 + n)
    ref = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    ctx.set_option(bgw.BGW_OPT_PAIR_KERNEL, kernel)
    try:
        got = _mtxel(ctx, s, prec=prec).cpu().numpy().astype(np.complex128)
    finally:
        ctx.set_option(bgw.BGW_OPT_PAIR_KERNEL, -1)
    tol = TOL64 if prec == 0 else TOL32_M
    assert _rel(got, ref) <= tol
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - ref) <= tol * scale)


@pytest.mark.parametrize("prec", [0, 1])
def test_mtxel_wide_eps_sphere_vs_oracle(ctx, prec):
    # an epsilon sphere reaching |G_x| = 6 = n / 4 on the 24 grid: the kernels
    # that keep only the outer quarters of each line cannot serve it, the
    # whole-line ones must
    s = synth.make_system("mw", a=14.0, fft=24, ecut_wfn=3.0, ecut_eps=9.0, nv=3, nc=5, seed=451)
    assert np.abs(s.geps).max() >= 6
    ref = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    got = _mtxel(ctx, s, prec=prec).cpu().numpy().astype(np.complex128)
    assert _rel(got, ref) <= (TOL64 if prec == 0 else TOL32_M)


# ------------------------------------------------------------------ chi, eps, inverse

def _chi(ctx, s, M, omega=None, chunks=None):
    from paper_1111_4429_gb300 import bgw
    nrow = 1 if omega is None else len(omega)
    chi = torch.zeros((nrow, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    cell = bgw.system_cell(s)
    if chunks is None:
        ctx.chi_sum(cell, s.nv, s.nc, s.ng, M, s.ev, s.ec, omega, 0, False, chi)
    else:
        # stream conduction chunks: M rows of a chunk are (v, c in chunk)
        Mv = M.view(s.nv, s.nc, s.ng)
        for k, (c0, c1) in enumerate(chunks):
            Mc = Mv[:, c0:c1].contiguous().view(-1, s.ng)
            ctx.chi_sum(cell, s.nv, c1 - c0, s.ng, Mc, s.ev, s.ec[c0:c1], omega, 0, k > 0, chi)
    ctx.sync()
    return chi


def test_chi_fp64_vs_oracle_c0(ctx):
    s = synth.config_system("c0")
    M = _mtxel(ctx, s)
    ref_m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    ref = oracle.chi(ref_m, oracle.chi_weights(s.ev, s.ec), s.omega)
    got = _chi(ctx, s, M)[0].cpu().numpy()
    assert _rel(got, ref) <= TOL64
    assert np.array_equal(got, np.conj(got).T)  # both triangles written, exactly Hermitian


def test_chi_fp64_chunked_accumulate_and_ragged_tiles(ctx):
    # ng = 231 (four 64-tiles, ragged), conduction streamed in uneven chunks
    s = synth.make_system("r", a=14.0, fft=24, ecut_wfn=6.0, ecut_eps=2.5, nv=5, nc=37, seed=77)
    M = _mtxel(ctx, s)
    ref_m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    ref = oracle.chi(ref_m, oracle.chi_weights(s.ev, s.ec), s.omega)
    got = _chi(ctx, s, M, chunks=[(0, 10), (10, 11), (11, 37)])[0].cpu().numpy()
    assert s.ng % 64 != 0 and s.ng > 128
    assert _rel(got, ref) <= TOL64


def test_chi_fp64_imaginary_frequencies(ctx):
    s = synth.config_system("c0")
    M = _mtxel(ctx, s)
    ref_m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    om = np.concatenate([[0.0], synth.gauss_legendre_frequencies(3)])
    got = _chi(ctx, s, M, omega=om).cpu().numpy()
    for f, w in enumerate(om):
        ref = oracle.chi(ref_m, oracle.chi_weights(s.ev, s.ec, w), s.omega)
        assert _rel(got[f], ref) <= TOL64
    static = oracle.chi(ref_m, oracle.chi_weights(s.ev, s.ec), s.omega)
    assert _rel(got[0], static) <= TOL64


def _epsinv(ctx, systems, chis):
    from paper_1111_4429_gb300 import bgw
    cells = [bgw.system_cell(s) for s in systems]
    eps = [torch.empty_like(x) for x in chis]
    inv = [torch.empty_like(x) for x in chis]
    ctx.epsinv(cells, [s.geps for s in systems], chis, eps, inv)
    ctx.sync()
    return [e.cpu().numpy() for e in eps], [i.cpu().numpy() for i in inv]


def test_epsinv_fp64_vs_oracle_batched_uneven(ctx):
    systems = [synth.config_system("c0"),
               synth.make_system("r", a=14.0, fft=24, ecut_wfn=6.0, ecut_eps=2.5, nv=5, nc=37, seed=78),
               synth.make_system("r2", a=12.0, fft=20, ecut_wfn=5.0, ecut_eps=3.3, nv=3, nc=20, seed=79)]
    refs, chis = [], []
    for s in systems:
        r = oracle.solve(s)
        refs.append(r)
        chis.append(_dev(r["chi"]))   # oracle chi in: tests eps formation + inversion alone
    eps, inv = _epsinv(ctx, systems, chis)
    assert len({s.ng for s in systems}) == 3
    for r, e, i in zip(refs, eps, inv):
        assert _rel(e, r["eps"]) <= TOL64
        assert _rel(i, r["epsinv"]) <= TOL64


def test_epsilon_whole_path_host_buffers_c0(ctx):
    from paper_1111_4429_gb300 import bgw
    s = synth.config_system("c0")
    r = oracle.solve(s)
    chi = np.zeros((1, s.ng, s.ng), dtype=np.complex128)
    inv = np.zeros((1, s.ng, s.ng), dtype=np.complex128)
    ctx.epsilon(bgw.system_cell(s), s.gv, s.cv, s.ev, s.gc, s.cc, s.ec, s.geps, None, 0, 25, chi, inv)
    assert _rel(chi[0], r["chi"]) <= TOL64
    assert _rel(inv[0], r["epsinv"]) <= TOL64


def test_epsilon_whole_path_frequencies_device_buffers(ctx):
    from paper_1111_4429_gb300 import bgw
    s = synth.make_system("r", a=14.0, fft=24, ecut_wfn=6.0, ecut_eps=2.5, nv=5, nc=37, seed=81)
    om = synth.gauss_legendre_frequencies(3)
    chi = torch.zeros((3, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    inv = torch.zeros_like(chi)
    ctx.epsilon(bgw.system_cell(s), s.gv, _dev(s.cv), s.ev, s.gc, _dev(s.cc), s.ec, s.geps, om, 0, 0, chi, inv)
    ctx.sync()
    m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    v = oracle.coulomb(s.bvec, s.q_frac, s.geps)
    for f, w in enumerate(om):
        x = oracle.chi(m, oracle.chi_weights(s.ev, s.ec, w), s.omega)
        _, ei = oracle.epsinv_sym(x, v)
        assert _rel(chi[f].cpu().numpy(), x) <= TOL64
        assert _rel(inv[f].cpu().numpy(), ei) <= TOL64


def test_epsinv_plane_wave_closed_form(ctx):
    from paper_1111_4429_gb300 import bgw
    s = _tiny(41, nv=4, nc=6)
    gen = np.random.default_rng(41)
    s.cv = np.zeros_like(s.cv)
    s.cc = np.zeros_like(s.cc)
    s.cv[np.arange(s.nv), gen.choice(s.gv.shape[0], s.nv, replace=False)] = 1.0
    s.cc[np.arange(s.nc), gen.choice(s.gc.shape[0], s.nc, replace=False)] = 1.0
    chi = np.zeros((1, s.ng, s.ng), dtype=np.complex128)
    inv = np.zeros_like(chi)
    ctx.epsilon(bgw.system_cell(s), s.gv, s.cv, s.ev, s.gc, s.cc, s.ec, s.geps, None, 0, 0, chi, inv)
    x = np.diag(chi[0]).real
    v = oracle.coulomb(s.bvec, s.q_frac, s.geps)
    assert np.abs(chi[0] - np.diag(np.diag(chi[0]))).max() <= 1e-14 * np.abs(chi[0]).max()
    assert np.allclose(np.diag(inv[0]).real, 1.0 / (1.0 - v * x), rtol=1e-14, atol=0)


# ------------------------------------------------------------------ full size (1 q, plain FP64)

def test_c1_full_size_sampled_parity(ctx):
    """c1 at full size in the bench's launch configuration (bgw_epsilon with
    device buffers, one chunk): sampled M rows, sampled chi entries and the
    inverse's residual, each against what the oracle computes one by one."""
    from paper_1111_4429_gb300 import bgw
    s = synth.config_system("c1")
    cell = bgw.system_cell(s)
    M = _mtxel(ctx, s)
    gen = np.random.default_rng(5)
    pairs = np.sort(gen.choice(s.npairs, 6, replace=False))
    pairs = np.concatenate([[0], pairs, [s.npairs - 1]])
    ref_rows = oracle.mtxel_fft_pairs(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft, pairs)
    got_rows = M[torch.as_tensor(pairs, device="cuda")].cpu().numpy()
    assert _rel(got_rows, ref_rows) <= TOL64
    chi = torch.zeros((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    inv = torch.zeros_like(chi)
    ctx.epsilon(cell, s.gv, _dev(s.cv), s.ev, s.gc, _dev(s.cc), s.ec, s.geps, None, 0, 0, chi, inv)
    ctx.sync()
    gi = np.sort(gen.choice(s.ng, 6, replace=False))
    gi = np.concatenate([[0], gi, [s.ng - 1]])
    mcols = oracle.mtxel_direct(s.gv, s.cv, s.gc, s.cc, s.geps[gi])
    ref_x = oracle.chi_entries(mcols, mcols, oracle.chi_weights(s.ev, s.ec), s.omega)
    got_x = chi[0][torch.as_tensor(gi, device="cuda")][:, torch.as_tensor(gi, device="cuda")].cpu().numpy()
    assert _rel(got_x, ref_x) <= TOL64
    # eps~ from the oracle's Coulomb factor and the GPU chi; eps~ eps~^-1 = I
    v = torch.as_tensor(np.sqrt(oracle.coulomb(s.bvec, s.q_frac, s.geps)), device="cuda")
    e = torch.eye(s.ng, dtype=torch.complex128, device="cuda") - v[:, None] * chi[0] * v[None, :]
    res = torch.linalg.matrix_norm(e @ inv[0] - torch.eye(s.ng, dtype=torch.complex128, device="cuda"))
    assert float(res) / math.sqrt(s.ng) <= 1e-13


# ------------------------------------------------------------------ tensor-core inverse

@pytest.mark.parametrize("which", ["c0", "ragged", "two"])
def test_epsinv_tensor_core_update_vs_oracle(ctx, which):
    """The sweep with its trailing updates on the tensor cores (FP16 slices,
    exact FP32 level sums, double-FP32 combination) keeps FP64-level accuracy:
    same 1e-12 bar as the FP64 FMA sweep, on the oracle's chi."""
    from paper_1111_4429_gb300 import bgw
    if which == "c0":
        systems = [synth.config_system("c0")]
    elif which == "ragged":
        systems = [synth.make_system("r", a=14.0, fft=24, ecut_wfn=6.0, ecut_eps=2.5, nv=5, nc=37, seed=78)]
    else:  # two matrices of different size in one batch, several 128-row tiles
        systems = [synth.make_system("r", a=20.52, fft=40, ecut_wfn=8.0, ecut_eps=3.0, nv=4, nc=90, seed=88),
                   synth.make_system("s", a=17.0, fft=40, ecut_wfn=8.0, ecut_eps=3.5, nv=4, nc=90, seed=89)]
    refs, chis = [], []
    for s in systems:
        r = oracle.solve(s)
        refs.append(r)
        chis.append(_dev(r["chi"]))
    ctx.set_option(bgw.BGW_OPT_INVERSE, 1)
    try:
        eps, inv = _epsinv(ctx, systems, chis)
    finally:
        ctx.set_option(bgw.BGW_OPT_INVERSE, -1)
    for r, i in zip(refs, inv):
        assert _rel(i, r["epsinv"]) <= TOL64


@pytest.mark.parametrize("which", ["c0", "two"])
def test_epsinv_tensor_core_update_five_slices(ctx, which):
    """Five slices per value (the mixed solves' default): the update error is
    near 2^-34 of its scale instead of 2^-48, so the bar is 2^14 times the
    FP64 one; the batch of two sizes covers ragged tiles."""
    from paper_1111_4429_gb300 import bgw
    if which == "c0":
        systems = [synth.config_system("c0")]
    else:
        systems = [synth.make_system("r", a=20.52, fft=40, ecut_wfn=8.0, ecut_eps=3.0, nv=4, nc=90, seed=88),
                   synth.make_system("s", a=17.0, fft=40, ecut_wfn=8.0, ecut_eps=3.5, nv=4, nc=90, seed=89)]
    refs = [oracle.solve(s) for s in systems]
    chis = [_dev(r["chi"]) for r in refs]
    ctx.set_option(bgw.BGW_OPT_INVERSE, 1)
    ctx.set_option(bgw.BGW_OPT_UPDATE_SLICES, 5)
    try:
        _, inv5 = _epsinv(ctx, systems, chis)
        ctx.set_option(bgw.BGW_OPT_UPDATE_SLICES, 7)
        _, inv7 = _epsinv(ctx, systems, chis)
    finally:
        ctx.set_option(bgw.BGW_OPT_INVERSE, -1)
        ctx.set_option(bgw.BGW_OPT_UPDATE_SLICES, 0)
    for r, a, b in zip(refs, inv5, inv7):
        assert _rel(a, r["epsinv"]) <= TOL64 * 2 ** 14
        assert _rel(b, r["epsinv"]) <= TOL64


@pytest.mark.parametrize("slices", [5, 7])
def test_epsinv_graph_replay_matches_direct(ctx, slices):
    """On a capturable stream, repeated bgw_epsinv calls with the same
    arguments replay a CUDA graph of the sweep: the replay reads the current
    chi (same buffer, new contents) and gives the direct run's result bit for
    bit, and the launch count grows by the graph's kernels."""
    from paper_1111_4429_gb300 import bgw
    systems = [synth.make_system("r", a=20.52, fft=40, ecut_wfn=8.0, ecut_eps=3.0, nv=4, nc=90, seed=88)]
    s = systems[0]
    r = oracle.solve(s)
    chi_a = _dev(r["chi"])
    chi_b = _dev(1.3 * r["chi"])
    cell = bgw.system_cell(s)
    buf = torch.empty_like(chi_a)
    out = torch.empty_like(chi_a)
    side = torch.cuda.Stream()
    ctx.set_option(bgw.BGW_OPT_INVERSE, 1)
    ctx.set_option(bgw.BGW_OPT_UPDATE_SLICES, slices)
    try:
        with torch.cuda.stream(side):
            results = []
            g0 = ctx.graph_stats()
            for src in (chi_a, chi_a, chi_b, chi_a):   # direct + capture, then replays
                buf.copy_(src)
                l0 = ctx.launch_count()
                ctx.epsinv([cell], [s.geps], [buf], None, [out])
                side.synchronize()
                results.append((out.cpu().numpy().copy(), ctx.launch_count() - l0))
            g1 = ctx.graph_stats()
        # direct results of the same inputs with graphs off (timing on runs directly)
        ctx.set_option(bgw.BGW_OPT_TIMING, 1)
        with torch.cuda.stream(side):
            direct = []
            for src in (chi_a, chi_b):
                buf.copy_(src)
                ctx.epsinv([cell], [s.geps], [buf], None, [out])
                side.synchronize()
                direct.append(out.cpu().numpy().copy())
    finally:
        ctx.set_option(bgw.BGW_OPT_TIMING, 0)
        ctx.set_option(bgw.BGW_OPT_INVERSE, -1)
        ctx.set_option(bgw.BGW_OPT_UPDATE_SLICES, 0)
    assert np.array_equal(results[0][0], direct[0])
    assert np.array_equal(results[1][0], direct[0])
    assert np.array_equal(results[2][0], direct[1])
    assert np.array_equal(results[3][0], direct[0])
    assert results[1][1] == results[0][1] > 50   # a replay counts the graph's kernels
    assert g1[1] == g0[1] + 3                        # calls 2-4 replayed
    assert _rel(results[0][0], r["epsinv"]) <= TOL64 * (2 ** 14 if slices == 5 else 1)


@pytest.mark.parametrize("slices,which", [(7, "one"), (7, "two"), (5, "one")])
def test_epsinv_update_item_widths_bit_identical(ctx, slices, which):
    """The bulk update's work-item width (the wide items or items of two
    column tiles, BGW_OPT_UPDATE_ITEMS) only regroups tiles among CTAs: the
    inverse is bit for bit the same under both and under the default rule,
    and meets the oracle's bar."""
    from paper_1111_4429_gb300 import bgw
    systems = [synth.make_system("r", a=20.52, fft=40, ecut_wfn=8.0, ecut_eps=3.0, nv=4, nc=90, seed=88)]
    if which == "two":
        systems.append(synth.make_system("s", a=17.0, fft=40, ecut_wfn=8.0, ecut_eps=3.5, nv=4, nc=90, seed=89))
    refs = [oracle.solve(s) for s in systems]
    chis = [_dev(r["chi"]) for r in refs]
    ctx.set_option(bgw.BGW_OPT_INVERSE, 1)
    ctx.set_option(bgw.BGW_OPT_UPDATE_SLICES, slices)
    try:
        _, rule = _epsinv(ctx, systems, chis)
        ctx.set_option(bgw.BGW_OPT_UPDATE_ITEMS, 0)
        _, wide = _epsinv(ctx, systems, chis)
        ctx.set_option(bgw.BGW_OPT_UPDATE_ITEMS, 1)
        _, narrow = _epsinv(ctx, systems, chis)
    finally:
        ctx.set_option(bgw.BGW_OPT_UPDATE_ITEMS, -1)
        ctx.set_option(bgw.BGW_OPT_INVERSE, -1)
        ctx.set_option(bgw.BGW_OPT_UPDATE_SLICES, 0)
    for r, a, w, n in zip(refs, rule, wide, narrow):
        assert np.array_equal(a, w) and np.array_equal(n, w)
        assert _rel(w, r["epsinv"]) <= TOL64 * (2 ** 14 if slices == 5 else 1)
