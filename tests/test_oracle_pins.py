"""Pins for the CPU oracle: closed forms, invariants and brute force.

The paper prints no numeric chi or eps^-1 values (its figures are
placeholders), so the oracle is pinned by mathematics: each test below fails
for a plausible mistake (a dropped conjugate, a wrong FFT sign or scale, a
missing 4/Omega, a transposed operand, v in place of v^{1/2}, a wrong pair
order or a wrong frequency weight).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1111_4429_gb300 import synth


def _tiny(seed=7, a=8.0, n=12, ew=4.0, ee=1.5, nv=3, nc=5, q=(0.1, 0.0, 0.0)):
    return synth.make_system("tiny", a=a, fft=n, ecut_wfn=ew, ecut_eps=ee, nv=nv, nc=nc,
                             seed=seed, q_frac=q)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# --------------------------------------------------------------------- spheres

def test_gsphere_strict_cutoff_and_order():
    bvec, _ = synth.cubic_cell(10.26)
    g = synth.gsphere(bvec, (0.1, 0, 0), 3.0)
    k = (g + np.array([0.1, 0, 0])) @ bvec
    e = np.einsum("ij,ij->i", k, k)
    assert np.all(e < 3.0)
    assert np.all(np.diff(e) >= -1e-15)
    # brute-force count over a generous box
    r = np.arange(-8, 9)
    gx, gy, gz = np.meshgrid(r, r, r, indexing="ij")
    allg = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1)
    ka = (allg + np.array([0.1, 0, 0])) @ bvec
    assert g.shape[0] == int(np.sum(np.einsum("ij,ij->i", ka, ka) < 3.0)) == 85
    assert len({tuple(x) for x in g.tolist()}) == g.shape[0]


@pytest.mark.parametrize("a,ecut,qx10", [(30.78, 6.0, 1), (30.78, 12.0, 1), (30.78, 12.0, 0), (20.52, 6.0, 5)])
def test_gsphere_order_is_exact(a, ecut, qx10):
    """The order of a sphere is the exact one, so it is the same on every
    machine: in a cubic cell |q + G|^2 b^-2 = (G_x + q_x)^2 + G_y^2 + G_z^2,
    which for q_x = qx10 / 10 is the integer (10 G_x + qx10)^2 + 100 (G_y^2 +
    G_z^2) over 100.  Lengths equal in exact arithmetic (G_y and G_z swapped,
    signs flipped) must follow the lexicographic order of (G_x, G_y, G_z),
    whatever the last bits of their floating-point lengths."""
    bvec, _ = synth.cubic_cell(a)
    g = synth.gsphere(bvec, (qx10 / 10.0, 0, 0), ecut).astype(np.int64)
    key = (10 * g[:, 0] + qx10) ** 2 + 100 * (g[:, 1] ** 2 + g[:, 2] ** 2)
    exact = np.lexsort((g[:, 2], g[:, 1], g[:, 0], key))
    assert np.array_equal(exact, np.arange(g.shape[0]))


def test_config_sphere_sizes():
    for name, ng, npw_c, npw_v in [("c0", 85, 587, 583), ("c1", 2120, 6031, 6059)]:
        p = synth.CONFIGS[name]
        bvec, _ = synth.cubic_cell(p["a"])
        assert synth.gsphere(bvec, (0.1, 0, 0), p["ecut_eps"]).shape[0] == ng
        assert synth.gsphere(bvec, (0, 0, 0), p["ecut_wfn"]).shape[0] == npw_c
        assert synth.gsphere(bvec, (0.1, 0, 0), p["ecut_wfn"]).shape[0] == npw_v


def test_bands_orthonormal():
    s = _tiny()
    for c in (s.cv, s.cc):
        assert np.allclose(c @ np.conj(c).T, np.eye(c.shape[0]), atol=1e-13)


def test_gauss_legendre_nodes_closed_form():
    # 2-point nodes +-1/sqrt(3), 3-point 0, +-sqrt(3/5), mapped from [-1,1] to [0,2]
    assert np.allclose(synth.gauss_legendre_frequencies(2), 1.0 + np.array([-1, 1]) / math.sqrt(3))
    assert np.allclose(synth.gauss_legendre_frequencies(3), 1.0 + np.array([-1, 0, 1]) * math.sqrt(0.6))
    w12 = synth.gauss_legendre_frequencies(12)
    assert abs(w12[0] - 0.018439365753281) < 1e-12 and abs(w12[-1] - 1.981560634246719) < 1e-12


# ---------------------------------------------------------------- matrix elements

def test_mtxel_direct_vs_fft_bruteforce():
    for seed, n in [(1, 12), (2, 16)]:
        s = _tiny(seed=seed, n=n)
        m1 = oracle.mtxel_direct(s.gv, s.cv, s.gc, s.cc, s.geps)
        m2 = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
        assert _rel(m2, m1) < 1e-13


def test_mtxel_c0_direct_vs_fft():
    s = synth.config_system("c0")
    m1 = oracle.mtxel_direct(s.gv, s.cv, s.gc, s.cc, s.geps)
    m2 = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    assert _rel(m2, m1) < 1e-13
    assert np.abs(m1).max() <= 1.0 + 1e-12          # Cauchy-Schwarz, sum |c|^2 = 1


def test_mtxel_fft_pairs_matches_full():
    s = _tiny(seed=3)
    full = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    pairs = [0, 4, 7, 14]
    sub = oracle.mtxel_fft_pairs(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft, pairs)
    assert np.allclose(sub, full[pairs], atol=1e-15)


def _plane_wave_system(seed=5):
    s = _tiny(seed=seed, nv=4, nc=6)
    gen = np.random.default_rng(seed)
    iv = gen.choice(s.gv.shape[0], s.nv, replace=False)
    ic = gen.choice(s.gc.shape[0], s.nc, replace=False)
    cv = np.zeros_like(s.cv)
    cc = np.zeros_like(s.cc)
    cv[np.arange(s.nv), iv] = 1.0
    cc[np.arange(s.nc), ic] = 1.0
    s.cv, s.cc = cv, cc
    return s, iv, ic


def test_mtxel_plane_wave_closed_form():
    # c_v = e_{G_v}, c_c = e_{G_c}  =>  M_vc(G) = 1 iff G = G_v - G_c, else 0.
    s, iv, ic = _plane_wave_system()
    expect = np.zeros((s.nv * s.nc, s.ng))
    gidx = {tuple(g): i for i, g in enumerate(s.geps.tolist())}
    for v in range(s.nv):
        for c in range(s.nc):
            d = tuple((s.gv[iv[v]] - s.gc[ic[c]]).tolist())
            if d in gidx:
                expect[v * s.nc + c, gidx[d]] = 1.0
    assert expect.sum() > 0
    for m in (oracle.mtxel_direct(s.gv, s.cv, s.gc, s.cc, s.geps),
              oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)):
        assert np.allclose(m, expect, atol=1e-14)


def test_mtxel_q0_joint_orthonormal_head_is_delta():
    # q = 0, one sphere, jointly orthonormal bands: M_nn'(G=0) = <n|n'> = delta.
    bvec, _ = synth.cubic_cell(8.0)
    g = synth.gsphere(bvec, (0, 0, 0), 4.0)
    c = synth.orthonormal_bands(np.random.default_rng(11), g.shape[0], 7)
    geps = synth.gsphere(bvec, (0, 0, 0), 1.5)
    assert tuple(geps[0]) == (0, 0, 0)
    m = oracle.mtxel_fft(g, c, g, c, geps, 12).reshape(7, 7, -1)
    assert np.allclose(m[:, :, 0], np.eye(7), atol=1e-13)
    md = oracle.mtxel_direct(g, c, g, c, geps).reshape(7, 7, -1)
    assert np.allclose(md[:, :, 0], np.eye(7), atol=1e-13)


def test_mtxel_parseval_full_grid():
    # Over every G of the grid: sum_G |F(G)|^2 = (1/N_r) sum_j |u_v u_c|^2.
    s = _tiny(seed=9, n=10, ew=2.5)
    n = s.fft
    r = np.arange(-n // 2, n // 2)
    gx, gy, gz = np.meshgrid(r, r, r, indexing="ij")
    gall = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1).astype(np.int32)
    m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, gall, n)
    uv = oracle.band_grids(s.gv, s.cv, n)
    uc = oracle.band_grids(s.gc, s.cc, n)
    for v in range(s.nv):
        for c in range(s.nc):
            lhs = np.sum(np.abs(m[v * s.nc + c]) ** 2)
            rhs = np.sum(np.abs(np.conj(uv[v]) * uc[c]) ** 2) / n ** 3
            assert abs(lhs - rhs) < 1e-12 * rhs


def test_band_grid_normalization():
    # sum_j |u_b(r_j)|^2 = N_r sum_G |c_b(G)|^2 = N_r (unnormalized inverse transform)
    s = _tiny(seed=4)
    u = oracle.band_grids(s.gc, s.cc, s.fft)
    assert np.allclose(np.sum(np.abs(u) ** 2, axis=(1, 2, 3)), s.fft ** 3, rtol=1e-13)


# -------------------------------------------------------------- polarizability

def test_chi_weights_pair_order_and_values():
    ev = np.array([-0.3, -0.1])
    ec = np.array([0.2, 0.5, 0.9])
    w = oracle.chi_weights(ev, ec)
    assert np.allclose(w, [1 / (-0.5), 1 / (-0.8), 1 / (-1.2), 1 / (-0.3), 1 / (-0.6), 1 / (-1.0)])
    wi = oracle.chi_weights(ev, ec, 0.7)
    d = -0.5
    assert abs(wi[0] - d / (d * d + 0.49)) < 1e-15
    # the imaginary-axis weight is the average of the two time orderings
    assert abs(wi[0] - 0.5 * (1 / (d - 0.7j) + 1 / (d + 0.7j)).real) < 1e-15


def test_chi_hand_example_conjugation_side():
    # One empty band c = e_0 and one occupied band v = (e_G1 + i e_G2)/sqrt(2):
    # M(G) = conj(c_v(G)), so M(G1) = 1/sqrt2, M(G2) = -i/sqrt2 and
    # chi_{G1 G2} = (4/Omega) w conj(M(G1)) M(G2) = -i (2/Omega) w.
    g = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.int32)
    gc = g[:1]
    cc = np.array([[1.0 + 0j]])
    cv = np.array([[0.0, 1.0, 1.0j]]) / math.sqrt(2.0)
    geps = g[1:]
    m = oracle.mtxel_direct(g, cv, gc, cc, geps)
    assert np.allclose(m, [[1 / math.sqrt(2), -1j / math.sqrt(2)]])
    mf = oracle.mtxel_fft(g, cv, gc, cc, geps, 6)
    assert np.allclose(mf, m, atol=1e-15)
    omega_cell, w = 100.0, np.array([-2.0])
    x = oracle.chi(m, w, omega_cell)
    assert np.allclose(x[0, 1], -1j * (2 / omega_cell) * w[0])
    assert np.allclose(x[0, 0], (4 / omega_cell) * w[0] * 0.5)
    assert np.allclose(oracle.chi_direct(m, w, omega_cell), x, atol=1e-15)


def test_chi_tier1_vs_tier2_and_hermitian_nsd():
    s = synth.config_system("c0")
    m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    w = oracle.chi_weights(s.ev, s.ec)
    x1 = oracle.chi_direct(m, w, s.omega)
    x2 = oracle.chi(m, w, s.omega)
    assert _rel(x2, x1) < 1e-14
    assert np.linalg.norm(x2 - np.conj(x2).T) < 1e-14 * np.linalg.norm(x2)
    assert np.linalg.eigvalsh(x2).max() <= 1e-14 * np.abs(x2).max()
    # trace identity: tr chi = (4/Omega) sum_p w_p ||M_p||^2
    assert abs(np.trace(x2) - (4 / s.omega) * np.sum(w * np.sum(np.abs(m) ** 2, 1))) < 1e-13 * abs(np.trace(x2))


def test_chi_plane_wave_closed_form_diagonal():
    s, iv, ic = _plane_wave_system(seed=8)
    m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    w = oracle.chi_weights(s.ev, s.ec)
    x = oracle.chi(m, w, s.omega)
    expect = np.zeros((s.ng, s.ng), dtype=np.complex128)
    gidx = {tuple(g): i for i, g in enumerate(s.geps.tolist())}
    for v in range(s.nv):
        for c in range(s.nc):
            d = tuple((s.gv[iv[v]] - s.gc[ic[c]]).tolist())
            if d in gidx:
                expect[gidx[d], gidx[d]] += (4 / s.omega) / (s.ev[v] - s.ec[c])
    assert np.allclose(x, expect, atol=1e-14)


# --------------------------------------------------------- dielectric matrix

def test_coulomb_closed_form():
    bvec, _ = synth.cubic_cell(10.26)
    b = 2 * math.pi / 10.26
    geps = np.array([[0, 0, 0], [1, 0, 0], [0, -1, 2]], dtype=np.int32)
    v = oracle.coulomb(bvec, (0.1, 0, 0), geps)
    expect = [4 * math.pi / (0.1 * b) ** 2, 4 * math.pi / (1.1 * b) ** 2,
              4 * math.pi / ((0.01 + 1 + 4) * b * b)]
    assert np.allclose(v, expect, rtol=1e-15)
    with pytest.raises(ValueError):
        oracle.coulomb(bvec, (0, 0, 0), geps)


def test_gauss_jordan_closed_forms_and_pivoting():
    a = np.array([[2.0 + 1j, 1.0], [3.0, 4.0 - 2j]])
    det = a[0, 0] * a[1, 1] - a[0, 1] * a[1, 0]
    expect = np.array([[a[1, 1], -a[0, 1]], [-a[1, 0], a[0, 0]]]) / det
    assert np.allclose(oracle.inv_gauss_jordan(a), expect, atol=1e-15)
    perm = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 2.0], [4.0, 0.0, 0.0]])  # zero leading pivot
    assert np.allclose(oracle.inv_gauss_jordan(perm) @ perm, np.eye(3), atol=1e-15)
    r = np.random.default_rng(0)
    b = r.standard_normal((40, 40)) + 1j * r.standard_normal((40, 40))
    assert _rel(oracle.inv_gauss_jordan(b), np.linalg.inv(b)) < 1e-12


def test_eps_spectrum_and_inverse_c0():
    s = synth.config_system("c0")
    r = oracle.solve(s, tier=2)
    e, ei = r["eps"], r["epsinv"]
    assert np.linalg.norm(e - np.conj(e).T) < 1e-14 * np.linalg.norm(e)
    assert np.linalg.eigvalsh(e).min() >= 1.0 - 1e-12
    lam = np.linalg.eigvalsh(0.5 * (ei + np.conj(ei).T))
    assert lam.min() > 0 and lam.max() <= 1.0 + 1e-12
    assert np.linalg.norm(e @ ei - np.eye(s.ng)) / math.sqrt(s.ng) < 1e-13
    assert _rel(oracle.inv_gauss_jordan(e), ei) < 1e-13


def test_eps_symmetric_vs_asymmetric_route_and_w_hermitian():
    s = synth.config_system("c0")
    r = oracle.solve(s)
    v = r["v"]
    ea = oracle.eps_asym(r["chi"], v)
    eia = oracle.inv(ea)
    sv = np.sqrt(v)
    # eps^-1 (paper's asymmetric) = V^{1/2} eps~^-1 V^{-1/2}
    assert _rel(sv[:, None] * r["epsinv"] / sv[None, :], eia) < 1e-13
    w = oracle.screened_w(eia, v)
    assert np.linalg.norm(w - np.conj(w).T) < 1e-12 * np.linalg.norm(w)


def test_eps_plane_wave_closed_form_diagonal():
    s, _, _ = _plane_wave_system(seed=12)
    r = oracle.solve(s)
    x = np.diag(r["chi"]).real
    expect = 1.0 / (1.0 - r["v"] * x)
    assert np.allclose(r["epsinv"], np.diag(expect), atol=1e-14)


def test_tier1_whole_chain_matches_tier2():
    s = _tiny(seed=21, nv=3, nc=7)
    r1 = oracle.solve(s, tier=1)
    r2 = oracle.solve(s, tier=2)
    for k in ("M", "chi", "eps", "epsinv"):
        assert _rel(r2[k], r1[k]) < 1e-13, k


# ------------------------------------------------------------ imaginary axis

def test_imaginary_frequency_limits_and_monotonicity():
    s = synth.config_system("c0")
    m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    v = oracle.coulomb(s.bvec, s.q_frac, s.geps)
    x0 = oracle.chi(m, oracle.chi_weights(s.ev, s.ec), s.omega)
    xw0 = oracle.chi(m, oracle.chi_weights(s.ev, s.ec, 0.0), s.omega)
    assert _rel(xw0, x0) < 1e-15
    prev_x, prev_ei = None, None
    for om in synth.gauss_legendre_frequencies(4):
        x = oracle.chi(m, oracle.chi_weights(s.ev, s.ec, om), s.omega)
        _, ei = oracle.epsinv_sym(x, v)
        if prev_x is not None:
            # chi(i w1) <= chi(i w2) <= 0 and eps~^-1(i w1) <= eps~^-1(i w2) <= I (Loewner)
            assert np.linalg.eigvalsh(prev_x - x).max() <= 1e-14
            assert np.linalg.eigvalsh(prev_ei - ei).max() <= 1e-12
        assert np.linalg.eigvalsh(x).max() <= 1e-14
        prev_x, prev_ei = x, 0.5 * (ei + np.conj(ei).T)
    xinf = oracle.chi(m, oracle.chi_weights(s.ev, s.ec, 1e6), s.omega)
    _, eiinf = oracle.epsinv_sym(xinf, v)
    assert np.abs(eiinf - np.eye(s.ng)).max() < 1e-8


# ------------------------------------------------------------ Coulomb truncations and W

def test_truncated_coulomb_closed_forms():
    bvec, _ = synth.cubic_cell(10.0)
    b = 2 * math.pi / 10.0
    geps = np.array([[0, 0, 0], [1, 0, 0], [0, 0, 1], [1, 1, 2]], dtype=np.int32)
    rc = 5.0
    vs = oracle.coulomb(bvec, (0, 0, 0), geps, "sphere", rc)
    assert abs(vs[0] - 2 * math.pi * rc * rc) < 1e-12             # k -> 0 limit
    assert abs(vs[1] - 4 * math.pi / b ** 2 * (1 - math.cos(rc * b))) < 1e-12
    # k r_c = 2 pi: the truncated interaction vanishes
    v0 = oracle.coulomb(bvec, (0, 0, 0), np.array([[1, 0, 0]], dtype=np.int32), "sphere", 10.0)
    assert abs(v0[0]) < 1e-12
    # small k: 4 pi/k^2 (1 - cos(r_c k)) -> 2 pi r_c^2 (1 - (r_c k)^2 / 12)
    tiny = oracle.coulomb(bvec, (1e-4, 0, 0), np.array([[0, 0, 0]], dtype=np.int32), "sphere", rc)
    kk = 1e-4 * b
    assert abs(tiny[0] - 2 * math.pi * rc * rc * (1 - (rc * kk) ** 2 / 12)) < 1e-9
    zc = 5.0
    vl = oracle.coulomb(bvec, (0.1, 0, 0), geps, "slab", zc)
    k0 = 0.1 * b
    assert abs(vl[0] - 4 * math.pi / k0 ** 2 * (1 - math.exp(-k0 * zc))) < 1e-9  # in-plane: cos(0) = 1
    kz = b                                                                          # [0,0,1] + q: k_xy = 0.1 b
    kxy = 0.1 * b
    expect = 4 * math.pi / (kxy ** 2 + kz ** 2) * (1 - math.exp(-kxy * zc) * math.cos(kz * zc))
    assert abs(vl[2] - expect) < 1e-12
    # both truncations are bounded by twice the bulk interaction and are >= 0
    vb = oracle.coulomb(bvec, (0.1, 0.2, 0.3), geps)
    for model in ("sphere", "slab"):
        vt = oracle.coulomb(bvec, (0.1, 0.2, 0.3), geps, model, 3.0)
        assert np.all(vt >= 0) and np.all(vt <= 2 * vb + 1e-12)
    with pytest.raises(ValueError):
        oracle.coulomb(bvec, (0, 0, 0), geps, "slab", zc)


def test_screened_w_routes_agree_and_hermitian_truncated():
    s = synth.config_system("c0")
    for model, rc in (("bulk", 0.0), ("sphere", 4.0), ("slab", 5.13)):
        r = oracle.solve(s, model=model, rc=rc)
        v = r["v"]
        w_sym = oracle.screened_w_sym(r["epsinv"], v)
        # the paper's route: asymmetric eps = I - v chi, W = eps^-1 v
        w_asym = oracle.screened_w(oracle.inv(oracle.eps_asym(r["chi"], v)), v)
        assert np.linalg.norm(w_sym - w_asym) <= 1e-12 * np.linalg.norm(w_asym)
        assert np.linalg.norm(w_sym - np.conj(w_sym).T) <= 1e-14 * np.linalg.norm(w_sym)
        # W = v^1/2 eps~^-1 v^1/2 with 0 < eps~^-1 <= I: 0 <= W <= V
        lam = np.linalg.eigvalsh(np.diag(v) - w_sym)
        assert lam.min() >= -1e-12 * v.max()


def _q0(qf, **kw):
    p = dict(synth.CONFIGS["c0"])
    p.update(kw)
    return synth.q0_system("q0", **p, q_frac=(qf, 0.0, 0.0))


def test_q0_head_direct_dot_and_limit():
    # At q0 the head M_vc(G=0) = <u_v(k+q0)|u_c> is a plain dot product of the
    # coefficient vectors over the common G (Eq. eqn_matrix_elem at G = 0); the
    # oracle's FFT route must agree, and the head v(q0) chi_00 -- the
    # macroscopic response -- must tend to a finite limit as q0 -> 0.
    heads = []
    for qf in (1e-3, 5e-4):
        s = _q0(qf)
        r = oracle.solve(s)
        assert tuple(s.geps[0]) == (0, 0, 0)
        idx = {tuple(g): i for i, g in enumerate(s.gc.tolist())}
        cvk = np.zeros((s.nv, s.gc.shape[0]), dtype=np.complex128)
        for j, g in enumerate(s.gv.tolist()):
            cvk[:, idx[tuple(g)]] = s.cv[:, j]
        m0 = (np.conj(cvk) @ s.cc.T).ravel()                       # [p], p = v*nc + c
        assert np.abs(m0).max() < 50 * np.linalg.norm(s.q_frac @ s.bvec)  # O(|q0|)
        mf = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps[:1], s.fft)[:, 0]
        assert np.abs(mf - m0).max() <= 1e-15
        w = oracle.chi_weights(s.ev, s.ec)
        head = r["v"][0] * (4.0 / s.omega) * np.sum(w * np.abs(m0) ** 2)
        assert abs(head - r["v"][0] * r["chi"][0, 0].real) <= 1e-12 * abs(head)
        heads.append(head)
        # the symmetrized wings sqrt(v0 vG) chi_0G stay O(1) although v0 ~ 1/q0^2
        wing = np.sqrt(r["v"][0] * r["v"][1:]) * r["chi"][0, 1:]
        assert np.abs(wing).max() < 1.0
    assert -20 < heads[0] < -1
    assert abs(heads[0] - heads[1]) <= 1e-3 * abs(heads[1])        # O(q0) approach to the limit


# ------------------------------------------------- real-axis (full-frequency) response

def test_real_axis_weights_limits_signs_and_conjugation():
    ev = np.array([-0.4, -0.05])
    ec = np.array([0.1, 0.35, 1.2])
    d = (ev[:, None] - ec[None, :]).ravel()
    e, dl = 0.3, 0.07
    wr = oracle.chi_weights_real(ev, ec, e, dl)
    wa = oracle.chi_weights_real(ev, ec, e, dl, advanced=True)
    # real and imaginary parts written out separately (upper signs: retarded)
    re = 0.5 * ((d - e) / ((d - e) ** 2 + dl ** 2) + (d + e) / ((d + e) ** 2 + dl ** 2))
    im = 0.5 * dl * (1 / ((d - e) ** 2 + dl ** 2) - 1 / ((d + e) ** 2 + dl ** 2))
    assert np.allclose(wr.real, re, rtol=1e-14, atol=0) and np.allclose(wr.imag, im, rtol=1e-13, atol=0)
    assert np.all(wr.imag < 0)                          # absorption: Im chi^r <= 0 for E > 0
    assert np.array_equal(wa, np.conj(wr))
    # E = i omega, delta = 0: the imaginary-axis weight; E = 0: Delta / (Delta^2 + delta^2)
    assert np.allclose(oracle.chi_weights_real(ev, ec, 0.8j, 0.0), oracle.chi_weights(ev, ec, 0.8), rtol=1e-15)
    assert np.allclose(oracle.chi_weights_real(ev, ec, 0.0, dl), oracle.chi_weights(ev, ec, dl), rtol=1e-15)
    assert np.allclose(oracle.chi_weights_real(ev, ec, 0.0, 0.0), oracle.chi_weights(ev, ec), rtol=1e-15)


def test_frequency_grid_closed_form():
    g = oracle.frequency_grid(0.1, 0.5, 2.0, 0.1)
    assert np.allclose(g, [0.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.7, 1.0, 1.4, 1.9], atol=1e-15)
    assert np.allclose(oracle.frequency_grid(0.25, 1.0, 2.0, 0.0), np.arange(9) * 0.25, atol=1e-15)
    g = oracle.frequency_grid(0.2, 1.0, 10.0, 0.05)
    steps = np.diff(g)
    assert np.allclose(steps[:5], 0.2) and np.allclose(np.diff(steps[5:]), 0.05) and g[-1] <= 10.0 + 1e-11
    assert g[-1] + steps[-1] + 0.05 > 10.0
    with pytest.raises(ValueError):
        oracle.frequency_grid(0.0, 1.0, 2.0, 0.1)


def test_real_axis_chi_structure():
    s = _tiny(seed=12, nv=3, nc=9)
    m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    for e in (0.2, 0.9):
        wr = oracle.chi_weights_real(s.ev, s.ec, e, 0.05)
        xr = oracle.chi(m, wr, s.omega)
        xa = oracle.chi(m, oracle.chi_weights_real(s.ev, s.ec, e, 0.05, advanced=True), s.omega)
        assert np.allclose(xa, np.conj(xr).T, atol=1e-15)
        assert np.linalg.norm(xr - np.conj(xr).T) > 1e-3 * np.linalg.norm(xr)   # not Hermitian
        # the anti-Hermitian part (chi - chi^H) / 2i is negative semidefinite
        lam = np.linalg.eigvalsh((xr - np.conj(xr).T) / 2j)
        assert lam.max() <= 1e-14 * np.abs(lam).max()
        assert np.allclose(oracle.chi_direct(m, wr, s.omega), xr, atol=1e-14)
    # E = 0: chi^r(0; delta) = chi(i omega = delta), real weights, Hermitian
    x0 = oracle.chi(m, oracle.chi_weights_real(s.ev, s.ec, 0.0, 0.3), s.omega)
    assert np.allclose(x0, oracle.chi(m, oracle.chi_weights(s.ev, s.ec, 0.3), s.omega), atol=1e-15)


def test_real_axis_plane_wave_closed_form_and_adjoint_inverse():
    s, iv, ic = _plane_wave_system(seed=8)
    e, dl = 0.6, 0.05
    r = oracle.solve_real(s, [e], dl)
    gidx = {tuple(g): i for i, g in enumerate(s.geps.tolist())}
    diag = np.zeros(s.ng, dtype=np.complex128)
    for v in range(s.nv):
        for c in range(s.nc):
            d = tuple((s.gv[iv[v]] - s.gc[ic[c]]).tolist())
            if d in gidx:
                dd = s.ev[v] - s.ec[c]
                diag[gidx[d]] += (4 / s.omega) * 0.5 * (1 / (dd - e - 1j * dl) + 1 / (dd + e + 1j * dl))
    assert np.allclose(r["chi"][0], np.diag(diag), atol=1e-14)
    assert np.allclose(r["epsinv"][0], np.diag(1.0 / (1.0 - r["v"] * diag)), atol=1e-13)
    # advanced = adjoint of retarded, through the whole chain
    s2 = _tiny(seed=13, nv=3, nc=9)
    rr = oracle.solve_real(s2, [0.4, 1.1], 0.04)
    ra = oracle.solve_real(s2, [0.4, 1.1], 0.04, advanced=True)
    for f in range(2):
        assert np.allclose(ra["epsinv"][f], np.conj(rr["epsinv"][f]).T, atol=1e-12)
        # tier 1 (Gauss-Jordan with partial pivoting) = tier 2 (library LU)
        assert _rel(oracle.inv_gauss_jordan(rr["eps"][f]), rr["epsinv"][f]) < 1e-13


# ------------------------------------------------------------------ real flavor

def test_realify_recovers_real_subspaces():
    gen = np.random.default_rng(21)
    npw, nb = 40, 7
    q, _ = np.linalg.qr(gen.standard_normal((npw, nb)))
    real = q.T                                        # real orthonormal bands
    e = np.array([-0.5, -0.3, -0.3, -0.3, 0.1, 0.4, 0.4])
    groups = [[1, 2, 3], [5, 6]]
    cplx = synth.scramble_phases(real, groups, seed=5)
    assert np.abs(cplx.imag).max() > 0.1              # genuinely complex input
    r = oracle.realify(cplx, e, 1e-9)
    assert r.dtype == np.float64
    assert np.allclose(r @ r.T, np.eye(nb), atol=1e-13)
    for g in [[0], [1, 2, 3], [4], [5, 6]]:
        # same subspace: the projectors agree (the basis inside it is not unique)
        pa, pb = real[g].T @ real[g], r[g].T @ r[g]
        assert np.abs(pa - pb).max() < 1e-13
    # a non-degenerate band is the original one up to sign
    assert min(np.abs(r[0] - real[0]).max(), np.abs(r[0] + real[0]).max()) < 1e-13
    # a subspace that is not real (no symmetry) has too few real directions
    bad = gen.standard_normal((1, npw)) + 1j * gen.standard_normal((1, npw))
    bad /= np.linalg.norm(bad)
    r1 = oracle.realify(bad, np.array([0.0]), 1e-9)   # one complex vector: Re and Im give 2 directions
    assert r1.shape == (1, npw)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.realify(np.zeros((1, npw), complex), np.array([0.0]), 1e-9)


def test_real_flavor_chain_is_real_and_matches_complex_path():
    s = synth.make_system("rf", a=8.0, fft=12, ecut_wfn=4.0, ecut_eps=1.5, nv=3, nc=5, seed=31, real=True)
    assert s.cv.dtype == np.float64 and s.cc.dtype == np.float64
    md = oracle.mtxel_direct(s.gv, s.cv, s.gc, s.cc, s.geps)
    mf = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft)
    assert np.abs(md.imag).max() == 0.0                 # a sum of real products
    assert np.abs(mf.imag).max() < 1e-15 and np.abs(mf - md).max() < 1e-15
    r = oracle.solve(s)
    assert np.abs(r["chi"].imag).max() < 1e-15 and np.abs(r["epsinv"].imag).max() < 1e-15
    x = r["chi"].real
    assert np.array_equal(x, x.T) or np.abs(x - x.T).max() < 1e-16
    # the same bands as complex arrays give the same chain
    s.cv = s.cv.astype(np.complex128)
    s.cc = s.cc.astype(np.complex128)
    rc = oracle.solve(s)
    assert np.abs(rc["epsinv"] - r["epsinv"]).max() < 1e-14


# ------------------------------------------------------------------ static COHSEX / bare exchange

def _sigma_case(seed=3):
    s = synth.make_system("sg", a=8.0, fft=16, ecut_wfn=2.0, ecut_eps=1.0, nv=2, nc=4, seed=seed)
    gen = np.random.default_rng(seed)
    go = s.gc
    co = synth.orthonormal_bands(gen, go.shape[0], 3)
    return s, go, co


def test_sigma_ch_sum_over_complete_inner_basis_equals_closed_form():
    # Inner bands = every plane wave of a k-q sphere that holds all G2 - G
    # (radius sqrt(E_wfn) + sqrt(E_eps)): completeness turns the sum form of
    # Eq. cohsex-ch-sum into Eq. cohsex-ch-exact, whatever W is.
    s, go, co = _sigma_case()
    ecut_i = (math.sqrt(2.0) + math.sqrt(1.0)) ** 2 + 1e-9
    gi = synth.gsphere(s.bvec, -np.asarray(s.q_frac), ecut_i)
    ci = np.eye(gi.shape[0], dtype=np.complex128)
    gen = np.random.default_rng(8)
    z = gen.standard_normal((s.ng, s.ng)) + 1j * gen.standard_normal((s.ng, s.ng))
    ei = np.eye(s.ng) + 0.1 * (z + np.conj(z).T)                 # any Hermitian eps~^-1
    v = oracle.coulomb(s.bvec, s.q_frac, s.geps)
    out = oracle.sigma_cohsex(gi, ci, 0, go, co, s.geps, ei, v, s.omega)
    assert np.abs(out["CH"] - out["CH_exact"]).max() <= 1e-13 * np.abs(out["CH_exact"]).max()
    # a truncated inner set does not reach the closed form
    out2 = oracle.sigma_cohsex(gi, ci[:20], 0, go, co, s.geps, ei, v, s.omega)
    assert np.abs(out2["CH"] - out2["CH_exact"]).max() > 1e-3 * np.abs(out2["CH_exact"]).max()


def test_sigma_unscreened_limit_and_real_forms():
    s, go, co = _sigma_case(seed=4)
    sb = synth.sigma_bands(s, 3, 10, 4, seed=6)
    v = oracle.coulomb(s.bvec, s.q_frac, s.geps)
    # eps^-1 = 1: W = V, so SX is the bare exchange and CH vanishes
    out = oracle.sigma_cohsex(sb.gi, sb.ci, sb.nocc, sb.go, sb.co, s.geps, np.eye(s.ng), v, s.omega)
    assert np.allclose(out["SX"], out["X"], rtol=1e-13, atol=0)
    assert np.abs(out["CH"]).max() < 1e-15 and np.abs(out["CH_exact"]).max() < 1e-15
    assert np.all(out["X"] < 0)
    # screened: quadratic forms of Hermitian matrices are real; screening
    # weakens exchange (0 < eps~^-1 <= I gives |SX| <= |X|)
    r = oracle.solve(s)
    out = oracle.sigma_cohsex(sb.gi, sb.ci, sb.nocc, sb.go, sb.co, s.geps, r["epsinv"], r["v"], s.omega)
    for k in ("SX", "CH", "CH_exact"):
        assert np.abs(out[k].imag).max() <= 1e-14 * np.abs(out[k].real).max()
    assert np.all(np.abs(out["SX"].real) <= np.abs(out["X"]) + 1e-15)
    assert np.all(out["CH"].real <= 1e-15)                      # W - V <= 0


def test_sigma_mtxel_fft_route_and_negated_g():
    s, go, co = _sigma_case(seed=5)
    sb = synth.sigma_bands(s, 2, 5, 2, seed=7)
    md = oracle.sigma_mtxel(sb.gi, sb.ci, sb.go, sb.co, s.geps)
    mf = oracle.mtxel_fft(sb.gi, sb.ci, sb.go, sb.co, -s.geps, s.fft)
    assert np.abs(md - mf).max() < 1e-14
    # M_{n''n}(-q, -G) = conj(M_{n n''}(+q, +G)) with the roles of the spheres swapped
    mswap = oracle.mtxel_direct(sb.go, sb.co, sb.gi, sb.ci, s.geps).reshape(2, 5, -1)
    assert np.abs(md.reshape(5, 2, -1) - np.conj(mswap.transpose(1, 0, 2))).max() < 1e-14


def test_sigma_plane_wave_closed_forms_fix_the_prefactors():
    """Every inner and outer band one plane wave: M_{n''n}(-G) is 1 exactly
    when G = G_n - G_i (inner band at G_i on the k - q sphere) and 0 otherwise,
    so the four sums of Eqs. hf-x, cohsex-sx, cohsex-ch-sum and cohsex-ch-exact
    collapse to sums of single matrix entries at G = G_n - G_i:
      X  = -(1/Omega) sum_{i occ} v(q + G),   SX = -(1/Omega) sum_{i occ} W_GG,
      CH = (1/(2 Omega)) sum_{i all} (W - V)_GG,
    and rho_n(D) = delta_{D,0} gives CH_exact = (1/(2 Omega)) sum_{G in geps} (W - V)_GG.
    A dropped 1/2, a spin factor 2 or 4/Omega in place of 1/Omega fails."""
    s = _tiny(seed=21, n=16, a=9.0, ew=4.0, ee=3.0)
    v = oracle.coulomb(s.bvec, s.q_frac, s.geps)
    gen = np.random.default_rng(22)
    z = gen.standard_normal((s.ng, s.ng)) + 1j * gen.standard_normal((s.ng, s.ng))
    ei = np.eye(s.ng) + 0.05 * (z + np.conj(z).T)
    sq = np.sqrt(v)
    W = sq[:, None] * ei * sq[None, :]
    go = synth.gsphere(s.bvec, (0.0, 0.0, 0.0), 1.0)          # outer plane waves at k = 0
    gi = synth.gsphere(s.bvec, -np.asarray(s.q_frac), 1.2)    # inner plane waves at k - q
    co = np.eye(go.shape[0], dtype=np.complex128)[:3]
    ci = np.eye(gi.shape[0], dtype=np.complex128)
    nocc = gi.shape[0] // 2
    out = oracle.sigma_cohsex(gi, ci, nocc, go, co, s.geps, ei, v, s.omega)
    gidx = {tuple(g): k for k, g in enumerate(s.geps.tolist())}
    for n in range(3):
        x = sx = ch = 0.0
        for i in range(gi.shape[0]):
            k = gidx.get(tuple((go[n] - gi[i]).tolist()))
            if k is None:
                continue
            if i < nocc:
                x -= v[k] / s.omega
                sx -= W[k, k].real / s.omega
            ch += (W[k, k].real - v[k]) / (2.0 * s.omega)
        che = np.sum(np.diag(W).real - v) / (2.0 * s.omega)
        assert x < 0 and abs(out["X"][n] - x) <= 1e-13 * abs(x)
        assert abs(out["SX"][n] - sx) <= 1e-13 * abs(sx)
        assert abs(out["CH"][n] - ch) <= 1e-13 * abs(ch)
        assert abs(out["CH_exact"][n] - che) <= 1e-13 * abs(che)


def _heg_exchange(k, kf):
    """Hartree-Fock exchange of the electron gas for one spin (Hartree units):
    -(2 kF / pi) F(k / kF), F(x) = 1/2 + (1 - x^2)/(4x) ln|(1 + x)/(1 - x)|,
    F(0) = 1 (the textbook result, independent of the paper)."""
    x = k / kf
    if x == 0.0:
        return -2.0 * kf / math.pi
    return -(2.0 * kf / math.pi) * (0.5 + (1.0 - x * x) / (4.0 * x) * math.log(abs((1.0 + x) / (1.0 - x))))


def test_sigma_exchange_of_the_electron_gas():
    """The bare exchange of Eq. hf-x with the q sum's 1/(N_q Omega), for
    plane-wave states filling a Fermi sphere |k - q + G_i| < kF (the electron
    gas: one orbital per plane wave and spin) and averaged over a 2x2x2 grid
    of q in the zone, approaches the textbook Hartree-Fock exchange
    -(2 kF / pi) F(k / kF).  The discrete q grid misses the neighbourhood of
    the integrable 1/|k - k'|^2 point, so the sum lies a few per cent below
    in magnitude at this cell (12 bohr, kF = 1.5 bohr^-1); a spin factor 2, a
    dropped 1/Omega or 4/Omega would be off by 100 % or more."""
    a, kf, nq = 12.0, 1.5, 2
    bvec, omega = synth.cubic_cell(a)
    go = np.zeros((1, 3), dtype=np.int32)                     # outer state: k = 0, G = 0
    co = np.ones((1, 1), dtype=np.complex128)
    xs = []
    for i in range(nq):
        for j in range(nq):
            for k in range(nq):
                q = np.array([(i + 0.5) / nq - 0.5, (j + 0.5) / nq - 0.5, (k + 0.5) / nq - 0.5])
                gi = synth.gsphere(bvec, -q, kf * kf)
                ci = np.eye(gi.shape[0], dtype=np.complex128)
                geps = synth.gsphere(bvec, q, 4.0 * kf * kf * 1.0001)
                v = oracle.coulomb(bvec, q, geps)
                out = oracle.sigma_cohsex(gi, ci, gi.shape[0], go, co, geps, np.eye(geps.shape[0]), v, omega)
                xs.append(out["X"][0])
    x = float(np.mean(xs))
    ref = _heg_exchange(0.0, kf)
    assert -0.09 < x / ref - 1.0 < 0.0, (x, ref)


# ------------------------------------------------------------ direct pins of helpers

def test_density_diag_two_plane_wave_closed_form():
    """rho_n(D) = sum_G2 conj(c(D + G2)) c(G2) for a band of two plane waves a at G1,
    b at G2 (|a|^2 + |b|^2 = 1): 1 at D = 0, conj(a) b at G1 - G2, conj(b) a at G2 - G1,
    0 elsewhere; and rho(-D) = conj(rho(D)) for a random band."""
    g = np.array([[0, 0, 0], [1, 0, 0], [0, 2, -1], [1, 1, 1]], dtype=np.int32)
    a, b = 0.6 * np.exp(0.3j), 0.8 * np.exp(-1.1j)
    c = np.zeros((1, 4), dtype=np.complex128)
    c[0, 1], c[0, 2] = a, b
    d12 = g[1] - g[2]
    deltas = np.array([[0, 0, 0], d12, -d12, [1, 0, 0], [0, 1, 0]], dtype=np.int32)
    rho = oracle.density_diag(g, c, deltas)[0]
    assert abs(rho[0] - 1.0) < 1e-15
    assert abs(rho[1] - np.conj(a) * b) < 1e-15
    assert abs(rho[2] - np.conj(b) * a) < 1e-15
    assert np.abs(rho[3:]).max() < 1e-15
    gen = np.random.default_rng(4)
    s = _tiny(seed=11)
    cr = synth.orthonormal_bands(gen, s.gc.shape[0], 2)
    dd = np.array([[1, 0, 0], [0, -1, 2], [2, 1, 0]], dtype=np.int32)
    p = oracle.density_diag(s.gc, cr, dd)
    m = oracle.density_diag(s.gc, cr, -dd)
    assert np.abs(p - np.conj(m)).max() < 1e-14
    assert np.abs(oracle.density_diag(s.gc, cr, np.zeros((1, 3), np.int32))[:, 0] - 1.0).max() < 1e-14


def test_chi_entries_are_the_entries_of_chi():
    """chi_entries on column subsets of M equals those entries of the tier-1 pair
    sum and the tier-2 product."""
    gen = np.random.default_rng(5)
    M = gen.standard_normal((12, 9)) + 1j * gen.standard_normal((12, 9))
    w = -gen.uniform(0.1, 2.0, 12)
    full1 = oracle.chi_direct(M, w, 37.0)
    full2 = oracle.chi(M, w, 37.0)
    rows, cols = [0, 3, 8], [1, 2, 3, 7]
    sub = oracle.chi_entries(M[:, rows], M[:, cols], w, 37.0)
    assert np.abs(sub - full1[np.ix_(rows, cols)]).max() <= 1e-13 * np.abs(full1).max()
    assert np.abs(sub - full2[np.ix_(rows, cols)]).max() <= 1e-13 * np.abs(full2).max()


def test_eps_sym_special_cases_and_similarity():
    """eps~ = I - v^1/2 chi v^1/2: the identity for chi = 0, 1 - v_G chi_GG on a
    diagonal chi, and V^-1/2 eps V^1/2 with eps = I - v chi the paper's asymmetric
    form (same spectrum)."""
    gen = np.random.default_rng(6)
    ng = 7
    v = gen.uniform(0.2, 3.0, ng)
    assert np.array_equal(oracle.eps_sym(np.zeros((ng, ng), np.complex128), v), np.eye(ng))
    d = -gen.uniform(0.0, 1.0, ng)
    e = oracle.eps_sym(np.diag(d).astype(np.complex128), v)
    assert np.abs(e - np.diag(1.0 - v * d)).max() < 1e-15
    z = gen.standard_normal((ng, ng)) + 1j * gen.standard_normal((ng, ng))
    chi = -(z @ np.conj(z).T) / ng
    es = oracle.eps_sym(chi, v)
    ea = oracle.eps_asym(chi, v)
    s = np.sqrt(v)
    assert np.abs(es - (ea * s[None, :]) / s[:, None]).max() < 1e-13
    assert np.allclose(np.sort(np.linalg.eigvalsh(es)), np.sort(np.linalg.eigvals(ea).real), atol=1e-12)
