"""Seeded synthetic inputs for the RPA epsilon path.

This module only *generates inputs*: integer G-vector lists on cutoff spheres,
orthonormal random plane-wave coefficients, sorted band energies, frequency
grids and request streams.  It holds none of the method's arithmetic (no
matrix elements, no polarizability, no Coulomb factor, no inversion), so both
the CPU oracle (through the tests) and the CUDA path can consume the same
arrays.

Conventions (BerkeleyGW paper, Appendix "Specification of file formats"):
G vectors are integer triples in reciprocal-lattice units, listed as a full
sphere; coefficients of each band are normalized so that the sum of their
squared magnitudes is one.  Cutoffs are in Rydberg, i.e. |k|^2 in bohr^-2.
Energies are in Hartree.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np

# Sub-seed order for one system (one base seed per configuration):
# valence coefficients, conduction coefficients, E_v, E_c, subblock, arrivals,
# the band set and the momentum matrix of a small-q system.
_STREAMS = ("cv", "cc", "ev", "ec", "subblock", "arrivals", "bands", "kp")


def cubic_cell(a: float):
    """Simple cubic cell of side a (bohr): reciprocal vectors (rows, bohr^-1) and volume."""
    b = 2.0 * math.pi / a
    bvec = np.eye(3) * b
    return bvec, a ** 3


def gsphere(bvec: np.ndarray, kfrac: Sequence[float], ecut: float) -> np.ndarray:
    """All integer G with |(G + k) . B|^2 < ecut (strict, FP64).

    Ordered by |(G+k)B|^2 ascending, ties broken lexicographically on
    (Gx, Gy, Gz).  Lengths that are equal in exact arithmetic (G vectors
    related by a symmetry of the cell) can differ in their last bits
    depending on the order of the floating-point sum, which differs between
    machines; lengths within a relative 1e-9 of their predecessor therefore
    count as ties, so the order -- and every input drawn in that order -- is
    the same on every machine.  Returns int32 [n][3].
    """
    bvec = np.asarray(bvec, dtype=np.float64)
    kf = np.asarray(kfrac, dtype=np.float64)
    radius = math.sqrt(ecut)
    # Bound each integer component: |G_i + k_i| <= radius * |a_i| / 2pi where
    # a_i is the real-space vector dual to b_i.  Use the inverse of B.
    binv = np.linalg.inv(bvec)  # columns: a_i / (2 pi) ... rows of B^-1
    lim = [int(math.ceil(radius * np.linalg.norm(binv[:, i]) + abs(kf[i]))) + 1 for i in range(3)]
    rng = [np.arange(-l, l + 1) for l in lim]
    gx, gy, gz = np.meshgrid(*rng, indexing="ij")
    g = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    kc = (g + kf) @ bvec
    e = np.einsum("ij,ij->i", kc, kc)
    keep = e < ecut
    g, e = g[keep], e[keep]
    by_len = np.argsort(e, kind="stable")
    es = e[by_len]
    tie_group = np.concatenate([[0], np.cumsum(np.diff(es) > 1e-9 * np.maximum(es[1:], 1e-300))])
    gs = g[by_len]
    order = by_len[np.lexsort((gs[:, 2], gs[:, 1], gs[:, 0], tie_group))]
    return np.ascontiguousarray(g[order].astype(np.int32))


def orthonormal_bands(gen: np.random.Generator, npw: int, nb: int) -> np.ndarray:
    """nb orthonormal coefficient vectors of length npw, band-major [nb][npw].

    Real and imaginary parts are i.i.d. N(0,1); the reduced QR of the
    [npw x nb] matrix gives the bands as Q's columns.
    """
    if nb > npw:
        raise ValueError(f"cannot orthonormalize {nb} bands on {npw} plane waves")
    a = gen.standard_normal((npw, nb)) + 1j * gen.standard_normal((npw, nb))
    q, _ = np.linalg.qr(a)
    return np.ascontiguousarray(q.T.astype(np.complex128))


def gauss_legendre_frequencies(nfreq: int, lo: float = 0.0, hi: float = 2.0) -> np.ndarray:
    """nfreq Gauss-Legendre nodes mapped linearly from [-1, 1] to [lo, hi] (Ha)."""
    x, _ = np.polynomial.legendre.leggauss(nfreq)
    return (lo + (x + 1.0) * 0.5 * (hi - lo)).astype(np.float64)


@dataclasses.dataclass
class System:
    """One q-point problem: everything bgw_mtxel/bgw_chi_sum/bgw_epsinv consume."""
    name: str
    a: float
    bvec: np.ndarray      # [3][3] rows b1,b2,b3 (bohr^-1)
    omega: float          # cell volume (bohr^3)
    q_frac: np.ndarray    # [3] crystal coordinates
    fft: int              # cubic FFT grid n
    gv: np.ndarray        # int32 [npw_v][3] valence sphere (|q+G|^2 < ecut_wfn)
    gc: np.ndarray        # int32 [npw_c][3] conduction sphere (|G|^2 < ecut_wfn)
    geps: np.ndarray      # int32 [ng][3] epsilon sphere (|q+G|^2 < ecut_eps)
    cv: np.ndarray        # complex128 [nv][npw_v]
    cc: np.ndarray        # complex128 [nc][npw_c]
    ev: np.ndarray        # float64 [nv] Ha, ascending
    ec: np.ndarray        # float64 [nc] Ha, ascending
    seed: int = 0

    @property
    def nv(self):
        return self.cv.shape[0]

    @property
    def nc(self):
        return self.cc.shape[0]

    @property
    def ng(self):
        return self.geps.shape[0]

    @property
    def npairs(self):
        return self.nv * self.nc


def orthonormal_real_bands(gen: np.random.Generator, npw: int, nb: int) -> np.ndarray:
    """nb real orthonormal coefficient vectors of length npw (real flavor):
    i.i.d. N(0,1) entries, reduced QR, bands as Q's columns."""
    if nb > npw:
        raise ValueError(f"cannot orthonormalize {nb} bands on {npw} plane waves")
    q, _ = np.linalg.qr(gen.standard_normal((npw, nb)))
    return np.ascontiguousarray(q.T.astype(np.float64))


def make_system(name: str, a: float, fft: int, ecut_wfn: float, ecut_eps: float,
                nv: int, nc: int, seed: int, q_frac=(0.1, 0.0, 0.0),
                ev_range=(-0.5, 0.0), ec_range=(0.04, 1.5), real: bool = False) -> System:
    """Build one seeded system with the recipe of the benchmark configurations.
    real = True draws real coefficients (the real flavor: inversion and
    time-reversal symmetry allow real wavefunctions in reciprocal space)."""
    bvec, omega = cubic_cell(a)
    q = np.asarray(q_frac, dtype=np.float64)
    gv = gsphere(bvec, q, ecut_wfn)
    gc = gsphere(bvec, (0.0, 0.0, 0.0), ecut_wfn)
    geps = gsphere(bvec, q, ecut_eps)
    ss = np.random.SeedSequence(seed).spawn(len(_STREAMS))
    gens = {k: np.random.Generator(np.random.PCG64(s)) for k, s in zip(_STREAMS, ss)}
    bands = orthonormal_real_bands if real else orthonormal_bands
    cv = bands(gens["cv"], gv.shape[0], nv)
    cc = bands(gens["cc"], gc.shape[0], nc)
    ev = np.sort(gens["ev"].uniform(ev_range[0], ev_range[1], nv))
    ec = np.sort(gens["ec"].uniform(ec_range[0], ec_range[1], nc))
    return System(name=name, a=a, bvec=bvec, omega=omega, q_frac=q, fft=fft, gv=gv, gc=gc,
                  geps=geps, cv=cv, cc=cc, ev=ev, ec=ec, seed=seed)


def q0_system(name: str, a: float, fft: int, ecut_wfn: float, ecut_eps: float, nv: int, nc: int,
              seed: int, q_frac=(0.001, 0.0, 0.0), p_scale: float = 0.5,
              ev_range=(-0.5, 0.0), ec_range=(0.04, 1.5)) -> System:
    """A system at a small q0 (the q -> 0 limit of Section "RPA Dielectric
    Matrix: epsilon" is taken at q0 about 1/1000 of the zone on a shifted grid).

    The occupied bands at k + q0 are not independent of the empty bands at k
    as in make_system: one orthonormal set on the k sphere gives the empty
    bands u_c and the unshifted occupied bands u_v, and the shifted occupied
    bands follow first-order k.p perturbation theory,
        u_v(k + q0) = u_v + |q0| sum_c P_vc / (E_v - E_c) u_c,
    re-orthonormalized, with a seeded complex momentum matrix P (entries of
    scale p_scale).  The head M_vc(G = 0) = <u_v(k + q0)|u_c> is then O(|q0|)
    and v(q0) chi_00 stays finite as q0 -> 0, as it does for an insulator.
    The coefficients are moved onto the k + q0 sphere by G vector (zero for a
    G the shifted sphere gains).
    """
    bvec, omega = cubic_cell(a)
    q = np.asarray(q_frac, dtype=np.float64)
    qlen = float(np.linalg.norm(q @ bvec))
    gv = gsphere(bvec, q, ecut_wfn)
    gc = gsphere(bvec, (0.0, 0.0, 0.0), ecut_wfn)
    geps = gsphere(bvec, q, ecut_eps)
    ss = np.random.SeedSequence(seed).spawn(len(_STREAMS))
    gens = {k: np.random.Generator(np.random.PCG64(s)) for k, s in zip(_STREAMS, ss)}
    u = orthonormal_bands(gens["bands"], gc.shape[0], nv + nc)
    uv, cc = u[:nv], np.ascontiguousarray(u[nv:])
    ev = np.sort(gens["ev"].uniform(ev_range[0], ev_range[1], nv))
    ec = np.sort(gens["ec"].uniform(ec_range[0], ec_range[1], nc))
    pm = p_scale * (gens["kp"].standard_normal((nv, nc)) + 1j * gens["kp"].standard_normal((nv, nc))) / math.sqrt(2)
    shifted = uv + qlen * ((pm / (ev[:, None] - ec[None, :])) @ cc)
    qq, _ = np.linalg.qr(shifted.T)
    on_k = qq.T
    index = {tuple(g): i for i, g in enumerate(gc.tolist())}
    cv = np.zeros((nv, gv.shape[0]), dtype=np.complex128)
    for j, g in enumerate(gv.tolist()):
        i = index.get(tuple(g))
        if i is not None:
            cv[:, j] = on_k[:, i]
    return System(name=name, a=a, bvec=bvec, omega=omega, q_frac=q, fft=fft, gv=gv, gc=gc,
                  geps=geps, cv=np.ascontiguousarray(cv), cc=cc, ev=ev, ec=ec, seed=seed)


# Benchmark configurations: plain FP64 oracle-sized (c0), plain FP64 larger cell
# (c1), mixed-precision large cell (c2).  Base seeds are fixed per configuration.
CONFIGS: Dict[str, dict] = {
    "c0": dict(a=10.26, fft=20, ecut_wfn=10.0, ecut_eps=3.0, nv=4, nc=60, seed=1000),
    "c1": dict(a=20.52, fft=40, ecut_wfn=12.0, ecut_eps=6.0, nv=32, nc=800, seed=1001),
    "c2": dict(a=30.78, fft=60, ecut_wfn=12.0, ecut_eps=6.0, nv=108, nc=3000, seed=1002),
}


def config_system(name: str, **overrides) -> System:
    p = dict(CONFIGS[name])
    p.update(overrides)
    return make_system(name, **p)


def scramble_phases(c: np.ndarray, groups: Sequence[Sequence[int]], seed: int) -> np.ndarray:
    """Complex coefficients as a plane-wave code returns them for real-flavor
    states: every band times a random global phase, and every listed
    degenerate group mixed by a random unitary matrix (the states of a
    degenerate subspace need not be eigenstates of inversion)."""
    gen = np.random.Generator(np.random.PCG64(seed))
    out = np.asarray(c, dtype=np.complex128) * np.exp(2j * np.pi * gen.uniform(size=c.shape[0]))[:, None]
    for g in groups:
        g = list(g)
        z = gen.standard_normal((len(g), len(g))) + 1j * gen.standard_normal((len(g), len(g)))
        u, _ = np.linalg.qr(z)
        out[g] = u @ out[g]
    return np.ascontiguousarray(out)


@dataclasses.dataclass
class SigmaBands:
    """Bands of a diagonal Sigma evaluation at one q: the outer bands n at k
    (k = 0 sphere) and the inner bands n'' at k - q (sphere at -q), the first
    nocc inner bands occupied."""
    go: np.ndarray
    co: np.ndarray
    gi: np.ndarray
    ci: np.ndarray
    nocc: int


def sigma_bands(system: System, n_outer: int, n_inner: int, nocc: int, seed: int) -> SigmaBands:
    """Seeded orthonormal outer and inner bands on the spheres of a system's
    cell and wavefunction cutoff (the cutoff read back from the system's
    conduction sphere)."""
    ecut = float(np.max(np.einsum("ij,ij->i", system.gc @ system.bvec, system.gc @ system.bvec))) + 1e-9
    go = gsphere(system.bvec, (0.0, 0.0, 0.0), ecut)
    gi = gsphere(system.bvec, -np.asarray(system.q_frac), ecut)
    gen = np.random.Generator(np.random.PCG64(seed))
    co = orthonormal_bands(gen, go.shape[0], n_outer)
    ci = orthonormal_bands(gen, gi.shape[0], n_inner)
    return SigmaBands(go=go, co=co, gi=gi, ci=ci, nocc=nocc)


def batched_q_systems(nq: int = 8, seed: int = 1003) -> List[System]:
    """The c1 cell at q = (0.05 j, 0, 0), j = 1..nq: uneven epsilon spheres."""
    out = []
    for j in range(1, nq + 1):
        out.append(make_system(f"c3_q{j}", a=20.52, fft=40, ecut_wfn=12.0, ecut_eps=6.0,
                               nv=32, nc=800, seed=seed + j, q_frac=(0.05 * j, 0.0, 0.0)))
    return out


def subblock_indices(ng: int, size: int, seed: int) -> np.ndarray:
    """Seeded principal-subblock indices (distinct, sorted)."""
    ss = np.random.SeedSequence(seed).spawn(len(_STREAMS))
    gen = np.random.Generator(np.random.PCG64(ss[_STREAMS.index("subblock")]))
    return np.sort(gen.permutation(ng)[:size])


def serve_requests(n: int = 200, seed: int = 1004):
    """Request mix of the served stream: scale s, eps cutoff, band counts.

    N_c is drawn uniform in [50, 1500] and clamped to the number of conduction
    plane waves available at the 10 Ry wavefunction cutoff.
    """
    gen = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for i in range(n):
        s = int(gen.integers(1, 4))
        e = float(gen.choice([3.0, 4.0, 6.0]))
        nc_draw = int(gen.integers(50, 1501))
        reqs.append(dict(index=i, s=s, ecut_eps=e, nv=4 * s ** 3, nc_draw=nc_draw,
                         seed=seed * 1000 + i))
    return reqs


def serve_systems(reqs, seed: int = 1004) -> List[System]:
    """Systems of a served stream built from one band set per cell scale s:
    the valence bands (N_v = 4 s^3) and the conduction bands of a request
    are the first N_v and N_c columns of one QR-orthonormalized Gaussian
    matrix per s (the first columns of Q depend only on the first columns of
    the matrix, so each request's bands are exactly those its own QR would
    give for that matrix), and every request draws its own energies from its
    seed.  Requests of one scale therefore share coefficient values, which
    keeps a stream of hundreds of requests cheap to generate; shapes and
    distributions are those of request_system."""
    masters = {}
    out = []
    q = (0.1, 0.0, 0.0)
    for r in reqs:
        sc = r["s"]
        if sc not in masters:
            a = 10.26 * sc
            bvec, omega = cubic_cell(a)
            gv = gsphere(bvec, q, 10.0)
            gc = gsphere(bvec, (0.0, 0.0, 0.0), 10.0)
            gen = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, sc])))
            cv = orthonormal_bands(gen, gv.shape[0], 4 * sc ** 3)
            cc = orthonormal_bands(gen, gc.shape[0], min(1500, gc.shape[0]))
            masters[sc] = (a, bvec, omega, gv, gc, cv, cc, {})
        a, bvec, omega, gv, gc, cv, cc, eps_spheres = masters[sc]
        e = r["ecut_eps"]
        if e not in eps_spheres:
            eps_spheres[e] = gsphere(bvec, q, e)
        nc = min(r["nc_draw"], cc.shape[0])
        ss = np.random.SeedSequence(r["seed"]).spawn(len(_STREAMS))
        gens = {k: np.random.Generator(np.random.PCG64(x)) for k, x in zip(_STREAMS, ss)}
        ev = np.sort(gens["ev"].uniform(-0.5, 0.0, cv.shape[0]))
        ec = np.sort(gens["ec"].uniform(0.04, 1.5, nc))
        out.append(System(name=f"req{r['index']}", a=a, bvec=bvec, omega=omega, q_frac=np.asarray(q), fft=20 * sc,
                          gv=gv, gc=gc, geps=eps_spheres[e], cv=cv, cc=cc[:nc], ev=ev, ec=ec, seed=r["seed"]))
    return out


def request_system(req: dict) -> System:
    s = req["s"]
    a = 10.26 * s
    bvec, _ = cubic_cell(a)
    npw_c = gsphere(bvec, (0, 0, 0), 10.0).shape[0]
    nc = min(req["nc_draw"], npw_c)
    return make_system(f"req{req['index']}", a=a, fft=20 * s, ecut_wfn=10.0,
                       ecut_eps=req["ecut_eps"], nv=req["nv"], nc=nc, seed=req["seed"])
