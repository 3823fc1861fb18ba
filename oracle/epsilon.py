"""Oracle arithmetic for one q-point of the RPA epsilon path (test infrastructure).

Notation follows the BerkeleyGW paper, Section "RPA Dielectric Matrix:
epsilon":

* Eq. (eqn_matrix_elem): M_nn'(k,q,G) = <n k+q| e^{i(q+G).r} |n' k>, the
  occupied band n on the q-shifted sphere, the empty band n' at k (= 0 here).
* Unnumbered equation after it: M = FFT^-1( phi*_{n,k+q}(r) phi_{n',k}(r) ).
* Eq. (eqn_static_xi): chi_GG'(q;0) = sum_v sum_c M*_vc(G) M_vc(G') / (E_v - E_c),
  with the 4/Omega prefactor (1/Omega from the implicit division by the
  super-cell volume in Section "Major Sections of the Code", with N_k = 1; 2
  for spin; 2 for the two time orderings).
* Eq. (eqn_static_xi_compact): the same sum as one matrix product over the
  composite pair index.
* Eq. (epsilon) and Eq. (untruncated_bare_coulomb): eps = delta - v chi,
  v(q+G) = 4 pi / |q+G|^2 (Hartree atomic units); the symmetrized form uses
  v^{1/2} on both sides (the paper's symmetric Coulomb alternative).
* Eq. (screened_interaction): W_GG' = eps^-1_GG' v(q+G').
* Eq. (retarded_advanced_epsilon) at E = i omega, delta -> 0: the pair weight
  becomes Delta / (Delta^2 + omega^2), Delta = E_v - E_c.
* Eq. (retarded_advanced_epsilon) on the real axis with broadening delta: complex
  weights, a non-Hermitian chi and eps~ (inverted with pivoting); the
  frequency grid of Fig. (frequency_grid).

Pair index p = v * nc + c (valence-major).  All floating point is float64 /
complex128.  G lists are integer triples in reciprocal-lattice units; FFT
indices are G mod n.
"""
from __future__ import annotations

import math
import os
from typing import Optional, Sequence

import numpy as np

try:  # scipy's pocketfft takes a thread count; numpy's does not.
    import scipy.fft as _sfft
except Exception:  # pragma: no cover
    _sfft = None


def _workers() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except Exception:  # pragma: no cover
        return os.cpu_count() or 1


def _ifftn(a, axes):
    if _sfft is not None:
        return _sfft.ifftn(a, axes=axes, workers=_workers())
    return np.fft.ifftn(a, axes=axes)


# ---------------------------------------------------------------------------
# Matrix elements, Eq. (eqn_matrix_elem)
# ---------------------------------------------------------------------------

def mtxel_direct(gv: np.ndarray, cv: np.ndarray, gc: np.ndarray, cc: np.ndarray,
                 geps: np.ndarray) -> np.ndarray:
    """Tier 1: M_vc(G) as the plane-wave convolution (the definition).

    With psi_{n k}(r) = Omega^{-1/2} sum_G c_n(G) e^{i(k+G).r} and the occupied
    band at k+q, the integral in Eq. (eqn_matrix_elem) keeps the terms with
    G_v = G + G_c, so M_vc(G) = sum_{G_c in S_c} conj(c_v(G + G_c)) c_c(G_c),
    with c_v(X) = 0 for X outside the valence sphere.  Returns complex128
    [nv * nc][ng], pair-major.
    """
    gv = np.asarray(gv, dtype=np.int64)
    gc = np.asarray(gc, dtype=np.int64)
    geps = np.asarray(geps, dtype=np.int64)
    nv, nc, ng = cv.shape[0], cc.shape[0], geps.shape[0]
    # Dense lookup of valence coefficient index by G over a bounding box.
    lo = gv.min(axis=0)
    hi = gv.max(axis=0)
    shape = tuple((hi - lo + 1).tolist())
    lut = -np.ones(shape, dtype=np.int64)
    lut[tuple((gv - lo).T)] = np.arange(gv.shape[0])
    cv_pad = np.concatenate([cv, np.zeros((nv, 1), dtype=cv.dtype)], axis=1)
    out = np.empty((nv, nc, ng), dtype=np.complex128)
    for ig in range(ng):
        x = gc + geps[ig] - lo
        inside = np.all((x >= 0) & (x < np.array(shape)), axis=1)
        idx = np.full(gc.shape[0], gv.shape[0], dtype=np.int64)  # -> zero column
        xi = x[inside]
        look = lut[tuple(xi.T)]
        idx[inside] = np.where(look >= 0, look, gv.shape[0])
        cvg = cv_pad[:, idx]                      # c_v(G + G_c), [nv][npw_c]
        out[:, :, ig] = np.conj(cvg) @ cc.T       # sum over G_c
    return out.reshape(nv * nc, ng)


def band_grids(g: np.ndarray, c: np.ndarray, n: int) -> np.ndarray:
    """u_b(r_j) = sum_G c_b(G) e^{+2 pi i G.j/n} on the n^3 grid (unnormalized):
    the bands in real space, the first step of the FFT form of the matrix
    elements (the unnumbered equation after Eq. eqn_matrix_elem).

    Returns complex128 [nb][n][n][n] indexed [b][jx][jy][jz].
    """
    nb = c.shape[0]
    grid = np.zeros((nb, n, n, n), dtype=np.complex128)
    gm = np.mod(np.asarray(g, dtype=np.int64), n)
    grid[:, gm[:, 0], gm[:, 1], gm[:, 2]] = c
    return _ifftn(grid, axes=(1, 2, 3)) * float(n ** 3)


def mtxel_fft_pairs(gv, cv, gc, cc, geps, n: int, pairs: Sequence[int]) -> np.ndarray:
    """Tier 2 (the FFT form after Eq. eqn_matrix_elem, as in mtxel_fft) for a
    subset of pairs p = v*nc + c (rows of M in that order)."""
    nc = cc.shape[0]
    pairs = np.asarray(pairs, dtype=np.int64)
    vs = np.unique(pairs // nc)
    cs = np.unique(pairs % nc)
    uv = band_grids(gv, cv[vs], n)
    uc = band_grids(gc, cc[cs], n)
    vpos = {int(v): i for i, v in enumerate(vs)}
    cpos = {int(c): i for i, c in enumerate(cs)}
    gm = np.mod(np.asarray(geps, dtype=np.int64), n)
    out = np.empty((pairs.size, geps.shape[0]), dtype=np.complex128)
    for i, p in enumerate(pairs):
        prod = np.conj(uv[vpos[int(p // nc)]]) * uc[cpos[int(p % nc)]]
        f = _ifftn(prod, axes=(0, 1, 2))
        out[i] = f[gm[:, 0], gm[:, 1], gm[:, 2]]
    return out


def mtxel_fft(gv: np.ndarray, cv: np.ndarray, gc: np.ndarray, cc: np.ndarray,
              geps: np.ndarray, n: int) -> np.ndarray:
    """Tier 2: M via the FFT of the real-space product (paper, after Eq. eqn_matrix_elem).

    M_vc(G) = (1/N_r) sum_j conj(u_v(r_j)) u_c(r_j) e^{+2 pi i G.j/n}, i.e. the
    inverse DFT (numpy's ifftn convention) of the product, read at G mod n.
    Exact (no aliasing) when n > max|G_v| + max|G_c| + max|G_eps| per axis.
    Returns complex128 [nv * nc][ng].
    """
    nv, nc = cv.shape[0], cc.shape[0]
    uv = band_grids(gv, cv, n)
    uc = band_grids(gc, cc, n)
    gm = np.mod(np.asarray(geps, dtype=np.int64), n)
    out = np.empty((nv, nc, geps.shape[0]), dtype=np.complex128)
    for v in range(nv):
        prod = np.conj(uv[v])[None] * uc
        f = _ifftn(prod, axes=(1, 2, 3))
        out[v] = f[:, gm[:, 0], gm[:, 1], gm[:, 2]]
    return out.reshape(nv * nc, geps.shape[0])


# ---------------------------------------------------------------------------
# Polarizability, Eq. (eqn_static_xi) / (eqn_static_xi_compact)
# ---------------------------------------------------------------------------

def chi_weights(ev: np.ndarray, ec: np.ndarray, omega: Optional[float] = None) -> np.ndarray:
    """Pair weights w_p, p = v*nc + c.

    Static (Eq. eqn_static_xi): w = 1 / (E_v - E_c).
    Imaginary frequency (Eq. retarded_advanced_epsilon at E = i omega,
    delta -> 0): (1/2)[1/(D - i w) + 1/(D + i w)] = D / (D^2 + w^2).
    """
    d = (np.asarray(ev, dtype=np.float64)[:, None] - np.asarray(ec, dtype=np.float64)[None, :]).ravel()
    if omega is None:
        return 1.0 / d
    return d / (d * d + float(omega) ** 2)


def chi_direct(M: np.ndarray, w: np.ndarray, cell_volume: float) -> np.ndarray:
    """Tier 1: explicit pair sum chi_GG' = (4/Omega) sum_p w_p conj(M_p(G)) M_p(G')."""
    ng = M.shape[1]
    out = np.zeros((ng, ng), dtype=np.complex128)
    for p in range(M.shape[0]):
        out += w[p] * np.outer(np.conj(M[p]), M[p])
    return out * (4.0 / cell_volume)


def chi(M: np.ndarray, w: np.ndarray, cell_volume: float) -> np.ndarray:
    """Tier 2: one matrix product over the composite pair index (Eq. eqn_static_xi_compact)."""
    return (4.0 / cell_volume) * (np.conj(M).T @ (w[:, None] * M))


def chi_entries(M_rows_g: np.ndarray, M_rows_gp: np.ndarray, w: np.ndarray,
                cell_volume: float) -> np.ndarray:
    """Eq. eqn_static_xi_compact restricted to given G (columns of M_rows_g)
    and G' (columns of M_rows_gp), with the 4/Omega of chi."""
    return (4.0 / cell_volume) * (np.conj(M_rows_g).T @ (w[:, None] * M_rows_gp))


# ---------------------------------------------------------------------------
# Real flavor (Section "Real and complex flavors")
# ---------------------------------------------------------------------------

def realify(c: np.ndarray, energies: np.ndarray, tol: float, rank_tol: float = 1e-8) -> np.ndarray:
    """Real coefficients from complex ones of states with inversion and
    time-reversal symmetry, as the paper prescribes: bands whose energies lie
    within tol of their neighbour form a degenerate subspace of n states; the
    2n vectors Re c_1, Im c_1, Re c_2, Im c_2, ... are orthonormalized in that
    order by Gram-Schmidt (a vector whose remainder is below rank_tol of its
    norm is dropped) and the first n kept.  A non-degenerate state (n = 1)
    thereby loses its global phase.  Raises if a subspace yields fewer than
    n independent real vectors."""
    c = np.asarray(c, dtype=np.complex128)
    e = np.asarray(energies, dtype=np.float64)
    nb = c.shape[0]
    out = np.zeros(c.shape, dtype=np.float64)
    start = 0
    while start < nb:
        stop = start + 1
        while stop < nb and abs(e[stop] - e[stop - 1]) <= tol:
            stop += 1
        n = stop - start
        basis = []
        for b in range(start, stop):
            for v in (c[b].real, c[b].imag):
                r = v.copy()
                for q in basis:
                    r -= (q @ r) * q
                nr = np.linalg.norm(r)
                if nr > rank_tol * max(np.linalg.norm(v), 1e-300):
                    basis.append(r / nr)
        if len(basis) < n:
            raise np.linalg.LinAlgError(f"bands {start}..{stop - 1}: only {len(basis)} real directions")
        out[start:stop] = np.array(basis[:n])
        start = stop
    return out


# ---------------------------------------------------------------------------
# Real-axis ("full-frequency") response, Eq. (retarded_advanced_epsilon)
# ---------------------------------------------------------------------------

def chi_weights_real(ev: np.ndarray, ec: np.ndarray, energy, delta: float,
                     advanced: bool = False) -> np.ndarray:
    """Complex pair weights of Eq. retarded_advanced_epsilon at frequency E.

    w_p = (1/2) [1/(D - E - s i delta) + 1/(D + E + s i delta)], D = E_v - E_c,
    s = +1 for the retarded function (upper signs), -1 for the advanced one.
    `energy` may be complex: E = i omega with delta = 0 gives the imaginary-axis
    weight D / (D^2 + omega^2) of chi_weights.
    """
    d = (np.asarray(ev, dtype=np.float64)[:, None] - np.asarray(ec, dtype=np.float64)[None, :]).ravel()
    s = -1.0 if advanced else 1.0
    e = complex(energy)
    return 0.5 * (1.0 / (d - e - s * 1j * delta) + 1.0 / (d + e + s * 1j * delta))


def frequency_grid(spacing: float, low_cutoff: float, high_cutoff: float, increment: float) -> np.ndarray:
    """Real-frequency grid of Section "RPA Dielectric Matrix: epsilon" (Fig.
    frequency_grid): 0, spacing, 2 spacing, ... while <= low_cutoff; after the
    last uniform point every step is `increment` longer than the one before,
    while the frequency stays <= high_cutoff.  Points k*spacing are formed by
    multiplication; a relative slack of 1e-12 absorbs rounding at the cutoffs.
    """
    if not (spacing > 0 and increment >= 0 and 0 <= low_cutoff <= high_cutoff):
        raise ValueError("need spacing > 0, increment >= 0, 0 <= low <= high")
    tol = 1e-12
    pts = []
    k = 0
    while k * spacing <= low_cutoff * (1 + tol) + tol:
        pts.append(k * spacing)
        k += 1
    e = pts[-1]
    step = spacing
    while True:
        step += increment
        e = e + step
        if e > high_cutoff * (1 + tol) + tol:
            break
        pts.append(e)
    return np.array(pts, dtype=np.float64)


# ---------------------------------------------------------------------------
# Dielectric matrix and its inverse, Eqs. (epsilon), (untruncated_bare_coulomb)
# ---------------------------------------------------------------------------

def coulomb(bvec: np.ndarray, q_frac: Sequence[float], geps: np.ndarray, model: str = "bulk",
            rc: float = 0.0) -> np.ndarray:
    """v(q+G) with q+G in Cartesian bohr^-1 (rows of bvec are b_i).

    bulk (Eq. untruncated_bare_coulomb): 4 pi / k^2.
    sphere (Section "Coulomb Interaction", spherical truncation at r_c):
        4 pi / k^2 (1 - cos(r_c k)), finite at k = 0 (limit 2 pi r_c^2).
    slab (same Section, truncation at z_c along the slab normal z):
        4 pi / k^2 (1 - exp(-k_xy z_c) cos(k_z z_c)), divergent at k = 0.

    The brackets are evaluated through the identities 1 - cos x = 2 sin^2(x/2)
    and 1 - e^-a cos b = -expm1(-a) + e^-a 2 sin^2(b/2), whose terms are all
    non-negative, so small r_c k loses no digits to cancellation.
    """
    k = (np.asarray(geps, dtype=np.float64) + np.asarray(q_frac, dtype=np.float64)) @ np.asarray(bvec, dtype=np.float64)
    k2 = np.einsum("ij,ij->i", k, k)
    if model == "sphere":
        v = np.empty_like(k2)
        nz = k2 > 0.0
        kk = np.sqrt(k2[nz])
        v[nz] = 4.0 * math.pi / k2[nz] * (2.0 * np.sin(0.5 * rc * kk) ** 2)
        v[~nz] = 2.0 * math.pi * rc * rc
        return v
    if np.any(k2 == 0.0):
        raise ValueError("q+G = 0: the Coulomb factor diverges for this model")
    if model == "bulk":
        return 4.0 * math.pi / k2
    if model == "slab":
        kxy = np.sqrt(k[:, 0] ** 2 + k[:, 1] ** 2)
        bracket = -np.expm1(-kxy * rc) + np.exp(-kxy * rc) * 2.0 * np.sin(0.5 * k[:, 2] * rc) ** 2
        return 4.0 * math.pi / k2 * bracket
    raise ValueError(f"unknown Coulomb model {model}")


def eps_sym(chi_m: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Symmetrized eps~ = I - v^{1/2} chi v^{1/2}."""
    s = np.sqrt(v)
    return np.eye(chi_m.shape[0], dtype=np.complex128) - s[:, None] * chi_m * s[None, :]


def eps_asym(chi_m: np.ndarray, v: np.ndarray) -> np.ndarray:
    """The paper's asymmetric eps_GG' = delta_GG' - v(q+G) chi_GG' (Eq. epsilon)."""
    return np.eye(chi_m.shape[0], dtype=np.complex128) - v[:, None] * chi_m


def screened_w(epsinv_asym: np.ndarray, v: np.ndarray) -> np.ndarray:
    """W_GG' = eps^-1_GG' v(q+G') (Eq. screened_interaction)."""
    return epsinv_asym * v[None, :]


def screened_w_sym(epsinv_sym: np.ndarray, v: np.ndarray) -> np.ndarray:
    """The same W from the symmetrized inverse: W = V^{1/2} eps~^-1 V^{1/2}."""
    s = np.sqrt(v)
    return s[:, None] * epsinv_sym * s[None, :]


def inv_gauss_jordan(a: np.ndarray) -> np.ndarray:
    """Tier 1 inverse: Gauss-Jordan elimination with partial pivoting, complex128.

    The pivot is the largest |a| in the column at or below the diagonal; ties go
    to the lowest row index.  The paper inverts with LAPACK ZGESV; the inverse
    is unique, pivoting changes only the rounding.
    """
    n = a.shape[0]
    aug = np.concatenate([np.array(a, dtype=np.complex128), np.eye(n, dtype=np.complex128)], axis=1)
    for k in range(n):
        piv = k + int(np.argmax(np.abs(aug[k:, k])))
        if aug[piv, k] == 0:
            raise np.linalg.LinAlgError("singular matrix")
        if piv != k:
            aug[[k, piv]] = aug[[piv, k]]
        aug[k] = aug[k] / aug[k, k]
        col = aug[:, k].copy()
        col[k] = 0.0
        aug -= col[:, None] * aug[k][None, :]
    return aug[:, n:]


def inv(a: np.ndarray) -> np.ndarray:
    """Tier 2 inverse: library LU (numpy.linalg.inv; the paper inverts eps
    with LAPACK's ZGESV, Section "RPA Dielectric Matrix: epsilon")."""
    return np.linalg.inv(a)


def epsinv_sym(chi_m: np.ndarray, v: np.ndarray, tier: int = 2):
    """eps~ and eps~^-1 from chi and v."""
    e = eps_sym(chi_m, v)
    return e, (inv_gauss_jordan(e) if tier == 1 else inv(e))


# ---------------------------------------------------------------------------
# Static COHSEX and bare exchange, Eqs. (cohsex-sx), (cohsex-ch-sum),
# (cohsex-ch-exact), (hf-x): diagonal elements for one q
# ---------------------------------------------------------------------------

def sigma_mtxel(g_inner, c_inner, g_outer, c_outer, geps) -> np.ndarray:
    """M_{n''n}(k, -q, -G) = <n'' k-q| e^{-i(q+G).r} |n k> for G in geps, the
    inner band n'' on the k-q sphere: sum_{G2} conj(c_n''(G2 - G)) c_n(G2).
    Returns [n_inner * n_outer][ng], pair p = n'' * n_outer + n."""
    return mtxel_direct(g_inner, c_inner, g_outer, c_outer, -np.asarray(geps))


def density_diag(g_outer, c_outer, deltas) -> np.ndarray:
    """rho_n(D) = M_nn(k, q = 0, D) = sum_{G2} conj(c_n(D + G2)) c_n(G2), [n][len(deltas)]:
    the band density of Eq. cohsex-ch-exact, the matrix element of Eq.
    eqn_matrix_elem of a band with itself at q = 0."""
    out = np.empty((c_outer.shape[0], len(deltas)), dtype=np.complex128)
    for n in range(c_outer.shape[0]):
        out[n] = mtxel_direct(g_outer, c_outer[n:n + 1], g_outer, c_outer[n:n + 1], deltas)[0]
    return out


def sigma_cohsex(g_inner, c_inner, nocc: int, g_outer, c_outer, geps, epsinv_sym_m, v, cell_volume: float):
    """Diagonal <n|Sigma|n> for one q (Hartree), with W = eps^-1 v = V^1/2
    eps~^-1 V^1/2 and the implicit 1/Omega of a q sum (one q point):
      X       = -(1/Omega) sum_{n'' occ} sum_G |M(G)|^2 v(q+G)               (hf-x)
      SX      = -(1/Omega) sum_{n'' occ} M^H W M                             (cohsex-sx)
      CH      = (1/(2 Omega)) sum_{n'' all inner} M^H (W - V) M              (cohsex-ch-sum)
      CH_exact = (1/(2 Omega)) sum_{G G'} rho_n(G - G') (W - V)_{G G'}       (cohsex-ch-exact)
    with M = M_{n''n}(k, -q, -G) and rho_n(D) = <n| e^{i D.r} |n>.  Eq.
    cohsex-ch-exact prints the argument as G' - G; the bra-ket it stands for,
    <n| e^{i(G - G').r} |n'>, and the completeness relation applied to the
    sum form both give G - G' in the convention of Eq. eqn_matrix_elem (the
    pin on a complete inner basis checks it).  Returns dict of [n_outer]
    arrays."""
    no = c_outer.shape[0]
    ni = c_inner.shape[0]
    M = sigma_mtxel(g_inner, c_inner, g_outer, c_outer, geps).reshape(ni, no, -1)
    s = np.sqrt(v)
    W = s[:, None] * epsinv_sym_m * s[None, :]
    WmV = W - np.diag(v)
    qW = np.einsum("abg,gh,abh->ab", np.conj(M), W, M)
    qV = np.einsum("abg,g,abg->ab", np.conj(M), v, M)
    qWV = np.einsum("abg,gh,abh->ab", np.conj(M), WmV, M)
    geps = np.asarray(geps, dtype=np.int64)
    diffs = (geps[:, None, :] - geps[None, :, :]).reshape(-1, 3)       # [G][G'] -> G - G'
    uniq, inv_idx = np.unique(diffs, axis=0, return_inverse=True)
    rho = density_diag(g_outer, c_outer, uniq.astype(np.int32))[:, inv_idx.ravel()].reshape(no, len(geps), len(geps))
    ch_exact = np.einsum("ngh,gh->n", rho, WmV) / (2.0 * cell_volume)
    return dict(X=-qV[:nocc].sum(0).real / cell_volume,
                SX=-qW[:nocc].sum(0) / cell_volume,
                CH=qWV.sum(0) / (2.0 * cell_volume),
                CH_exact=ch_exact)


def solve_real(system, energies: Sequence[float], delta: float, advanced: bool = False,
               model: str = "bulk", rc: float = 0.0):
    """Real-axis chain for one q-point (Eq. retarded_advanced_epsilon in the
    symmetric Coulomb form): per frequency E, chi^{r/a}(E), eps~ = I - V^1/2
    chi V^1/2 (no longer Hermitian) and its inverse by an LU with partial
    pivoting.  Returns dict(M, chi[f], eps[f], epsinv[f], v)."""
    M = mtxel_fft(system.gv, system.cv, system.gc, system.cc, system.geps, system.fft)
    v = coulomb(system.bvec, system.q_frac, system.geps, model, rc)
    xs, es, eis = [], [], []
    for e in energies:
        x = chi(M, chi_weights_real(system.ev, system.ec, e, delta, advanced), system.omega)
        ee, ei = epsinv_sym(x, v)
        xs.append(x)
        es.append(ee)
        eis.append(ei)
    return dict(M=M, chi=np.array(xs), eps=np.array(es), epsinv=np.array(eis), v=v)


def solve(system, omega: Optional[float] = None, tier: int = 2, model: str = "bulk", rc: float = 0.0):
    """Whole chain for one q-point: returns dict(M, chi, eps, epsinv, v)."""
    if tier == 1:
        M = mtxel_direct(system.gv, system.cv, system.gc, system.cc, system.geps)
    else:
        M = mtxel_fft(system.gv, system.cv, system.gc, system.cc, system.geps, system.fft)
    w = chi_weights(system.ev, system.ec, omega)
    x = chi_direct(M, w, system.omega) if tier == 1 else chi(M, w, system.omega)
    v = coulomb(system.bvec, system.q_frac, system.geps, model, rc)
    e, ei = epsinv_sym(x, v, tier=tier)
    return dict(M=M, chi=x, eps=e, epsinv=ei, v=v)
