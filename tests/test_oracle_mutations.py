"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake in the oracle (a replaced function,
in-process and on the CPU only, restored afterwards) and runs every pin of
``test_oracle_pins.py`` but the slow electron-gas one; at least one pin must
fail.  The mistakes are the kinds that would let the oracle and a kernel
agree on a wrong answer: a dropped or misplaced conjugate, a wrong transform
sign or scale, a dropped prefactor, a wrong weight or pair order, v in place
of v^{1/2}, q dropped from v, a missing row swap, a wrong frequency grid or
sign convention, a wrong Sigma prefactor.
"""
import contextlib
import importlib.util
import inspect
import itertools
import os

import numpy as np
import pytest

import oracle
from oracle import epsilon as E

_PINS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "test_oracle_pins.py")
_SLOW = {"test_sigma_exchange_of_the_electron_gas"}


def _load_pins():
    spec = importlib.util.spec_from_file_location("oracle_pins_for_mutations", _PINS_PATH)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _pin_calls(mod):
    """Every (name, function, kwargs) of the pin module, parametrizations expanded."""
    calls = []
    for name, fn in sorted(vars(mod).items()):
        if not name.startswith("test_") or not callable(fn) or name in _SLOW:
            continue
        grids = []
        for mark in getattr(fn, "pytestmark", []):
            if mark.name != "parametrize":
                continue
            names, values = mark.args[0], mark.args[1]
            names = [n.strip() for n in names.split(",")] if isinstance(names, str) else list(names)
            rows = [v if len(names) > 1 else (v,) for v in values]
            grids.append([dict(zip(names, r)) for r in rows])
        params = set(inspect.signature(fn).parameters)
        for combo in itertools.product(*grids) if grids else [()]:
            kw = {}
            for d in combo:
                kw.update(d)
            if set(kw) == params:
                calls.append((name, fn, kw))
    return calls


@contextlib.contextmanager
def _planted(name, fn):
    """Replace oracle function `name` in the module and in the package namespace."""
    saved = [(m, getattr(m, name)) for m in (E, oracle) if hasattr(m, name)]
    try:
        for m, _ in saved:
            setattr(m, name, fn)
        yield
    finally:
        for m, f in saved:
            setattr(m, name, f)


# ---------------------------------------------------------------- the mistakes

def _mtxel_fft_no_conj(gv, cv, gc, cc, geps, n):
    nv, nc = cv.shape[0], cc.shape[0]
    uv, uc = E.band_grids(gv, cv, n), E.band_grids(gc, cc, n)
    gm = np.mod(np.asarray(geps, dtype=np.int64), n)
    out = np.empty((nv, nc, geps.shape[0]), dtype=np.complex128)
    for v in range(nv):
        f = np.fft.ifftn(uv[v][None] * uc, axes=(1, 2, 3))
        out[v] = f[:, gm[:, 0], gm[:, 1], gm[:, 2]]
    return out.reshape(nv * nc, -1)


def _mtxel_fft_forward_sign(gv, cv, gc, cc, geps, n):
    nv, nc = cv.shape[0], cc.shape[0]
    uv, uc = E.band_grids(gv, cv, n), E.band_grids(gc, cc, n)
    gm = np.mod(np.asarray(geps, dtype=np.int64), n)
    out = np.empty((nv, nc, geps.shape[0]), dtype=np.complex128)
    for v in range(nv):
        f = np.fft.fftn(np.conj(uv[v])[None] * uc, axes=(1, 2, 3)) / n ** 3
        out[v] = f[:, gm[:, 0], gm[:, 1], gm[:, 2]]
    return out.reshape(nv * nc, -1)


def _mtxel_direct_conj_other(gv, cv, gc, cc, geps):
    # sum_Gc c_v(G + G_c) conj(c_c(G_c)): the conjugate of the right sum
    return np.conj(_ORIG["mtxel_direct"](gv, cv, gc, cc, geps))


def _band_grids_unscaled(g, c, n):
    return _ORIG["band_grids"](g, c, n) / float(n ** 3)


def _chi_transposed(M, w, cell_volume):
    return (4.0 / cell_volume) * (M.T @ (w[:, None] * np.conj(M)))


def _chi_no_prefactor(M, w, cell_volume):
    return np.conj(M).T @ (w[:, None] * M)


def _chi_direct_no_prefactor(M, w, cell_volume):
    return _ORIG["chi_direct"](M, w, cell_volume) * (cell_volume / 4.0)


def _weights_sign(ev, ec, omega=None):
    return -_ORIG["chi_weights"](ev, ec, omega)


def _weights_two_delta(ev, ec, omega=None):
    w = _ORIG["chi_weights"](ev, ec, omega)
    return w if omega is None else 2.0 * w


def _weights_pair_order(ev, ec, omega=None):
    return _ORIG["chi_weights"](ev, ec, omega).reshape(len(ev), len(ec)).T.ravel()


def _coulomb_no_q(bvec, q_frac, geps, model="bulk", rc=0.0):
    return _ORIG["coulomb"](bvec, np.zeros(3), geps, model, rc)


def _coulomb_sphere_argument(bvec, q_frac, geps, model="bulk", rc=0.0):
    return _ORIG["coulomb"](bvec, q_frac, geps, model, 2.0 * rc if model == "sphere" else rc)


def _eps_sym_v(chi_m, v):
    return np.eye(chi_m.shape[0], dtype=np.complex128) - v[:, None] * chi_m * v[None, :]


def _gauss_jordan_no_swap(a):
    n = a.shape[0]
    aug = np.concatenate([np.array(a, dtype=np.complex128), np.eye(n, dtype=np.complex128)], axis=1)
    for k in range(n):
        if aug[k, k] == 0:
            raise np.linalg.LinAlgError("zero pivot")
        aug[k] = aug[k] / aug[k, k]
        col = aug[:, k].copy()
        col[k] = 0.0
        aug -= col[:, None] * aug[k][None, :]
    return aug[:, n:]


def _weights_real_no_advanced(ev, ec, energy, delta, advanced=False):
    return _ORIG["chi_weights_real"](ev, ec, energy, delta, False)


def _grid_constant_steps(spacing, low_cutoff, high_cutoff, increment):
    pts = list(np.arange(0.0, low_cutoff * (1 + 1e-12) + 1e-12, spacing))
    e = pts[-1]
    while e + spacing + increment <= high_cutoff * (1 + 1e-12) + 1e-12:
        e += spacing + increment
        pts.append(e)
    return np.array(pts)


def _sigma_ch_prefactor(*args, **kw):
    out = dict(_ORIG["sigma_cohsex"](*args, **kw))
    out["CH"] = 2.0 * out["CH"]
    out["CH_exact"] = 2.0 * out["CH_exact"]
    return out


def _sigma_x_sign(*args, **kw):
    out = dict(_ORIG["sigma_cohsex"](*args, **kw))
    out["X"] = -out["X"]
    return out


def _sigma_sx_screening_dropped(g_inner, c_inner, nocc, g_outer, c_outer, geps, epsinv_sym_m, v, cell_volume):
    return _ORIG["sigma_cohsex"](g_inner, c_inner, nocc, g_outer, c_outer, geps,
                                 np.eye(len(v), dtype=np.complex128), v, cell_volume)


def _slab_normal_x(bvec, q_frac, geps, model="bulk", rc=0.0):
    if model != "slab":
        return _ORIG["coulomb"](bvec, q_frac, geps, model, rc)
    perm = np.asarray(bvec, dtype=np.float64)[:, [2, 1, 0]]   # the slab normal taken along x
    return _ORIG["coulomb"](perm, q_frac, geps, model, rc)


def _w_v_on_the_left(epsinv_asym, v):
    return v[:, None] * epsinv_asym


def _eps_asym_v_on_the_right(chi_m, v):
    return np.eye(chi_m.shape[0], dtype=np.complex128) - chi_m * v[None, :]


def _sigma_mtxel_plus_g(g_inner, c_inner, g_outer, c_outer, geps):
    return _ORIG["mtxel_direct"](g_inner, c_inner, g_outer, c_outer, np.asarray(geps))


def _density_reversed(g_outer, c_outer, deltas):
    return _ORIG["density_diag"](g_outer, c_outer, -np.asarray(deltas))


def _broadening_sign(ev, ec, energy, delta, advanced=False):
    return _ORIG["chi_weights_real"](ev, ec, energy, -delta, advanced)


def _pairs_c_major(gv, cv, gc, cc, geps, n, pairs):
    nv, nc = cv.shape[0], cc.shape[0]
    pairs = np.asarray(pairs, dtype=np.int64)
    swapped = (pairs % nv) * nc + (pairs // nv) % nc
    return _ORIG["mtxel_fft_pairs"](gv, cv, gc, cc, geps, n, swapped)


def _realify_real_parts(c, energies, tol, rank_tol=1e-8):
    r = np.asarray(c).real.copy()
    return r / np.linalg.norm(r, axis=1, keepdims=True)


_ORIG = {n: getattr(E, n) for n in ("mtxel_direct", "band_grids", "chi_direct", "chi_weights", "coulomb",
                                     "chi_weights_real", "sigma_cohsex", "density_diag", "mtxel_fft_pairs")}

MISTAKES = {
    "product without the conjugate": [("mtxel_fft", _mtxel_fft_no_conj)],
    "forward FFT sign on the product": [("mtxel_fft", _mtxel_fft_forward_sign)],
    "convolution conjugates the other band": [("mtxel_direct", _mtxel_direct_conj_other)],
    "band grids without the n^3 scale": [("band_grids", _band_grids_unscaled)],
    "chi conjugated on the other index": [("chi", _chi_transposed)],
    "chi without 4/Omega": [("chi", _chi_no_prefactor), ("chi_direct", _chi_direct_no_prefactor)],
    "weight sign flipped": [("chi_weights", _weights_sign)],
    "frequency weight doubled": [("chi_weights", _weights_two_delta)],
    "pair order transposed": [("chi_weights", _weights_pair_order)],
    "q dropped from v": [("coulomb", _coulomb_no_q)],
    "sphere truncation argument doubled": [("coulomb", _coulomb_sphere_argument)],
    "v in place of v^1/2": [("eps_sym", _eps_sym_v)],
    "Gauss-Jordan without row swaps": [("inv_gauss_jordan", _gauss_jordan_no_swap)],
    "advanced weights as retarded": [("chi_weights_real", _weights_real_no_advanced)],
    "frequency steps not growing": [("frequency_grid", _grid_constant_steps)],
    "Coulomb hole without the 1/2": [("sigma_cohsex", _sigma_ch_prefactor)],
    "exchange sign flipped": [("sigma_cohsex", _sigma_x_sign)],
    "screened exchange unscreened": [("sigma_cohsex", _sigma_sx_screening_dropped)],
    "slab normal along x": [("coulomb", _slab_normal_x)],
    "W with v on the wrong side": [("screened_w", _w_v_on_the_left)],
    "asymmetric eps with v on the right": [("eps_asym", _eps_asym_v_on_the_right)],
    "Sigma matrix elements at +G": [("sigma_mtxel", _sigma_mtxel_plus_g)],
    "band density at G' - G": [("density_diag", _density_reversed)],
    "broadening with the wrong sign": [("chi_weights_real", _broadening_sign)],
    "sampled pairs read conduction-major": [("mtxel_fft_pairs", _pairs_c_major)],
    "real flavour from the real parts alone": [("realify", _realify_real_parts)],
}


def test_every_pin_passes_unplanted():
    mod = _load_pins()
    calls = _pin_calls(mod)
    assert len(calls) >= 40
    for name, fn, kw in calls:
        fn(**kw)


@pytest.mark.parametrize("mistake", sorted(MISTAKES))
def test_planted_mistake_fails_a_pin(mistake):
    mod = _load_pins()
    caught = []
    with contextlib.ExitStack() as stack:
        for name, fn in MISTAKES[mistake]:
            stack.enter_context(_planted(name, fn))
        for name, fn, kw in _pin_calls(mod):
            try:
                with np.errstate(all="ignore"):
                    fn(**kw)
            except Exception:   # an assertion or an error the mistake provokes
                caught.append(name)
    assert caught, f"no pin fails with the planted mistake: {mistake}"
