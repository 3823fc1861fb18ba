"""Thin Python binding of libbgw.so (include/bgw.h), argument marshalling only.

Every step of the path runs in the library's CUDA kernels; this module turns
torch tensors into pointers, host numpy arrays into C arrays, and status
codes into exceptions.  The library must have been built (``build()`` in
``__graft_entry__`` or ``python paper_1111_4429_gb300/_build.py``); there is
no fallback when it is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbgw.so")

BGW_OK, BGW_EINVAL, BGW_ENOMEM, BGW_ECUDA, BGW_ETIMEOUT, BGW_ENUMERIC, BGW_EBUSY, BGW_ECANCELED, \
    BGW_EUNSUPPORTED = range(9)
BGW_PREC_FP64, BGW_PREC_MIX_FP16, BGW_PREC_MIX_BF16 = 0, 1, 2
PREC = {"fp64": BGW_PREC_FP64, "mix_fp16": BGW_PREC_MIX_FP16, "mix_bf16": BGW_PREC_MIX_BF16}

# Every symbol include/bgw.h declares.
EXPORTS = ("bgw_create", "bgw_destroy", "bgw_last_error", "bgw_sync", "bgw_mem_stats", "bgw_launch_count",
           "bgw_graph_stats",
           "bgw_mtxel",
           "bgw_set_option", "bgw_timing_report", "bgw_chi_sum", "bgw_epsinv", "bgw_epsinv_noalloc", "bgw_screened_w",
           "bgw_chi_sum_real", "bgw_epsinv_general", "bgw_epsilon_real", "bgw_frequency_grid",
           "bgw_epsinv_rflavor", "bgw_real_coefficients", "bgw_sigma_cohsex",
           "bgw_epsilon",
           "bgw_epsilon_batch", "bgw_serve_open", "bgw_serve_submit", "bgw_serve_poll", "bgw_serve_cancel",
           "bgw_serve_close")
BGW_OPT_CHI_SEGMENT_PAIRS, BGW_OPT_TIMING, BGW_OPT_AUTOTUNE, BGW_OPT_CHI_CHUNK_PAIRS, BGW_OPT_INVERSE = 1, 2, 3, 4, 5
BGW_OPT_HEAD = 6
BGW_OPT_SIGMA_DENSITY = 7
BGW_OPT_UPDATE_SLICES = 8
BGW_OPT_DOUBLE_FP32 = 9
BGW_OPT_WAIT_LIMIT_NS = 10
BGW_OPT_PAIR_KERNEL = 11
BGW_OPT_UPDATE_ITEMS = 12
BGW_FLAVOR_REAL = 0x100
BGW_COULOMB_BULK, BGW_COULOMB_SPHERE, BGW_COULOMB_SLAB = 0, 1, 2
COULOMB_MODELS = {"bulk": BGW_COULOMB_BULK, "sphere": BGW_COULOMB_SPHERE, "slab": BGW_COULOMB_SLAB}


class BgwError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bgw error {code}: {msg}")
        self.code = code


class Cell(ctypes.Structure):
    _fields_ = [("bvec", (ctypes.c_double * 3) * 3), ("omega", ctypes.c_double),
                ("q_frac", ctypes.c_double * 3), ("fft", ctypes.c_int * 3),
                ("coulomb", ctypes.c_int), ("coulomb_cut", ctypes.c_double)]


class Problem(ctypes.Structure):
    _fields_ = [("cell", Cell),
                ("nv", ctypes.c_int), ("npw_v", ctypes.c_int), ("gv", ctypes.POINTER(ctypes.c_int32)),
                ("cv", ctypes.c_void_p), ("ev", ctypes.POINTER(ctypes.c_double)),
                ("nc", ctypes.c_int), ("npw_c", ctypes.c_int), ("gc", ctypes.POINTER(ctypes.c_int32)),
                ("cc", ctypes.c_void_p), ("ec", ctypes.POINTER(ctypes.c_double)),
                ("ng", ctypes.c_int), ("geps", ctypes.POINTER(ctypes.c_int32))]


class ServeOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_int), ("prec", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("problem", Problem), ("epsinv_out", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("hbm_bytes", ctypes.c_uint64)]


def make_cell(bvec, omega: float, q_frac, n: int, coulomb: str = "bulk", cut: float = 0.0) -> Cell:
    c = Cell()
    c.coulomb = COULOMB_MODELS[coulomb]
    c.coulomb_cut = float(cut)
    b = np.asarray(bvec, dtype=np.float64)
    for i in range(3):
        for j in range(3):
            c.bvec[i][j] = float(b[i, j])
        c.q_frac[i] = float(q_frac[i])
        c.fft[i] = int(n)
    c.omega = float(omega)
    return c


def system_cell(s, coulomb: str = "bulk", cut: float = 0.0) -> Cell:
    return make_cell(s.bvec, s.omega, s.q_frac, s.fft, coulomb, cut)


_lib = None


def load() -> ctypes.CDLL:
    """Load libbgw.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it first (python paper_1111_4429_gb300/_build.py)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32p, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)
    cellp = ctypes.POINTER(Cell)
    ci = ctypes.c_int
    lib.bgw_create.argtypes = [ctypes.POINTER(vp), ci, ctypes.c_uint64]
    lib.bgw_destroy.argtypes = [vp]
    lib.bgw_last_error.argtypes = [vp]
    lib.bgw_last_error.restype = ctypes.c_char_p
    lib.bgw_sync.argtypes = [vp, vp]
    lib.bgw_mem_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    lib.bgw_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.bgw_graph_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    lib.bgw_set_option.argtypes = [vp, ci, ctypes.c_int64]
    lib.bgw_timing_report.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t, ci]
    lib.bgw_mtxel.argtypes = [vp, cellp, ci, ci, i32p, vp, ci, ci, i32p, vp, ci, i32p, ci, vp, vp]
    lib.bgw_chi_sum.argtypes = [vp, cellp, ci, ci, ci, vp, dp, dp, ci, dp, ci, ci, vp, vp]
    lib.bgw_epsinv.argtypes = [vp, ci, cellp, ctypes.POINTER(ci), ctypes.POINTER(i32p), ctypes.POINTER(vp),
                               ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    lib.bgw_epsinv_noalloc.argtypes = [cellp, ci, i32p, vp, vp, vp, vp]
    lib.bgw_epsilon_batch.argtypes = [vp, ci, ctypes.POINTER(Problem), ci, dp, ci, ctypes.POINTER(vp), vp]
    lib.bgw_serve_open.argtypes = [vp, ctypes.POINTER(ServeOpts), ctypes.POINTER(vp)]
    lib.bgw_serve_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    lib.bgw_serve_poll.argtypes = [vp, ctypes.c_uint64, ci, ctypes.POINTER(Result)]
    lib.bgw_serve_cancel.argtypes = [vp, ctypes.c_uint64]
    lib.bgw_serve_close.argtypes = [vp]
    lib.bgw_epsilon.argtypes = [vp, cellp, ci, ci, i32p, vp, dp, ci, ci, i32p, vp, dp, ci, i32p, ci, dp, ci,
                                ci, vp, vp, vp]
    cd = ctypes.c_double
    lib.bgw_screened_w.argtypes = [vp, ci, cellp, ctypes.POINTER(ci), ctypes.POINTER(i32p), ctypes.POINTER(vp),
                                   ctypes.POINTER(vp), vp]
    lib.bgw_chi_sum_real.argtypes = [vp, cellp, ci, ci, ci, vp, dp, dp, ci, dp, cd, ci, ci, ci, vp, vp]
    lib.bgw_epsinv_general.argtypes = [vp, ci, cellp, ctypes.POINTER(ci), ctypes.POINTER(i32p), ctypes.POINTER(vp),
                                       ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    lib.bgw_epsilon_real.argtypes = [vp, cellp, ci, ci, i32p, vp, dp, ci, ci, i32p, vp, dp, ci, i32p, ci, dp, cd,
                                     ci, ci, ci, vp, vp, vp]
    lib.bgw_frequency_grid.argtypes = [cd, cd, cd, cd, ci, dp, ctypes.POINTER(ci)]
    lib.bgw_epsinv_rflavor.argtypes = lib.bgw_epsinv.argtypes
    lib.bgw_real_coefficients.argtypes = [ci, ci, vp, dp, cd, dp]
    lib.bgw_sigma_cohsex.argtypes = [vp, cellp, ci, ci, i32p, vp, ci, ci, i32p, vp, ci, ci, i32p, vp, ci, dp, vp]
    for name in EXPORTS:
        getattr(lib, name).restype = ctypes.c_char_p if name == "bgw_last_error" else ctypes.c_int
    _lib = lib
    return lib


def _i32(a: np.ndarray):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ptr(t) -> Optional[int]:
    """Address of a torch tensor or numpy array (host or device), or None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def epsinv_noalloc(cell: Cell, geps, chi, eps, epsinv, stream=None) -> None:
    """bgw_epsinv_noalloc: the inverse of one matrix with no device allocation
    (scratch in a fixed array inside the library; ng <= 4096; current device)."""
    lib = load()
    ge_, gep = _i32(geps)
    rc = lib.bgw_epsinv_noalloc(ctypes.byref(cell), ge_.shape[0], gep, _ptr(chi), _ptr(eps), _ptr(epsinv),
                                _stream(stream))
    if rc != BGW_OK:
        raise BgwError(rc, "bgw_epsinv_noalloc failed")


def real_coefficients(c: np.ndarray, energies, tol: float) -> np.ndarray:
    """bgw_real_coefficients: real-flavor coefficients (host only)."""
    lib = load()
    cz = np.ascontiguousarray(c, dtype=np.complex128)
    e = np.ascontiguousarray(energies, dtype=np.float64)
    out = np.zeros(cz.shape, dtype=np.float64)
    rc = lib.bgw_real_coefficients(cz.shape[0], cz.shape[1], cz.ctypes.data, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   ctypes.c_double(tol), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != BGW_OK:
        raise BgwError(rc, "bgw_real_coefficients failed")
    return out


def frequency_grid(spacing: float, low_cutoff: float, high_cutoff: float, increment: float) -> np.ndarray:
    """bgw_frequency_grid: the paper's real-frequency grid (host only)."""
    lib = load()
    n = ctypes.c_int(0)
    args = [ctypes.c_double(spacing), ctypes.c_double(low_cutoff), ctypes.c_double(high_cutoff),
            ctypes.c_double(increment)]
    rc = lib.bgw_frequency_grid(*args, 0, None, ctypes.byref(n))
    if rc != BGW_OK:
        raise BgwError(rc, "bgw_frequency_grid: bad parameters")
    out = np.zeros(n.value, dtype=np.float64)
    rc = lib.bgw_frequency_grid(*args, n.value, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                ctypes.byref(n))
    if rc != BGW_OK:
        raise BgwError(rc, "bgw_frequency_grid failed")
    return out


class Context:
    """One bgw_ctx on one device (see include/bgw.h)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.lib = load()
        self.device = device
        h = ctypes.c_void_p()
        rc = self.lib.bgw_create(ctypes.byref(h), device, hbm_budget_bytes)
        if rc != BGW_OK:
            raise BgwError(rc, f"bgw_create failed on device {device}")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.bgw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != BGW_OK:
            raise BgwError(rc, self.lib.bgw_last_error(self.h).decode())

    def sync(self, stream=None):
        self._check(self.lib.bgw_sync(self.h, _stream(stream)))

    def mem_stats(self):
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self.lib.bgw_mem_stats(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def launch_count(self) -> int:
        a = ctypes.c_uint64()
        self._check(self.lib.bgw_launch_count(self.h, ctypes.byref(a)))
        return a.value

    def graph_stats(self):
        """(graphs held, replays so far): bgw_graph_stats."""
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self.lib.bgw_graph_stats(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_option(self, option: int, value: int):
        self._check(self.lib.bgw_set_option(self.h, option, value))

    def timing_report(self, reset: bool = True) -> dict:
        import json
        buf = ctypes.create_string_buffer(4096)
        self._check(self.lib.bgw_timing_report(self.h, buf, len(buf), int(bool(reset))))
        return {k: (int(v[0]), float(v[1])) for k, v in json.loads(buf.value.decode()).items()}

    def mtxel(self, cell: Cell, gv, cv, gc, cc, geps, prec: int, M, stream=None):
        gv_, gvp = _i32(gv)
        gc_, gcp = _i32(gc)
        ge_, gep = _i32(geps)
        self._check(self.lib.bgw_mtxel(self.h, ctypes.byref(cell), cv.shape[0], gv_.shape[0], gvp, _ptr(cv),
                                       cc.shape[0], gc_.shape[0], gcp, _ptr(cc), ge_.shape[0], gep, prec,
                                       _ptr(M), _stream(stream)))
        return M

    def chi_sum(self, cell: Cell, nv: int, nc: int, ng: int, M, ev, ec, omega, prec: int, accumulate: bool,
                chi, stream=None):
        ev_, evp = _f64(ev)
        ec_, ecp = _f64(ec)
        om_, omp = _f64(omega)
        nfreq = 0 if om_ is None else om_.shape[0]
        self._check(self.lib.bgw_chi_sum(self.h, ctypes.byref(cell), nv, nc, ng, _ptr(M), evp, ecp, nfreq, omp,
                                         prec, int(bool(accumulate)), _ptr(chi), _stream(stream)))
        return chi

    def epsinv(self, cells: Sequence[Cell], gepss: Sequence[np.ndarray], chis, eps, epsinvs, stream=None):
        n = len(cells)
        carr = (Cell * n)(*cells)
        keep = [_i32(g) for g in gepss]
        ng = (ctypes.c_int * n)(*[k[0].shape[0] for k in keep])
        gp = (ctypes.POINTER(ctypes.c_int32) * n)(*[k[1] for k in keep])
        cp = (ctypes.c_void_p * n)(*[_ptr(x) for x in chis])
        ep = None if eps is None else (ctypes.c_void_p * n)(*[_ptr(x) for x in eps])
        ip = (ctypes.c_void_p * n)(*[_ptr(x) for x in epsinvs])
        self._check(self.lib.bgw_epsinv(self.h, n, carr, ng, gp, cp, ep, ip, _stream(stream)))
        return epsinvs

    def chi_sum_real(self, cell: Cell, nv: int, nc: int, ng: int, M, ev, ec, energy, delta: float,
                     advanced: bool, prec: int, accumulate: bool, chi, stream=None):
        ev_, evp = _f64(ev)
        ec_, ecp = _f64(ec)
        e_, ep = _f64(energy)
        self._check(self.lib.bgw_chi_sum_real(self.h, ctypes.byref(cell), nv, nc, ng, _ptr(M), evp, ecp,
                                              e_.shape[0], ep, ctypes.c_double(delta), int(advanced), prec,
                                              int(accumulate), _ptr(chi), _stream(stream)))
        return chi

    def epsinv_general(self, cells: Sequence[Cell], gepss: Sequence[np.ndarray], chis, eps, epsinvs, stream=None):
        n = len(cells)
        carr = (Cell * n)(*cells)
        keep = [_i32(g) for g in gepss]
        ng = (ctypes.c_int * n)(*[k[0].shape[0] for k in keep])
        gp = (ctypes.POINTER(ctypes.c_int32) * n)(*[k[1] for k in keep])
        cp = (ctypes.c_void_p * n)(*[_ptr(x) for x in chis])
        ep = None if eps is None else (ctypes.c_void_p * n)(*[_ptr(x) for x in eps])
        ip = (ctypes.c_void_p * n)(*[_ptr(x) for x in epsinvs])
        self._check(self.lib.bgw_epsinv_general(self.h, n, carr, ng, gp, cp, ep, ip, _stream(stream)))
        return epsinvs

    def epsilon_real(self, cell: Cell, gv, cv, ev, gc, cc, ec, geps, energy, delta: float, advanced: bool,
                     prec: int, nc_chunk: int, chi, epsinv, stream=None):
        gv_, gvp = _i32(gv)
        gc_, gcp = _i32(gc)
        ge_, gep = _i32(geps)
        ev_, evp = _f64(ev)
        ec_, ecp = _f64(ec)
        e_, ep = _f64(energy)
        self._check(self.lib.bgw_epsilon_real(self.h, ctypes.byref(cell), cv.shape[0], gv_.shape[0], gvp, _ptr(cv),
                                              evp, cc.shape[0], gc_.shape[0], gcp, _ptr(cc), ecp, ge_.shape[0], gep,
                                              e_.shape[0], ep, ctypes.c_double(delta), int(advanced), prec, nc_chunk,
                                              _ptr(chi), _ptr(epsinv), _stream(stream)))
        return epsinv

    def epsinv_rflavor(self, cells: Sequence[Cell], gepss: Sequence[np.ndarray], chis, eps, epsinvs, stream=None):
        n = len(cells)
        carr = (Cell * n)(*cells)
        keep = [_i32(g) for g in gepss]
        ng = (ctypes.c_int * n)(*[k[0].shape[0] for k in keep])
        gp = (ctypes.POINTER(ctypes.c_int32) * n)(*[k[1] for k in keep])
        cp = (ctypes.c_void_p * n)(*[_ptr(x) for x in chis])
        ep = None if eps is None else (ctypes.c_void_p * n)(*[_ptr(x) for x in eps])
        ip = (ctypes.c_void_p * n)(*[_ptr(x) for x in epsinvs])
        self._check(self.lib.bgw_epsinv_rflavor(self.h, n, carr, ng, gp, cp, ep, ip, _stream(stream)))
        return epsinvs

    def sigma_cohsex(self, cell: Cell, go, co, gi, ci, nocc: int, geps, epsinv, stream=None,
                     prec: int = 0) -> np.ndarray:
        """bgw_sigma_cohsex: returns [4][no] (X, SX, CH sum form, CH closed form), Hartree."""
        go_, gop = _i32(go)
        gi_, gip = _i32(gi)
        ge_, gep = _i32(geps)
        out = np.zeros((4, co.shape[0]), dtype=np.float64)
        self._check(self.lib.bgw_sigma_cohsex(self.h, ctypes.byref(cell), co.shape[0], go_.shape[0], gop, _ptr(co),
                                              ci.shape[0], gi_.shape[0], gip, _ptr(ci), nocc, ge_.shape[0], gep,
                                              _ptr(epsinv), prec, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                              _stream(stream)))
        return out

    def screened_w(self, cells: Sequence[Cell], gepss: Sequence[np.ndarray], epsinvs, ws, stream=None):
        n = len(cells)
        carr = (Cell * n)(*cells)
        keep = [_i32(g) for g in gepss]
        ng = (ctypes.c_int * n)(*[k[0].shape[0] for k in keep])
        gp = (ctypes.POINTER(ctypes.c_int32) * n)(*[k[1] for k in keep])
        ip = (ctypes.c_void_p * n)(*[_ptr(x) for x in epsinvs])
        wp = (ctypes.c_void_p * n)(*[_ptr(x) for x in ws])
        self._check(self.lib.bgw_screened_w(self.h, n, carr, ng, gp, ip, wp, _stream(stream)))
        return ws

    def epsilon(self, cell: Cell, gv, cv, ev, gc, cc, ec, geps, omega, prec: int, nc_chunk: int, chi, epsinv,
                stream=None):
        gv_, gvp = _i32(gv)
        gc_, gcp = _i32(gc)
        ge_, gep = _i32(geps)
        ev_, evp = _f64(ev)
        ec_, ecp = _f64(ec)
        om_, omp = _f64(omega)
        nfreq = 0 if om_ is None else om_.shape[0]
        self._check(self.lib.bgw_epsilon(self.h, ctypes.byref(cell), cv.shape[0], gv_.shape[0], gvp, _ptr(cv), evp,
                                         cc.shape[0], gc_.shape[0], gcp, _ptr(cc), ecp, ge_.shape[0], gep, nfreq,
                                         omp, prec, nc_chunk, _ptr(chi), _ptr(epsinv), _stream(stream)))
        return epsinv

    def epsilon_batch(self, systems, cvs, ccs, omega, prec: int, epsinvs, stream=None, cells=None):
        """bgw_epsilon_batch over q-points: `systems` give the host arrays (G
        lists, energies, cell), `cvs`/`ccs` the device coefficient tensors,
        `epsinvs` the device outputs [max(1,nfreq)][ng][ng] per q-point;
        `cells` (optional) replaces the systems' cells, e.g. to select a
        truncated Coulomb interaction."""
        n = len(systems)
        keep = []
        probs = (Problem * n)()
        for k, s in enumerate(systems):
            gv_, gvp = _i32(s.gv)
            gc_, gcp = _i32(s.gc)
            ge_, gep = _i32(s.geps)
            ev_, evp = _f64(s.ev)
            ec_, ecp = _f64(s.ec)
            keep += [gv_, gc_, ge_, ev_, ec_]
            p = probs[k]
            p.cell = cells[k] if cells is not None else make_cell(s.bvec, s.omega, s.q_frac, s.fft)
            p.nv, p.npw_v, p.gv, p.cv, p.ev = cvs[k].shape[0], gv_.shape[0], gvp, _ptr(cvs[k]), evp
            p.nc, p.npw_c, p.gc, p.cc, p.ec = ccs[k].shape[0], gc_.shape[0], gcp, _ptr(ccs[k]), ecp
            p.ng, p.geps = ge_.shape[0], gep
        om_, omp = _f64(omega)
        nfreq = 0 if om_ is None else om_.shape[0]
        outs = (ctypes.c_void_p * n)(*[_ptr(x) for x in epsinvs])
        self._check(self.lib.bgw_epsilon_batch(self.h, n, probs, nfreq, omp, prec, outs, _stream(stream)))
        return epsinvs


def _problem(s, cv, cc, keep):
    """Fill a Problem from a synthetic system; cv/cc are arrays or tensors."""
    gv_, gvp = _i32(s.gv)
    gc_, gcp = _i32(s.gc)
    ge_, gep = _i32(s.geps)
    ev_, evp = _f64(s.ev)
    ec_, ecp = _f64(s.ec)
    keep += [gv_, gc_, ge_, ev_, ec_, cv, cc]
    p = Problem()
    p.cell = make_cell(s.bvec, s.omega, s.q_frac, s.fft)
    p.nv, p.npw_v, p.gv, p.cv, p.ev = cv.shape[0], gv_.shape[0], gvp, _ptr(cv), evp
    p.nc, p.npw_c, p.gc, p.cc, p.ec = cc.shape[0], gc_.shape[0], gcp, _ptr(cc), ecp
    p.ng, p.geps = ge_.shape[0], gep
    return p


class Server:
    """bgw_serve_*: requests of different sizes, admitted by an HBM budget
    and run concurrently on per-slot streams."""

    def __init__(self, ctx: "Context", hbm_budget_bytes: int = 0, max_slots: int = 4, prec: int = BGW_PREC_MIX_FP16):
        """ctx: the Context whose device serves the requests (read at open)."""
        self.lib = load()
        o = ServeOpts(hbm_budget_bytes, max_slots, prec)
        h = ctypes.c_void_p()
        rc = self.lib.bgw_serve_open(ctx.h, ctypes.byref(o), ctypes.byref(h))
        if rc != BGW_OK:
            raise BgwError(rc, "bgw_serve_open failed")
        self.h = h
        self._outs = {}

    def submit(self, system, out) -> int:
        """Queue one request (host cv/cc taken from `system`); `out` is a host
        array [ng][ng] complex128 that receives eps~^-1."""
        keep = []
        r = Request()
        r.problem = _problem(system, np.ascontiguousarray(system.cv), np.ascontiguousarray(system.cc), keep)
        r.epsinv_out = _ptr(out)
        t = ctypes.c_uint64()
        rc = self.lib.bgw_serve_submit(self.h, ctypes.byref(r), ctypes.byref(t))
        if rc != BGW_OK:
            raise BgwError(rc, "bgw_serve_submit failed")
        self._outs[t.value] = out
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 0):
        """Result of a request, or None while it is still pending."""
        res = Result()
        rc = self.lib.bgw_serve_poll(self.h, ticket, timeout_ms, ctypes.byref(res))
        if rc == BGW_EBUSY:
            return None
        if rc != BGW_OK:
            raise BgwError(rc, "bgw_serve_poll failed")
        self._outs.pop(ticket, None)
        return {"status": res.status, "latency_ms": res.latency_ms, "queue_ms": res.queue_ms,
                "hbm_bytes": res.hbm_bytes}

    def cancel(self, ticket: int) -> int:
        return self.lib.bgw_serve_cancel(self.h, ticket)

    def close(self):
        if getattr(self, "h", None):
            self.lib.bgw_serve_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
