"""CPU-side checks of the boundary: the library builds, loads and exports every
symbol that include/bgw.h declares (no compute call without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(bgw_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1111_4429_gb300 import _build
    _build.build()
    from paper_1111_4429_gb300 import bgw
    return bgw.load()


def test_header_declares_the_entry_points():
    d = _declared()
    for name in ("bgw_create", "bgw_destroy", "bgw_mtxel", "bgw_chi_sum", "bgw_epsinv", "bgw_epsilon",
                 "bgw_sync", "bgw_last_error", "bgw_mem_stats"):
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_binding_lists_every_declared_symbol():
    from paper_1111_4429_gb300 import bgw
    assert sorted(bgw.EXPORTS) == sorted(n for n in _declared() if n in bgw.EXPORTS)
    assert set(_declared()) <= set(bgw.EXPORTS) | {n for n in _declared() if n.startswith("bgw_")}


def test_cell_struct_layout():
    from paper_1111_4429_gb300 import bgw
    # double bvec[3][3]; double omega; double q_frac[3]; int fft[3]; int coulomb; double coulomb_cut
    assert ctypes.sizeof(bgw.Cell) == 8 * 9 + 8 + 8 * 3 + 4 * 3 + 4 + 8
    assert bgw.Cell.omega.offset == 72 and bgw.Cell.q_frac.offset == 80 and bgw.Cell.fft.offset == 104
    assert bgw.Cell.coulomb.offset == 116 and bgw.Cell.coulomb_cut.offset == 120


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1111_4429_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, re.M), f


def test_frequency_grid_host_matches_oracle():
    from paper_1111_4429_gb300 import bgw
    import numpy as np
    import oracle
    for args in [(0.1, 0.5, 2.0, 0.1), (0.25, 1.0, 2.0, 0.0), (0.2, 1.0, 10.0, 0.05), (0.01, 3.0, 60.0, 0.01),
                 (0.5, 0.0, 0.0, 0.0)]:
        assert np.array_equal(bgw.frequency_grid(*args), oracle.frequency_grid(*args))
    import pytest
    for bad in [(0.0, 1.0, 2.0, 0.1), (0.1, 1.0, 0.5, 0.1), (0.1, 1.0, 2.0, -0.1)]:
        with pytest.raises(bgw.BgwError):
            bgw.frequency_grid(*bad)


def test_real_coefficients_host_matches_oracle_subspaces():
    from paper_1111_4429_gb300 import bgw, synth
    import numpy as np
    import oracle
    gen = np.random.default_rng(4)
    q, _ = np.linalg.qr(gen.standard_normal((50, 8)))
    real = q.T
    e = np.array([-0.6, -0.2, -0.2, 0.0, 0.3, 0.3, 0.3, 0.9])
    cplx = synth.scramble_phases(real, [[1, 2], [4, 5, 6]], seed=9)
    got = bgw.real_coefficients(cplx, e, 1e-9)
    ref = oracle.realify(cplx, e, 1e-9)
    assert np.allclose(got @ got.T, np.eye(8), atol=1e-13)
    for g in [[0], [1, 2], [3], [4, 5, 6], [7]]:
        assert np.abs(got[g].T @ got[g] - ref[g].T @ ref[g]).max() < 1e-13
    import pytest
    with pytest.raises(bgw.BgwError):
        bgw.real_coefficients(np.zeros((1, 50), complex), np.array([0.0]), 1e-9)


def test_binding_constants_match_the_header():
    """Every BGW_* enumerator the binding names has the header's value (the
    options, precisions, flavour flag, Coulomb models and status codes)."""
    from paper_1111_4429_gb300 import bgw
    txt = ""
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt += open(os.path.join(ROOT, "include", h)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    header = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", txt, flags=re.S):
        for name, val in re.findall(r"\b(BGW_[A-Z0-9_]+)\s*=\s*(0x[0-9a-fA-F]+|-?\d+)", body):
            header[name] = int(val, 0)
    names = [n for n in dir(bgw) if n.startswith("BGW_") and isinstance(getattr(bgw, n), int)]
    assert len(names) >= 15
    for n in names:
        assert n in header, n
        assert getattr(bgw, n) == header[n], n
    for n in ("BGW_OPT_UPDATE_SLICES", "BGW_OPT_DOUBLE_FP32", "BGW_OPT_SIGMA_DENSITY", "BGW_OPT_HEAD",
              "BGW_OPT_PAIR_KERNEL", "BGW_OPT_UPDATE_ITEMS", "BGW_OPT_WAIT_LIMIT_NS"):
        assert n in names


def test_frequency_grid_error_codes():
    """The documented codes of bgw_frequency_grid: EINVAL for a negative low
    cutoff or more than 2^24 points, ENOMEM for a short output (the count is
    still written, nothing past max_points), and a NULL output to count."""
    import ctypes
    import numpy as np
    from paper_1111_4429_gb300 import bgw
    lib = bgw.load()
    d = ctypes.c_double
    n = ctypes.c_int(-1)
    assert lib.bgw_frequency_grid(d(0.1), d(-0.5), d(2.0), d(0.1), 0, None, ctypes.byref(n)) == bgw.BGW_EINVAL
    assert lib.bgw_frequency_grid(d(1e-9), d(1.0), d(1.0), d(0.0), 0, None, ctypes.byref(n)) == bgw.BGW_EINVAL
    assert lib.bgw_frequency_grid(d(0.1), d(0.5), d(2.0), d(0.1), 0, None, ctypes.byref(n)) == bgw.BGW_OK
    full = n.value
    assert full == len(bgw.frequency_grid(0.1, 0.5, 2.0, 0.1))
    out = np.full(full, -7.0)
    n2 = ctypes.c_int(-1)
    rc = lib.bgw_frequency_grid(d(0.1), d(0.5), d(2.0), d(0.1), full - 2,
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(n2))
    assert rc == bgw.BGW_ENOMEM and n2.value == full
    assert np.all(out[full - 2:] == -7.0)


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No fallback: with the shared library missing, loading the binding
    raises instead of computing anything another way."""
    import pytest
    from paper_1111_4429_gb300 import bgw
    monkeypatch.setattr(bgw, "_lib", None)
    monkeypatch.setattr(bgw, "LIB_PATH", str(tmp_path / "libbgw.so"))
    with pytest.raises(ImportError):
        bgw.load()
    with pytest.raises(ImportError):
        bgw.frequency_grid(0.1, 0.5, 2.0, 0.1)
