"""The mixed-precision large-cell workload at full size against the FP64 oracle.

a = 30.78 bohr (a cell of the (20,20) nanotube supercell's volume), 60^3 grid,
12 Ry wavefunction spheres (20,422 / 20,341 coefficients), 6 Ry epsilon
sphere (N_G = 7180), N_v = 108, N_c = 3000: K = 324,000 pairs, streamed in
conduction chunks of 500 bands (54,000 pairs, 3.1 GB of complex64 M per
chunk) through bgw_epsilon on device buffers, chi summed on the tensor cores
(split FP16, FP32 segments, FP64 sum), eps~ and its inverse FP64-level.

The full oracle solve takes tens of minutes on a host, so its values come
from tests/golden/c2_oracle.npz (written by make_c2_golden.py beside it, which
calls only the input generator and the oracle): the seeded 256 x 256
principal subblock of chi and eps~^-1 and the diagonal of eps~^-1.  The test
also checks sampled rows of M against the oracle's FFT route element by
element, and the residual of eps~ eps~^-1 = I over the whole matrix.
Bars: eps~^-1 1e-6 (the mixed path's), chi 1e-5, M 1e-5 (FP32 FFTs).
"""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_1111_4429_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
GOLDEN = os.path.join(GOLDEN_DIR, "c2_oracle.npz")
if GOLDEN_DIR not in sys.path:
    sys.path.insert(0, GOLDEN_DIR)
NC_CHUNK = 500


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def c2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = np.load(GOLDEN)
    from make_c2_golden import fingerprint, g_digest
    s = synth.config_system("c2")
    assert s.ng == 7180 and s.npairs == 324000
    assert g_digest(s) == str(g["g_digest"]), "the G lists differ from the golden run's"
    fp = fingerprint(s)
    assert np.allclose(fp, g["fingerprint"], rtol=0, atol=1e-12), "regenerated inputs differ from the golden run's"
    return s, g


@pytest.fixture(scope="module")
def solved(c2):
    from paper_1111_4429_gb300 import bgw
    s, g = c2
    ctx = bgw.Context(0)
    cv = torch.from_numpy(s.cv).cuda()
    cc = torch.from_numpy(s.cc).cuda()
    chi = torch.empty((1, s.ng, s.ng), dtype=torch.complex128, device="cuda")
    inv = torch.empty_like(chi)
    ctx.epsilon(bgw.system_cell(s), s.gv, cv, s.ev, s.gc, cc, s.ec, s.geps, None, bgw.BGW_PREC_MIX_FP16,
                NC_CHUNK, chi, inv)
    ctx.sync()
    return ctx, cv, cc, chi[0], inv[0]


def test_c2_mixed_subblocks_vs_oracle(c2, solved):
    s, g = c2
    _, _, _, chi, inv = solved
    idx = torch.from_numpy(g["idx"]).cuda()
    chi_sub = chi[idx][:, idx].cpu().numpy()
    inv_sub = inv[idx][:, idx].cpu().numpy()
    inv_diag = torch.diagonal(inv).cpu().numpy()
    e_chi = _rel(chi_sub, g["chi_sub"])
    e_inv = _rel(inv_sub, g["epsinv_sub"])
    e_diag = _rel(inv_diag, g["epsinv_diag"])
    print(f"c2 mixed vs oracle: chi subblock {e_chi:.3e}, eps~^-1 subblock {e_inv:.3e}, diagonal {e_diag:.3e}")
    assert e_chi <= 1e-5
    assert e_inv <= 1e-6
    assert e_diag <= 1e-6
    # the whole matrices: Hermitian chi (mirrored exactly), Frobenius norms
    assert bool(torch.equal(chi, chi.conj().T.resolve_conj()))
    assert abs(float(torch.linalg.matrix_norm(chi)) / float(g["chi_fro"]) - 1) <= 1e-5
    assert abs(float(torch.linalg.matrix_norm(inv)) / float(g["epsinv_fro"]) - 1) <= 1e-6


def test_c2_mixed_inverse_residual(c2, solved):
    s, _ = c2
    _, _, _, chi, inv = solved
    sv = torch.from_numpy(np.sqrt(oracle.coulomb(s.bvec, s.q_frac, s.geps))).cuda()
    eps = torch.eye(s.ng, dtype=torch.complex128, device="cuda") - sv[:, None] * chi * sv[None, :]
    r = torch.linalg.matrix_norm(eps @ inv - torch.eye(s.ng, dtype=torch.complex128, device="cuda"))
    resid = float(r) / np.sqrt(s.ng)
    print(f"c2 ||eps~ eps~^-1 - I||_F / sqrt(N_G) = {resid:.3e}")
    assert resid <= 1e-11


def test_c2_mixed_sampled_m_rows_vs_oracle(c2, solved):
    from paper_1111_4429_gb300 import bgw
    s, _ = c2
    ctx, cv, cc, _, _ = solved
    c0 = s.nc - NC_CHUNK       # the last conduction chunk, as bgw_epsilon streams it
    M = torch.empty((s.nv * NC_CHUNK, s.ng), dtype=torch.complex64, device="cuda")
    ctx.mtxel(bgw.system_cell(s), s.gv, cv, s.gc, cc[c0:], s.geps, bgw.BGW_PREC_MIX_FP16, M)
    ctx.sync()
    gen = np.random.Generator(np.random.PCG64(2002))
    rows = np.sort(gen.choice(s.nv * NC_CHUNK, 8, replace=False))
    rows[0], rows[-1] = 0, s.nv * NC_CHUNK - 1
    got = M[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.complex128)
    # global pair index of chunk row r = v * NC_CHUNK + c: v * N_c + c0 + c
    pairs = (rows // NC_CHUNK) * s.nc + c0 + rows % NC_CHUNK
    ref = oracle.mtxel_fft_pairs(s.gv, s.cv, s.gc, s.cc, s.geps, s.fft, pairs)
    for k in range(len(rows)):
        assert _rel(got[k], ref[k]) <= 1e-5
        assert np.all(np.abs(got[k] - ref[k]) <= 1e-5 * np.abs(ref[k]).max())
