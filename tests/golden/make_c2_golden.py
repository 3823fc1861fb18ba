"""Writes tests/golden/c2_oracle.npz: FP64 oracle values of the mixed-precision
large-cell workload (a = 30.78 bohr, 60^3 grid, 12 Ry wavefunction and 6 Ry
epsilon spheres: N_G = 7180, N_v = 108, N_c = 3000, K = 324,000 pairs).

The whole oracle solve takes tens of minutes on a host, too long for a test,
so this script runs it once and stores what the GPU test compares against:
the seeded random 256 x 256 principal subblock (indices from the workload's
"subblock" sub-seed) of chi and of eps~^-1, the diagonal of eps~^-1, and a
fingerprint of the generated inputs -- a digest of the G lists and sampled
coefficients and energies -- so a test can tell that it regenerated the same
system on another machine.  It calls only the input generator and oracle/: the matrix
elements by the FFT route of Eq. eqn_matrix_elem, chi as the product of Eq.
eqn_static_xi_compact summed over conduction-band chunks (the pair sum split
into parts), eps~ = I - v^1/2 chi v^1/2 and its library inverse.

Usage: python tests/golden/make_c2_golden.py [--chunk NC] [--save-chi PATH]
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1111_4429_gb300 import synth  # noqa: E402


def g_digest(s) -> str:
    """SHA-256 of the three G lists (valence, conduction, epsilon sphere) in
    their order: equal digests mean the same integer inputs, exactly."""
    h = hashlib.sha256()
    for g in (s.gv, s.gc, s.geps):
        h.update(np.ascontiguousarray(g, dtype="<i4").tobytes())
    return h.hexdigest()


def fingerprint(s) -> np.ndarray:
    """Generated values that pin the floating-point inputs (compared to
    ~1e-12): energies at both ends and coefficients at 64 seeded positions
    of the first, middle and last bands."""
    gen = np.random.Generator(np.random.PCG64(7))
    iv = gen.integers(0, s.cv.shape[1], 64)
    ic = gen.integers(0, s.cc.shape[1], 64)
    parts = [s.ev[:4], s.ec[:4], s.ec[-4:]]
    for b in (0, s.nv // 2, s.nv - 1):
        parts.append(s.cv[b, iv].view(np.float64))
    for b in (0, s.nc // 2, s.nc - 1):
        parts.append(s.cc[b, ic].view(np.float64))
    return np.concatenate(parts)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--chunk", type=int, default=100, help="conduction bands per oracle chunk")
    ap.add_argument("--save-chi", default=None, help="also write the full chi (.npy) here")
    ap.add_argument("--out", default=os.path.join(HERE, "c2_oracle.npz"))
    args = ap.parse_args()

    t0 = time.perf_counter()
    s = synth.config_system("c2")
    t_gen = time.perf_counter() - t0
    print(f"inputs: N_G {s.ng}, N_v {s.nv}, N_c {s.nc}, npw {s.gv.shape[0]}/{s.gc.shape[0]} ({t_gen:.1f} s)",
          flush=True)
    chi = np.zeros((s.ng, s.ng), dtype=np.complex128)
    t_m = t_x = 0.0
    for c0 in range(0, s.nc, args.chunk):
        c1 = min(s.nc, c0 + args.chunk)
        t = time.perf_counter()
        m = oracle.mtxel_fft(s.gv, s.cv, s.gc, s.cc[c0:c1], s.geps, s.fft)
        t_m += time.perf_counter() - t
        t = time.perf_counter()
        chi += oracle.chi(m, oracle.chi_weights(s.ev, s.ec[c0:c1]), s.omega)
        t_x += time.perf_counter() - t
        del m
        print(f"  conduction bands {c0}..{c1 - 1}: M {t_m:.0f} s, chi {t_x:.0f} s", flush=True)
    t = time.perf_counter()
    v = oracle.coulomb(s.bvec, s.q_frac, s.geps)
    eps, epsinv = oracle.epsinv_sym(chi, v)
    t_inv = time.perf_counter() - t
    idx = synth.subblock_indices(s.ng, 256, s.seed)
    resid = float(np.linalg.norm(eps @ epsinv - np.eye(s.ng)) / np.sqrt(s.ng))
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    np.savez(args.out,
             idx=idx,
             chi_sub=chi[np.ix_(idx, idx)],
             epsinv_sub=epsinv[np.ix_(idx, idx)],
             epsinv_diag=np.ascontiguousarray(np.diagonal(epsinv)),
             fingerprint=fingerprint(s),
             g_digest=np.array(g_digest(s)),
             chi_fro=np.array(np.linalg.norm(chi)),
             epsinv_fro=np.array(np.linalg.norm(epsinv)),
             residual=np.array(resid),
             seconds=np.array([t_gen, t_m, t_x, t_inv]),
             cores=np.array(cores))
    if args.save_chi:
        np.save(args.save_chi, chi)
    print(f"written {args.out}: M {t_m:.0f} s, chi {t_x:.0f} s, inverse {t_inv:.0f} s on {cores} cores; "
          f"||eps eps^-1 - I||/sqrt(N_G) = {resid:.2e}", flush=True)


if __name__ == "__main__":
    main()
