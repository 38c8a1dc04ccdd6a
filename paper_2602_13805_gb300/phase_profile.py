"""Per-phase time of the cluster loop (use_graph = 3) from in-kernel global-timer marks.

Builds the instrumented library (build.py --stamps), runs a reconstruction of each named
workload with it and prints, per phase of one iteration, the microseconds between the barrier
marks of thread 0 of the first CTA, averaged over iterations 5..8.  The marks sit right after
existing barriers, so the instrumented loop does the same work in the same order.

    python -m paper_2602_13805_gb300.phase_profile c2 c1 cP
"""
from __future__ import annotations

import ctypes
import os
import sys

import numpy as np

PHASES = [
    "synthesis T' = Wy^T alpha, all rows (Eq. 9); r_d = (G_S Phi) alpha - E_sca (Eq. 16)",
    "(no work: J on own rows runs inside the exchange barrier below)",
    "row DFT of J at own columns (T' what)",
    "column convolution with the G_D spectrum -> row owners; J on own rows between arrive and wait of the cluster barrier",
    "inverse row DFT (G_D J)",
    "s and the per-incidence sums + grid barrier",
    "R-hat, chi-hat from the sums over incidences (Eq. 6, 7; split over the grid: + grid barrier)",
    "TV / bridge pieces (Eq. 18, 19)",
    "residual, cotangent on chi, adjoint inputs u, v",
    "row DFTs of u and v -> column owners + cluster barrier",
    "column convolution with the conjugated spectrum, + v (kept local)",
    "x-analysis: column data x conj(what)",
    "y-analysis partials -> all CTAs + cluster barrier",
    "gradient sum + (G_S Phi)^H r_d + Adam step",
]


def main(names):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_2602_13805_gb300 import build, pdf
    import scenes
    import torch

    pdf.load(build.build(stamps=True))
    for name in names:
        w = scenes.workload(name, iters=20)
        prob = pdf.Problem.from_workload(w, esca=np.ones((w.ni, w.nr), np.complex64))
        prob.solve(iters=20, use_graph=3)
        torch.cuda.synchronize()
        buf = (ctypes.c_uint64 * 64)()
        st = pdf.load().pdf_phase_stamps(buf)
        if st != 0:
            raise RuntimeError(f"pdf_phase_stamps failed ({st})")
        s = np.array(buf[:], dtype=np.int64).reshape(4, 16)[:, :15].astype(np.float64)
        d = np.diff(s, axis=1).mean(axis=0) / 1e3
        it_us = (s[:, 14] - s[:, 0]).mean() / 1e3
        print(f"\n{name}: {w.nx}x{w.ny}, Ni={w.ni}, Nr={w.nr}, K={w.kx}; {it_us:.1f} us per iteration "
              f"(marks 0..14; the step from the Adam mark to the next iteration's first mark is not included)")
        print("| phase | us | share |\n|---|---:|---:|")
        for n, v in zip(PHASES, d):
            print(f"| {n} | {v:.2f} | {100 * v / it_us:.0f}% |")
        prob.close()


if __name__ == "__main__":
    main(sys.argv[1:] or ["c2"])
