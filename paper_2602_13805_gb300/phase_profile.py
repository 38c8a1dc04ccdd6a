"""Per-phase time of the cluster loop (use_graph = 3) from in-kernel global-timer marks.

Builds the instrumented library (build.py --stamps), runs a reconstruction of each named
workload with it and prints, per phase of one iteration, the microseconds between the barrier
marks of thread 0 of the first CTA, averaged over iterations 5..8.  The marks sit right after
existing barriers, so the instrumented loop does the same work in the same order.

    python -m paper_2602_13805_gb300.phase_profile c2 c1 cP
    python -m paper_2602_13805_gb300.phase_profile --fcnn 64 c2     (the network form)
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


NET_PHASES = [
    "network forward: h1 rows per CTA -> all (cluster barrier), h2, output rows -> alpha_p in all (cluster barrier)",
    "chain rule per incidence (dL/dy, dz2 partials -> all + cluster barrier, dz1, vectors out) + grid barrier",
    "dL/d theta on this CTA's slice of theta (sums over incidences) + Adam step",
    "grid barrier publishing theta",
]


def main(names, fcnn=0):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_2602_13805_gb300 import build, pdf
    import scenes
    import torch

    pdf.load(build.build(stamps=True))
    for name in names:
        w = scenes.workload(name, iters=20)
        prob = pdf.Problem.from_workload(w, esca=np.ones((w.ni, w.nr), np.complex64))
        net = {}
        if fcnn > 0:
            net = dict(fcnn_hidden=fcnn,
                       fcnn_params0=torch.from_numpy(scenes.fcnn_params(w.ky, w.kx, fcnn, seed=0)).cuda())
        out = prob.solve(iters=20, use_graph=3, **net)
        torch.cuda.synchronize()
        if out["loop_mode"] != 3:
            print(f"\n{name}: the cluster loop did not run (loop_mode {out['loop_mode']})")
            prob.close()
            continue
        buf = (ctypes.c_uint64 * 80)()
        st = pdf.load().pdf_phase_stamps(buf)
        if st != 0:
            raise RuntimeError(f"pdf_phase_stamps failed ({st})")
        s = np.array(buf[:], dtype=np.int64).reshape(4, 20).astype(np.float64)
        if fcnn > 0:
            # iteration: 0 -> 16 (forward) -> 1 .. 14 -> 15 (chain rule + barrier) -> 17 (theta) -> next 0
            m = s[:, [0, 16] + list(range(1, 15)) + [15, 17]]
            d = np.diff(m, axis=1).mean(axis=0) / 1e3
            tail = (s[1:, 0] - s[:-1, 17]).mean() / 1e3
            names_ = NET_PHASES[:1] + PHASES + NET_PHASES[1:3] + NET_PHASES[3:]
            vals = list(d) + [tail]
            it_us = (s[1:, 0] - s[:-1, 0]).mean() / 1e3
            print(f"\n{name} with the network (H = {fcnn}): {w.nx}x{w.ny}, Ni={w.ni}, Nr={w.nr}, K={w.kx}; "
                  f"{it_us:.1f} us per iteration (first mark to the next iteration's)")
        else:
            d = np.diff(s[:, :15], axis=1).mean(axis=0) / 1e3
            names_, vals = PHASES, list(d)
            it_us = (s[:, 14] - s[:, 0]).mean() / 1e3
            print(f"\n{name}: {w.nx}x{w.ny}, Ni={w.ni}, Nr={w.nr}, K={w.kx}; {it_us:.1f} us per iteration "
                  f"(marks 0..14; the step from the Adam mark to the next iteration's first mark is not included)")
        print("| phase | us | share |\n|---|---:|---:|")
        for n, v in zip(names_, vals):
            print(f"| {n} | {v:.2f} | {100 * v / it_us:.0f}% |")
        prob.close()


if __name__ == "__main__":
    args = sys.argv[1:]
    h = 0
    if "--fcnn" in args:
        i = args.index("--fcnn")
        h = int(args[i + 1])
        del args[i:i + 2]
    main(args or ["c2"], fcnn=h)
