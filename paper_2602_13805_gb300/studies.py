"""Robustness studies built from the finished solver, on one GPU: batches of independent
reconstructions (Sec. 4.5, antenna position uncertainty; the loss-term and CCO ablations that
Sec. 4 discusses).

    python -m paper_2602_13805_gb300.studies jitter --workload cP --sigma-mm 1 2 3 --realisations 100
    python -m paper_2602_13805_gb300.studies ablation --workload c2 [--fcnn 256]

Jitter: realisation r at deviation sigma measures the scene with every transmitter and receiver
moved by independent Gaussian offsets (standard deviation sigma on each coordinate), through the
GPU forward solver, plus the workload's noise (one fixed noise draw, so realisations differ only
in the antenna positions); the reconstruction assumes the nominal circle.  sigma is given in
millimetres at the paper's 400 MHz (lambda = 0.75 m) and converted to wavelengths.
Ablation: one scene and its data reconstructed with each regulariser weight set to zero in turn,
and with the CCO post-processing off.
Each line of output is a JSON object; RelErr is measured after the CCO unless the CCO is off.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

LAMBDA_M = 299792458.0 / 400e6          # wavelength of the paper's 400 MHz measurements


def jitter_rng(seed: int, sigma_index: int, r: int) -> np.random.Generator:
    """Generator of realisation r at the sigma_index-th deviation."""
    return np.random.default_rng([seed, sigma_index, r])


def realisation_geometry(w, sigma_lambda: float, rng: np.random.Generator):
    """Perturbed (tx, rx) of one realisation: nominal circle plus Gaussian offsets."""
    import scenes
    tx, rx = scenes.geometry(w)
    return scenes.perturb_antennas(tx, sigma_lambda, rng), scenes.perturb_antennas(rx, sigma_lambda, rng)


def measure(w, chi_dev, tx, rx, noise_seed: int):
    """Scattered field of the scene for antennas at (tx, rx), GPU forward solver plus the workload's
    noise: complex64 numpy [ni][nr]."""
    import scenes
    from paper_2602_13805_gb300 import pdf
    prob = pdf.Problem.from_workload(w, tx=tx, rx=rx)
    try:
        esca, _, _ = prob.forward(chi_dev, tol=1e-6, max_iter=3000)
        e = esca.cpu().numpy().astype(np.complex128)
    finally:
        prob.close()
    return scenes.add_awgn(e, w.noise, np.random.default_rng(1000 + noise_seed)).astype(np.complex64)


class Reconstructor:
    """A nominal-geometry problem and the solve options of one study."""

    def __init__(self, w, chi_true, fcnn: int = 0, **cfg):
        import torch
        import scenes
        from paper_2602_13805_gb300 import pdf
        self.w = w
        self.prob = pdf.Problem.from_workload(w, **cfg)
        self.chi_dev = torch.from_numpy(chi_true.astype(np.complex64)).cuda()
        self.net = {}
        if fcnn > 0:
            self.net = dict(fcnn_hidden=fcnn,
                            fcnn_params0=torch.from_numpy(scenes.fcnn_params(w.ky, w.kx, fcnn, seed=0)).cuda())

    def run(self, esca, apply_cco=True):
        import torch
        self.prob.set_data(torch.from_numpy(esca).cuda())
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = self.prob.solve(iters=self.w.iters, chi_true=self.chi_dev, apply_cco=apply_cco, **self.net)
        b.record()
        torch.cuda.synchronize()
        return dict(relerr=out["relerr"], relerr_cco=out["relerr_cco"], ms=a.elapsed_time(b),
                    loss=float(out["terms"][0]), loop_mode=out["loop_mode"])

    def close(self):
        self.prob.close()


def jitter_study(name: str, sigmas_mm, realisations: int, fcnn: int = 0, seed: int = 0):
    import torch
    import scenes
    w = scenes.workload(name)
    chi = scenes.make_scene(w, seed)
    rec = Reconstructor(w, chi, fcnn)
    chi_dev = torch.from_numpy(chi.astype(np.complex64)).cuda()
    tx0, rx0 = scenes.geometry(w)
    base = rec.run(measure(w, chi_dev, tx0, rx0, seed))
    rows = []
    t0 = time.perf_counter()
    for si, smm in enumerate(sigmas_mm):
        sig = smm * 1e-3 / LAMBDA_M
        rel, ms = [], []
        for r in range(realisations):
            tx, rx = realisation_geometry(w, sig, jitter_rng(seed, si, r))
            o = rec.run(measure(w, chi_dev, tx, rx, seed))
            rel.append(o["relerr_cco"])
            ms.append(o["ms"])
        rel = np.array(rel)
        rows.append(dict(sigma_mm=smm, sigma_lambda=sig, realisations=realisations,
                         relerr_cco_min=float(rel.min()), relerr_cco_q1=float(np.quantile(rel, 0.25)),
                         relerr_cco_median=float(np.median(rel)), relerr_cco_q3=float(np.quantile(rel, 0.75)),
                         relerr_cco_max=float(rel.max()), spread=float(rel.max() - rel.min()),
                         ms_per_reconstruction=float(np.mean(ms))))
    rec.close()
    return dict(study="antenna position jitter", workload=name, fcnn_hidden=fcnn, iters=w.iters,
                nominal_relerr_cco=base["relerr_cco"], rows=rows, wall_s=time.perf_counter() - t0,
                note="per realisation: GPU forward solve at the perturbed antennas, reconstruction at the nominal ones")


ABLATIONS = [("full", {}, True), ("no L_Bound", dict(lambda_bound=0.0), True), ("no L_TV", dict(lambda_tv=0.0), True),
             ("no L_Bridge", dict(lambda_bridge=0.0), True), ("no CCO", {}, False)]


def ablation_study(name: str, fcnn: int = 0, seed: int = 0):
    import torch
    import scenes
    w = scenes.workload(name)
    chi = scenes.make_scene(w, seed)
    chi_dev = torch.from_numpy(chi.astype(np.complex64)).cuda()
    tx0, rx0 = scenes.geometry(w)
    esca = measure(w, chi_dev, tx0, rx0, seed)
    rows = []
    for label, cfg, cco in ABLATIONS:
        rec = Reconstructor(w, chi, fcnn, **cfg)
        o = rec.run(esca, apply_cco=cco)
        rec.close()
        rows.append(dict(variant=label, relerr=o["relerr"], relerr_cco=o["relerr_cco"] if cco else None,
                         final_loss=o["loss"], ms=o["ms"]))
    return dict(study="ablation", workload=name, fcnn_hidden=fcnn, iters=w.iters, rows=rows)


def main(argv=None):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["jitter", "ablation"])
    ap.add_argument("--workload", default="cP")
    ap.add_argument("--sigma-mm", type=float, nargs="+", default=[1.0, 2.0, 3.0])
    ap.add_argument("--realisations", type=int, default=100)
    ap.add_argument("--fcnn", type=int, default=0)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    from paper_2602_13805_gb300 import build, pdf
    pdf.load(build.build())
    if a.study == "jitter":
        out = jitter_study(a.workload, a.sigma_mm, a.realisations, a.fcnn, a.seed)
    else:
        out = ablation_study(a.workload, a.fcnn, a.seed)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
