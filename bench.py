"""Benchmark: one PDF reconstruction per step on a synthetic scene (GPU, C ABI).

A step is one whole reconstruction of the workload.  Default: the largest configuration, a
192x192 grid over a 4-lambda DOI, 64 line-source incidences, 128 receivers on a 6-lambda circle,
a high-contrast lossy ring (eps_r 5) with a lossy disk and ellipse, 10 % AWGN, K = 31 x 31 Fourier
coefficients, BP + CSI initialisation, then 300 Adam iterations at lr 1e-2 on the weights of the
coefficient-correcting network (the paper's optimiser, hidden width 64), CCO post-processing.
Measured data are synthesised on the GPU by the library's own forward solver (pdf_forward); the
scene and the noise come from the seeded input generators.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c5] [--fcnn 64] [--impl ours|reference]

N > 1 (torchrun): independent replicas, one scene per rank, no data-path collective
("replicas only"); the timing is the max over ranks.  `--impl reference` times the
FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import scenes  # noqa: E402

METRIC = "ms per PDF reconstruction"
L2_BYTES = 129 * 1024 * 1024
FLUSH_BYTES = 512 * 1024 * 1024


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def combine_ranks(total_ms, e2e_ms, steps, world, device):
    """Whole-job figures of `world` replicas that each timed `steps` reconstructions.

    The slowest rank sets the job time (all-reduce MAX; no collective when world == 1).  Returns
    (ms per reconstruction at whole-job throughput, end-to-end ms per reconstruction, the max
    total ms of the timed region)."""
    import torch
    t = torch.tensor([total_ms, e2e_ms], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    total, e2e = float(t[0]), float(t[1])
    return total / (steps * world), e2e / world, total


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def bytes_model(w):
    """Algorithmic bytes per launch of the column-convolution kernel (the largest FFT stage).

    Reads and writes the row-transformed planes [ni][ny][Px] once each and reads the
    kernel spectrum [Py][Px] once: 2 * ni * ny * Px * 8 + Px * Py * 8 bytes.
    """
    px = next_smooth(2 * w.nx)
    py = next_smooth(2 * w.ny)
    return 2 * w.ni * w.ny * px * 8 + px * py * 8


def next_smooth(n):
    best = 1 << 30
    p2 = 1
    while p2 < (1 << 20):
        p = p2
        while p < (1 << 20):
            if n <= p < best:
                best = p
            p *= 3
        p2 *= 2
    return best


def kernel_bytes(w):
    """Algorithmic DRAM bytes per launch of each hot-path kernel (c64 = 8 bytes).

    U = ni*M*8 (one field over all incidences), A = ni*ny*Px*8 (row-transformed planes),
    C = ni*K^2*8 (the coefficients), T = ni*ny*kx*8 (x-analysed rows).
    """
    px, py = next_smooth(2 * w.nx), next_smooth(2 * w.ny)
    M = w.nx * w.ny
    U = w.ni * M * 8
    A = w.ni * w.ny * px * 8
    GS = w.nr * M * 8
    C = w.ni * w.kx * w.ky * 8
    GF = w.nr * w.kx * w.ky * 8
    T = w.ni * w.ny * w.kx * 8
    D = w.ni * w.nr * 8
    return {
        "k_synth_rowfft": U + A + C,                           # write J, write A, read alpha
        "k_colconv": 2 * A + px * py * 8,                      # read + write A, read spectrum
        "k_rowifft_state": A + 4 * U + 4 * M * 8,              # read A, J, E_inc; write s, r; R, chi, D
        "k_gs_partial": U + GS,                                # read J, G_S
        "k_gsf_fwd": GF + C + D,                               # read G_S Phi, alpha; write r_d
        "k_adj_rowfft": 4 * U + A + 2 * M * 8,                 # read J, s, r; write v; write A
        "k_colconv(conj)": 2 * A + px * py * 8,
        "k_gsh": GS + U,                                       # read G_S, write G_S^H r_d
        "k_adj_rowifft_ana": A + U + T,                        # read A, v; write T2
        "k_ana_y": T + C,                                      # read T2; write the gradient
        "k_gsf_adj": GF + D + 2 * C,                           # read G_S Phi, r_d; update the gradient
        "k_synth_rowfft+k_gsf_fwd": U + A + C + GF + 2 * D,    # synthesis tiles with the data residual
    }


# the CUDA kernel behind each profiled stage of the register-FFT path at the bench's sizes
KERNEL_OF_STAGE = {"k_colconv": "kf_colconv_2p<P/16>", "k_synth_rowfft": "kf_synth_2p<P/16>",
                   "k_synth_rowfft+k_gsf_fwd": "kf_synth_2p<P/16>", "k_ana_y": "k_ana_y_cp", "k_gsf_adj": "k_gsf_adj_cp",
                   "k_adj_rowifft_ana": "kf_adj_ana_p<P>", "k_rowifft_state": "kf_rowifft_sums<P> + k_state_combine",
                   "k_adj_rowfft": "kf_adj_rowfft<P>", "k_gsf_fwd": "k_gsf_fwd_p"}

# DRAM bytes (read + write) per launch from one ncu capture, by (workload, stage); None until the
# kernel has been captured in its current form (see profiles/)
TRAFFIC_PER_LAUNCH = {("c5", "k_colconv"): 38964992 + 19456}      # kf_colconv_2p<24>, the ncu summary in profiles/


def cluster_flops(w, fold=1, hidden=0):
    """Algorithmic FP32 flops of one iteration of the fused loop (linear algebra only).

    Per incidence: synthesis T' = Wy^T alpha (ny ky kx complex MACs) and J = T' Wx (ny nx kx), the
    same two contractions again for the analysis (adjoint), G_D and G_D^H as zero-padded FFT
    convolutions (2 ny row + 2 Px column transforms of length P at 5 P log2 P flops, plus Px Py
    complex products, each), and the data term forward and adjoint: with the folded operator
    (fold = 1, the only form the fused loop runs) (G_S Phi) alpha and its adjoint, nr ky kx complex
    MACs each; unfolded (fold = 0) G_S J and G_S^H r_d, nr M each.  A complex MAC is 8 flops, a
    complex product 6.  With the coefficient-correcting network (hidden width H > 0, D = 2 ky kx
    outputs) also its forward pass (H D + H H + D H real MACs), the chain rule to the hidden layers
    (D H + H H) and the weight gradients (H D + H H + D H) per incidence, 2 flops a MAC.  The
    pointwise CIE / regulariser work and the Adam updates are not counted, so this is a lower bound
    on the work done.
    """
    px, py = next_smooth(2 * w.nx), next_smooth(2 * w.ny)
    M = w.nx * w.ny
    syn = 8 * (w.ny * w.ky * w.kx + w.ny * w.nx * w.kx)
    fft = lambda n: 5 * n * np.log2(n)
    gd = (2 * w.ny * fft(px) + 2 * px * fft(py)) + 6 * px * py
    gs = 8 * w.nr * (w.ky * w.kx if fold else M)
    H, D = hidden, 2 * w.ky * w.kx
    net = 2 * (3 * (H * D + H * H + D * H) - H * D) if H > 0 else 0
    return float(w.ni * (2 * syn + 2 * gd + 2 * gs + net))


def hbm_model(w, loop_ms, peaks, fold=1):
    """Whole-iteration HBM fractions by the two byte models of the hot path: B_min = U + 2|G|
    (E_inc once, the data operator forward and adjoint) and B_model = 11 U + 2|G| (plus one HBM
    round trip of the padded intermediate per 2-D transform and the J / r hand-off), U = Ni M 8
    bytes, |G| the data operator the path reads: the folded G_S Phi, Nr ky kx 8 bytes (fold = 1),
    or G_S, Nr M 8 bytes (fold = 0); over the loop time per iteration against the measured copy
    peak."""
    if not loop_ms or w.iters <= 0:
        return None
    M = w.nx * w.ny
    U, GS = 8 * w.ni * M, 8 * w.nr * (w.ky * w.kx if fold else M)
    bmin, bmodel = U + 2 * GS, 11 * U + 2 * GS
    t = loop_ms * 1e-3 / w.iters
    hbm = float(peaks.get("hbm_gbs", 6800.0)) * 1e9
    return {"B_min_MB": bmin / 1e6, "B_model_MB": bmodel / 1e6, "t_iter_us": t * 1e6,
            "frac_min": bmin / t / hbm, "frac_model": bmodel / t / hbm,
            "peak_gbs": hbm / 1e9, "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "data_operator": "folded G_S Phi [nr][ky kx]" if fold else "G_S [nr][M]",
            "note": "at c1-c3 the working set is L2-resident, so these are fractions of the HBM "
                    "roofline by algorithmic bytes, not DRAM traffic"}


def fp32_peak_tflops(peaks):
    """FP32 (non-tensor) FMA peak: 152 SMs x 128 lanes x 2 flops x the SM clock (max 2070 MHz)."""
    return 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def bench_config(w, args, world):
    """The workload description shared by both arms of the benchmark."""
    net = (f", Adam on the weights of the coefficient-correcting network (two hidden layers of {args.fcnn})"
           if args.fcnn > 0 else "")
    return {"workload": f"{w.name}: {w.nx}x{w.ny} grid, {w.side} lambda DOI, Ni={w.ni}, Nr={w.nr}, "
                        f"K={w.kx}x{w.ky}, {w.iters} Adam iterations, BP+CSI init, CCO{net}",
            "iters": w.iters, "lr": args.lr, "precision": args.precision, "loop": args.loop,
            "fcnn_hidden": args.fcnn,
            "fold_gs": args.fold, "parallelism": "replicas" if world > 1 else "single",
            "l2": "flushed between reconstructions (512 MB write); working set L2-resident within one"}


def run_ours(args, rank, world, local):
    import torch
    from paper_2602_13805_gb300 import pdf

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    w = bench_workload(args)
    seed = rank
    chi_true = scenes.make_scene(w, seed)
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    prob = pdf.Problem.from_workload(w, precision=args.precision, fold_gs=args.fold)
    setup_first_ms = (time.perf_counter() - t_setup) * 1e3     # pdf_setup returns synchronised
    chi_d = torch.from_numpy(chi_true.astype(np.complex64)).cuda()
    esca_clean, _, fwd_iters = prob.forward(chi_d, tol=1e-5, max_iter=3000)
    esca = scenes.add_awgn(esca_clean.cpu().numpy().astype(np.complex128), w.noise,
                           np.random.default_rng(1000 + seed)).astype(np.complex64)
    esca_d = torch.from_numpy(esca).cuda()
    prob.set_data(esca_d)
    stream = torch.cuda.current_stream()
    net = {}
    if args.fcnn > 0:                                   # the network's seeded initial weights
        net = dict(fcnn_hidden=args.fcnn,
                   fcnn_params0=torch.from_numpy(scenes.fcnn_params(w.ky, w.kx, args.fcnn, seed=0)).cuda())
    opts = pdf.solve_opts(iters=w.iters, lr=args.lr, init=0, chi_true=chi_d, apply_cco=1, use_graph=args.loop, **net)
    chi_out = torch.empty((w.ny, w.nx), dtype=torch.complex64, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        pdf.pdf_set_data(prob.h, esca_d)
        pdf.pdf_solve(prob.h, opts, chi_out, None, None, report=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # one reported solve for RelErr / loss (outside the timed region)
    rep = pdf.pdf_solve(prob.h, opts, chi_out, None, None, report=True)

    # --- device-resident timed region -------------------------------------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(torch.cuda.current_device())
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = pdf.pdf_launch_count()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                                  # evict L2 between reconstructions (untimed)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = pdf.pdf_launch_count() - launches0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)

    # --- end-to-end through the public API with host buffers ---------------------------
    esca_pinned = torch.from_numpy(esca).pin_memory()
    chi_host = torch.empty((w.ny, w.nx), dtype=torch.complex64).pin_memory()
    esca_np = esca_pinned.numpy()
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        e2e_ev[k][0].record(stream)
        pdf.pdf_set_data(prob.h, esca_np)              # H2D from pinned host memory
        pdf.pdf_solve(prob.h, opts, chi_out, None, None, report=False)
        chi_host.copy_(chi_out, non_blocking=True)     # D2H of the result
        e2e_ev[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = sum(a.elapsed_time(b) for a, b in e2e_ev) / args.steps

    # --- the iteration loop alone: the same solve with 0 iterations, subtracted --------------
    loop_ms = None
    if w.iters > 0:
        opts0 = pdf.solve_opts(iters=0, lr=args.lr, init=0, chi_true=chi_d, apply_cco=1, use_graph=args.loop, **net)
        ev0 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            ev0[k][0].record(stream)
            pdf.pdf_solve(prob.h, opts0, chi_out, None, None, report=False)
            ev0[k][1].record(stream)
        torch.cuda.synchronize()
        ms0 = sum(a.elapsed_time(b) for a, b in ev0) / args.steps
        loop_ms = total_ms / args.steps - ms0

    # --- per-kernel timing (CUDA events between consecutive kernels of pdf_loss_grad) ----
    alpha_probe = torch.zeros((w.ni, w.ky, w.kx), dtype=torch.complex64, device="cuda")
    pdf.pdf_solve(prob.h, pdf.solve_opts(iters=0, init=0, apply_cco=0), None, None, alpha_probe, report=False)
    prof = pdf.pdf_profile_loss_grad(prob.h, alpha_probe, reps=50)
    kb = kernel_bytes(w)
    per_iter_ms = sum(t for _, t in prof)
    # the dominant kernel: the column convolution runs twice per evaluation (G_D and G_D^H, the
    # same kernel), so its two stages count together; achieved = algorithmic bytes per launch /
    # the mean event-timed launch
    stage = dict(prof)
    agg = {}
    for n, t in prof:
        if n in kb:
            base = n.replace("(conj)", "")
            agg.setdefault(base, []).append(t)
    dom_name = max(agg, key=lambda k: sum(agg[k]))
    dom_ms = sum(agg[dom_name]) / len(agg[dom_name])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = kb[dom_name] / (dom_ms * 1e-3) / 1e9
    fma_tflops = pdf.pdf_fp32_fma_peak(10)             # measured FP32 FMA peak (burst)
    if rep.loop_mode == 3 and loop_ms is not None:
        fl = cluster_flops(w, args.fold, args.fcnn) * w.iters
        ach32 = fl / (loop_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": "k_cluster_solve", "achieved": ach32, "peak": fma_tflops,
                    "unit": "TFLOP/s", "frac": ach32 / fma_tflops, "traffic": None,
                    "flops_per_launch": fl, "launch_ms": loop_ms,
                    "peak_derived": fp32_peak_tflops(peaks),
                    "note": "one launch runs the whole Adam loop; algorithmic FP32 flops (FFT convolutions, "
                            "Fourier synthesis/analysis, the folded data operator G_S Phi and its "
                            "adjoint, the network's products when it is on) / the launch's CUDA-event time "
                            "(solve minus the same solve with 0 iterations); peak = FP32 FMA throughput "
                            "measured by pdf_fp32_fma_peak on this GPU (peak_derived: 152 SMs x 128 FP32 "
                            "lanes x 2 x max SM clock); the loop is latency- and barrier-bound at this size; "
                            "traffic null: ncu does not capture this cluster launch",
                    "peak_source": "measured (FMA microbenchmark, burst)"}
    else:
        roofline = {"bound": "hbm", "kernel": KERNEL_OF_STAGE.get(dom_name, dom_name), "achieved": achieved,
                    "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                    "traffic": TRAFFIC_PER_LAUNCH.get((w.name, dom_name)),
                    "bytes_per_launch": kb[dom_name], "launch_ms": dom_ms,
                    "launches_per_iteration": len(agg[dom_name]),
                    "share_of_loss_grad": sum(agg[dom_name]) / per_iter_ms,
                    "note": "algorithmic bytes per launch (kernel_bytes, the per-kernel byte model) / the mean CUDA-event "
                            "duration of its launches inside one loss-and-gradient evaluation on the "
                            "launching stream; peak = the measured copy bandwidth; traffic = DRAM read + "
                            "write bytes per launch from one ncu capture of this kernel at this workload",
                    "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}

    # --- equal contrast RelErr: the split-BF16 tensor-core contractions against this solve ------
    eq = equal_relerr(w, args, esca_d, chi_d, net, rep.relerr_cco, total_ms / args.steps) if args.equal else None

    # --- operator assembly (pdf_setup), outside "ms per reconstruction": host geometry, the
    # FP64 Green's-function, incident-field and G_S assembly on the device, workspace allocation
    setup_ms = []
    for _ in range(3):
        torch.cuda.synchronize()
        t_setup = time.perf_counter()
        p2 = pdf.Problem.from_workload(w, precision=args.precision, fold_gs=args.fold)
        setup_ms.append((time.perf_counter() - t_setup) * 1e3)
        p2.close()

    # max over ranks
    ms_per_recon, e2e_per_recon, total_ms = combine_ranks(total_ms, e2e_ms, args.steps, world, "cuda")
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": ms_per_recon, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == 0 else "f32+bf16",
            "dtype_note": "complex64 (fp32 pairs) throughout, fp64 sums over incidences" if args.precision == 0 else
                          "complex64 FFT path, split-BF16 tensor-core contractions with fp32 accumulation, "
                          "fp64 sums over incidences",
            "data": "synthetic (seeded scene, GPU forward solver, AWGN)",
            "config": bench_config(w, args, world),
            "step_ms": {"median": statistics.median(step_ms), "min": min(step_ms), "max": max(step_ms),
                        "note": "rank 0's timed steps; value is their mean (max over ranks)"},
            "iters_per_s": (w.iters * world / (loop_ms * 1e-3)) if loop_ms else None,
            "iters_per_s_note": "iterations / loop time (the solve minus the same solve with 0 "
                                "iterations), all ranks",
            "hbm_model": hbm_model(w, loop_ms, peaks, args.fold),
            "equal_relerr": eq,
            "relerr": rep.relerr, "relerr_cco": rep.relerr_cco, "final_loss": rep.terms[0],
            "e2e": {"value": e2e_per_recon, "unit": "ms", "h2d_bytes_per_step": int(esca.nbytes),
                    "d2h_bytes_per_step": int(w.nx * w.ny * 8)},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "loop_mode": rep.loop_mode,
            "cluster_size": next((r[0] for r in pdf.pdf_cluster_plan(prob.h) if r[3]), None)
            if rep.loop_mode == 3 else None,
            "kernels_ms": {n: round(t, 5) for n, t in prof},
            "loss_grad_ms": per_iter_ms,
            "kernels_note": "kernels_ms / loss_grad_ms: one loss-and-gradient evaluation by the stand-alone "
                            "kernels (the graph loop's iteration), timed with events between launches",
            "clocks": clk,
            "wall_s": wall,
            "forward_solver_iters": fwd_iters,
            "setup_ms": {"first": setup_first_ms, "median_of_3": float(np.median(setup_ms)),
                         "note": "pdf_setup wall time (host geometry + FP64 operator assembly on the device + allocation), once per geometry, excluded from value"},
        }
        if not args.no_cpu:
            out["cpu_baseline"] = cpu_baseline(w, args.cpu_iters, args.fcnn)
    prob.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def _oracle_case(w, seed=0):
    from oracle.forward import forward_solve
    from oracle.green import Operators
    from oracle.problem import from_workload
    p = from_workload(w)
    ops = Operators(p)
    chi = scenes.make_scene(w, seed)
    _, _, esca = forward_solve(ops, chi)
    esca = scenes.add_awgn(esca, w.noise, np.random.default_rng(1000 + seed))
    return ops, esca, chi


def bench_workload(args):
    """The named workload, with --iters overriding its iteration count (both arms)."""
    if args.iters is not None:
        return scenes.workload(args.workload, iters=args.iters)
    return scenes.workload(args.workload)


def cpu_baseline(w, iters, fcnn=0, budget_s=15.0):
    """FP64 oracle on the host, every core through scipy.fft's workers: BP + CSI init, then Adam
    iterations (on alpha, or on the network's weights when fcnn > 0) until `budget_s` seconds of
    iterations have run (at least 2, at most `iters` and the workload's own count), scaled to a
    full reconstruction (init + w.iters iterations)."""
    from scipy import fft as sfft
    from oracle import fcnn as onet
    from oracle import loss, solve
    cores = os.cpu_count()
    with sfft.set_workers(cores):
        ops, esca, chi = _oracle_case(w)
        t0 = time.perf_counter()
        _, R0, _ = solve.bp_init(ops, esca)
        a = solve.csi_step(ops, esca, R0)
        t_init = time.perf_counter() - t0
        t0 = time.perf_counter()
        n = 0
        cap = min(iters, w.iters)
        if fcnn > 0:
            th = scenes.fcnn_params(w.ky, w.kx, fcnn, seed=0).astype(np.float64)
            opt = onet.AdamReal(lr=1e-2)
            while n < cap and (n < 2 or time.perf_counter() - t0 < budget_s):
                _, g = onet.loss_grad_theta(ops, esca, a, th, fcnn)
                th = opt.step(th, g)
                n += 1
        else:
            opt = solve.Adam(lr=1e-2)
            while n < cap and (n < 2 or time.perf_counter() - t0 < budget_s):
                _, g = loss.loss_grad(ops, esca, a)
                a = opt.step(a, g)
                n += 1
        t_it = (time.perf_counter() - t0) / max(n, 1)
    ms = (t_init + t_it * w.iters) * 1e3
    form = "on the network's weights" if fcnn > 0 else "on alpha"
    return {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": f"BP+CSI init ({t_init:.2f} s) + {n} Adam iterations {form} (FP64 NumPy/SciPy, "
                      f"{t_it:.3f} s each), the per-iteration time scaled to the workload's {w.iters}; "
                      f"scipy.fft workers = {cores}, BLAS threads default"}


def equal_relerr(w, args, esca_d, chi_d, net, target, ms_plain):
    """Wall time to the plain FP32 solve's final contrast RelErr (after CCO) with the split-BF16
    tensor-core contractions (precision 1), same form, start and data: a solve with a RelErr
    history every 5 iterations finds the first iteration count that reaches the target (the full
    count when only the final iterate does: the history stops before it), then a solve of exactly
    that many iterations is timed (CUDA events, median of 3 after one warm-up).
    The learned warm start is not part of this default comparison (it needs a trained network:
    bench.py --warm-start)."""
    import torch
    from paper_2602_13805_gb300 import pdf
    ch = pdf.Problem.from_workload(w, precision=1, fold_gs=args.fold)
    ch.set_data(esca_d)
    every = 5
    out = ch.solve(iters=w.iters, lr=args.lr, init=0, chi_true=chi_d, history_every=every, use_graph=args.loop, **net)
    h = out["history"].cpu().numpy()
    row = next((r for r in range(h.shape[0]) if h[r, 7] <= target), None)
    k = w.iters if row is None else row * every
    opts = pdf.solve_opts(iters=k, lr=args.lr, init=0, chi_true=chi_d, apply_cco=1, use_graph=args.loop, **net)
    chi_out = torch.empty((w.ny, w.nx), dtype=torch.complex64, device="cuda")
    _timed_solve(ch, opts, chi_out)
    ms = statistics.median(_timed_solve(ch, opts, chi_out) for _ in range(3))
    rep = pdf.pdf_solve(ch.h, opts, chi_out, None, None, report=True)
    ch.close()
    return {"target_relerr_cco": target, "plain": {"form": "FP32 contractions", "iters": w.iters, "ms": ms_plain,
                                                   "relerr_cco": target},
            "chosen": {"form": "split-BF16 tensor-core contractions (synthesis and analysis), FP32 FFT convolutions",
                       "iters_to_target": k, "reached": row is not None or rep.relerr_cco <= target, "ms": ms,
                       "relerr_cco": rep.relerr_cco},
            "speedup": ms_plain / ms,
            "note": "same network form, BP + CSI start and data; the chosen arm is timed for the first iteration "
                    "count (multiple of 5) whose RelErr after CCO is at or below the plain arm's final one"}


def _timed_solve(prob, opts, chi_out):
    """CUDA-event milliseconds of one pdf_solve on the current stream."""
    import torch
    from paper_2602_13805_gb300 import pdf
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    pdf.pdf_solve(prob.h, opts, chi_out, None, None, report=False)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def run_warm(args):
    """Learned warm start vs the plain FP32 solve at equal contrast RelErr (c4 / c5 shapes).

    For each held-out scene: the plain FP32 solve (BP + CSI, w.iters Adam iterations) gives the
    target RelErr (after CCO) and its time; the chosen form (network inference + warm-started solve
    at the requested precision, BP + CSI fallback) is run with a RelErr history to find the first
    iteration at which it reaches the target, and is then timed for exactly that many iterations."""
    import torch
    from paper_2602_13805_gb300 import pdf
    from paper_2602_13805_gb300.warmstart import WarmStartMLP, generate, predict_alpha, train
    w = bench_workload(args)
    prob = pdf.Problem.from_workload(w, fold_gs=args.fold)
    chosen = pdf.Problem.from_workload(w, precision=args.precision, fold_gs=args.fold)
    t0 = time.perf_counter()
    train_set = generate(prob, w, args.train_scenes, seed0=1000)
    test_set = generate(prob, w, args.test_scenes, seed0=0)
    t_data = time.perf_counter() - t0
    sizes = [2 * w.ni * w.nr, 1024, 1024, 1024, 2 * (1 + w.ni) * w.kx * w.ky]
    net = WarmStartMLP(sizes, batch_max=args.batch, seed=0)
    t0 = time.perf_counter()
    hist = train(net, train_set, steps=args.train_steps, batch=args.batch, lr=1e-3, log_every=max(1, args.train_steps // 10))
    t_train = time.perf_counter() - t0
    chi_out = torch.empty((w.ny, w.nx), dtype=torch.complex64, device="cuda")
    every = 5
    rows = []
    for s_ in range(args.test_scenes):
        esca = test_set.esca[s_].contiguous()
        chi_t = test_set.chi[s_].contiguous()
        prob.set_data(esca)
        chosen.set_data(esca)
        plain_opts = pdf.solve_opts(iters=w.iters, lr=args.lr, init=0, chi_true=chi_t, apply_cco=1, use_graph=args.loop)
        _timed_solve(prob, plain_opts, chi_out)                               # warm-up (graph build)
        ms_plain = _timed_solve(prob, plain_opts, chi_out)
        rep = pdf.pdf_solve(prob.h, plain_opts, chi_out, None, None, report=True)
        target = rep.relerr_cco
        # chosen form: inference + warm-started solve; find the iteration count reaching the target
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_ev.record()
        a0 = predict_alpha(net, esca, w)
        b_ev.record()
        torch.cuda.synchronize()
        ms_inf = a_ev.elapsed_time(b_ev)
        out = chosen.solve(iters=w.iters, lr=args.lr, init=3, alpha0=a0, chi_true=chi_t, history_every=every)
        h = out["history"].cpu().numpy()
        reach = next((r * every for r in range(h.shape[0]) if h[r, 7] <= target), None)
        k = w.iters if reach is None else reach
        opts_k = pdf.solve_opts(iters=k, lr=args.lr, init=3, alpha0=a0, chi_true=chi_t, apply_cco=1, use_graph=args.loop)
        _timed_solve(chosen, opts_k, chi_out)
        ms_chosen = ms_inf + _timed_solve(chosen, opts_k, chi_out)
        rows.append(dict(relerr_plain=target, relerr_chosen_final=out["relerr_cco"], iters_to_target=reach,
                         used_warm=out["used_warm_start"], ms_plain=ms_plain, ms_chosen=ms_chosen, ms_inference=ms_inf))
    net.close()
    reached = [r for r in rows if r["iters_to_target"] is not None]
    return {
        "metric": "ms to reach the plain FP32 solve's contrast RelErr", "unit": "ms", "higher_is_better": False,
        "value": float(np.mean([r["ms_chosen"] for r in rows])),
        "plain_fp32_ms": float(np.mean([r["ms_plain"] for r in rows])),
        "speedup": float(np.mean([r["ms_plain"] for r in rows]) / np.mean([r["ms_chosen"] for r in rows])),
        "reached": f"{len(reached)}/{len(rows)}",
        "mean_iters_to_target": float(np.mean([r["iters_to_target"] for r in reached])) if reached else None,
        "warm_start_kept": int(sum(r["used_warm"] for r in rows)),
        "relerr_plain_mean": float(np.mean([r["relerr_plain"] for r in rows])),
        "relerr_chosen_final_mean": float(np.mean([r["relerr_chosen_final"] for r in rows])),
        "config": {"workload": w.name, "train_scenes": args.train_scenes, "test_scenes": args.test_scenes,
                   "train_steps": args.train_steps, "batch": args.batch, "precision": args.precision,
                   "mlp": sizes, "iters": w.iters},
        "train_loss": hist, "data_seconds": t_data, "train_seconds": t_train, "per_scene": rows,
        "data": "synthetic (seeded scenes, GPU forward solver, 5-10% AWGN)",
    }


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w = bench_workload(args)
    iters = min(args.cpu_iters, w.iters)
    times = []
    # each step a bounded sample (a few seconds of iterations) so that W + K steps end in minutes
    budget = max(2.0, 60.0 / max(1, args.warmup + args.steps))
    r = None
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(w, iters, args.fcnn, budget_s=budget)
        if k >= args.warmup:
            times.append(r["value"])
    v = sum(times) / len(times)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded scene, oracle forward solver, AWGN)",
            "config": bench_config(w, args, world),
            "cpu_baseline": {"value": v, "unit": "ms", "cores": r["cores"], "kind": "oracle",
                             "sample": "per step: " + r["sample"]},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--fcnn", type=int, default=64,
                    help="hidden width of the coefficient-correcting network whose weights Adam optimises "
                         "(the paper's optimiser; 0: Adam on the coefficients directly)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c5")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iters", type=int, default=None)
    ap.add_argument("--lr", type=float, default=1e-2)
    ap.add_argument("--cpu-iters", type=int, default=50)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1])
    ap.add_argument("--warm-start", action="store_true")
    ap.add_argument("--no-equal", dest="equal", action="store_false",
                    help="skip the equal-RelErr comparison with the split-BF16 contractions")
    ap.add_argument("--loop", type=int, default=3, choices=[0, 1, 2, 3],
                    help="0 eager launches, 1 CUDA graph, 2 persistent cooperative kernel, "
                         "3 cluster kernel (default; the graph where the problem does not qualify)")
    ap.add_argument("--fold", type=int, default=1, choices=[0, 1],
                    help="1 data term through the folded operator G_S Phi (default), 0 G_S applied to J")
    ap.add_argument("--train-scenes", type=int, default=20000)
    ap.add_argument("--test-scenes", type=int, default=10)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=256)
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.warm_start:
        out = run_warm(args) if rank == 0 else None
    else:
        out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
