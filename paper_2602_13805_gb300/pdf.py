"""Thin Python binding of the C ABI in include/pdf.h (argument marshalling only).

Every numerical step runs in the CUDA library libpdf.so; this module only
converts torch tensors / numpy arrays to pointers and sizes and checks status
codes.  Importing it does not load the library; the first call does, and raises
PDFError if libpdf.so is missing (build it with paper_2602_13805_gb300.build).

Functions keep the C names: pdf_setup, pdf_set_data, pdf_loss_grad, pdf_apply_op,
pdf_solve, pdf_forward, pdf_destroy.  `Problem` bundles a handle with its sizes,
and `PDFLossGrad` exposes the loss/gradient to torch.autograd (Sec. 3.2; the
gradient is the library's hand-written adjoint).
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdf.so")

PDF_OK, PDF_EINVAL, PDF_ENOMEM, PDF_ECUDA, PDF_ENONFINITE, PDF_ETIMEOUT, PDF_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
OP_GD, OP_GDH, OP_GS, OP_GSH, OP_SYN, OP_ANA, OP_CCO, OP_CHI, OP_EINC = range(9)
TERM_NAMES = ("L", "State", "Data", "Bound", "TV", "Bridge")


class PDFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"pdf status {status}: {msg}")
        self.status = status


class pdf_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("side_x", ctypes.c_double), ("side_y", ctypes.c_double),
        ("k0", ctypes.c_double),
        ("ni", ctypes.c_int32), ("nr", ctypes.c_int32),
        ("tx_xy", ctypes.POINTER(ctypes.c_double)), ("rx_xy", ctypes.POINTER(ctypes.c_double)),
        ("inc_kind", ctypes.c_int32),
        ("kx", ctypes.c_int32), ("ky", ctypes.c_int32),
        ("beta_re", ctypes.c_double), ("beta_im", ctypes.c_double),
        ("lambda_bound", ctypes.c_double), ("lambda_tv", ctypes.c_double), ("lambda_bridge", ctypes.c_double),
        ("tau_b", ctypes.c_double), ("eps_tv", ctypes.c_double), ("eps_abs", ctypes.c_double),
        ("q_min", ctypes.c_double),
        ("precision", ctypes.c_int32), ("fft_path", ctypes.c_int32),
        ("fold_gs", ctypes.c_int32),
        ("cco_in_loss", ctypes.c_int32), ("cco_radius", ctypes.c_int32),
        ("cco_eps", ctypes.c_double), ("cco_eta_max", ctypes.c_double), ("cco_tau", ctypes.c_double),
        ("cco_delta", ctypes.c_double),
    ]


class pdf_solve_opts(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32), ("init", ctypes.c_int32),
        ("lr", ctypes.c_double), ("adam_b1", ctypes.c_double), ("adam_b2", ctypes.c_double),
        ("adam_eps", ctypes.c_double),
        ("alpha0", ctypes.c_void_p), ("chi_true", ctypes.c_void_p),
        ("apply_cco", ctypes.c_int32), ("cco_radius", ctypes.c_int32),
        ("cco_eps", ctypes.c_double), ("cco_eta_max", ctypes.c_double), ("cco_tau", ctypes.c_double),
        ("cco_delta", ctypes.c_double),
        ("use_graph", ctypes.c_int32), ("history_every", ctypes.c_int32),
        ("history", ctypes.c_void_p),
        ("fcnn_hidden", ctypes.c_int32), ("fcnn_params0", ctypes.c_void_p),
        ("barrier_wait_cycles", ctypes.c_int64),
    ]


class pdf_solve_report(ctypes.Structure):
    _fields_ = [
        ("iters_run", ctypes.c_int32), ("nonfinite", ctypes.c_int32),
        ("terms", ctypes.c_double * 6),
        ("relerr", ctypes.c_double), ("relerr_cco", ctypes.c_double),
        ("used_warm_start", ctypes.c_int32), ("loop_mode", ctypes.c_int32),
    ]


_lib = None

EXPORTS = ("pdf_config_default", "pdf_setup", "pdf_set_data", "pdf_loss_grad", "pdf_apply_op",
           "pdf_solve_opts_default", "pdf_solve", "pdf_forward", "pdf_launch_count", "pdf_destroy",
           "pdf_last_error", "pdf_profile_loss_grad", "pdf_kernel_name", "pdf_gs_apply_static",
           "pdf_stage_name", "pdf_mlp_create", "pdf_mlp_destroy", "pdf_mlp_set_params", "pdf_mlp_get_params",
           "pdf_mlp_forward", "pdf_mlp_loss_grad", "pdf_mlp_train_step", "pdf_mlp_error_flag",
           "pdf_phase_stamps", "pdf_cluster_plan", "pdf_fp32_fma_peak", "pdf_mlp_features")


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libpdf.so (once) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise PDFError(PDF_EUNSUPPORTED, f"{path} is missing: build it with `python -m paper_2602_13805_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    lib.pdf_config_default.argtypes = [ctypes.POINTER(pdf_config)]
    lib.pdf_config_default.restype = None
    lib.pdf_setup.argtypes = [ctypes.POINTER(pdf_config), vp, ctypes.c_int, vp, ctypes.POINTER(vp)]
    lib.pdf_setup.restype = ctypes.c_int
    lib.pdf_set_data.argtypes = [vp, vp, ctypes.c_int, vp]
    lib.pdf_set_data.restype = ctypes.c_int
    lib.pdf_loss_grad.argtypes = [vp, vp, vp, vp, vp]
    lib.pdf_loss_grad.restype = ctypes.c_int
    lib.pdf_apply_op.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.pdf_apply_op.restype = ctypes.c_int
    lib.pdf_solve_opts_default.argtypes = [ctypes.POINTER(pdf_solve_opts)]
    lib.pdf_solve_opts_default.restype = None
    lib.pdf_solve.argtypes = [vp, ctypes.POINTER(pdf_solve_opts), vp, vp, vp, ctypes.POINTER(pdf_solve_report), vp]
    lib.pdf_solve.restype = ctypes.c_int
    lib.pdf_forward.argtypes = [vp, vp, vp, vp, dbl, i32, ctypes.POINTER(i32), vp]
    lib.pdf_forward.restype = ctypes.c_int
    lib.pdf_launch_count.argtypes = []
    lib.pdf_launch_count.restype = ctypes.c_uint64
    lib.pdf_destroy.argtypes = [vp]
    lib.pdf_destroy.restype = None
    lib.pdf_profile_loss_grad.argtypes = [vp, vp, i32, ctypes.POINTER(ctypes.c_float), i32, vp]
    lib.pdf_profile_loss_grad.restype = i32
    lib.pdf_phase_stamps.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    lib.pdf_phase_stamps.restype = ctypes.c_int
    lib.pdf_fp32_fma_peak.argtypes = [i32, ctypes.POINTER(dbl), vp]
    lib.pdf_fp32_fma_peak.restype = ctypes.c_int
    lib.pdf_cluster_plan.argtypes = [vp, ctypes.POINTER(i32), i32]
    lib.pdf_cluster_plan.restype = i32
    lib.pdf_kernel_name.argtypes = [i32]
    lib.pdf_kernel_name.restype = ctypes.c_char_p
    lib.pdf_stage_name.argtypes = [vp, i32]
    lib.pdf_stage_name.restype = ctypes.c_char_p
    lib.pdf_gs_apply_static.argtypes = [vp, vp, vp, i32, i32, i32, vp]
    lib.pdf_gs_apply_static.restype = ctypes.c_int
    lib.pdf_mlp_create.argtypes = [i32, ctypes.POINTER(i32), i32, ctypes.POINTER(vp)]
    lib.pdf_mlp_create.restype = ctypes.c_int
    lib.pdf_mlp_destroy.argtypes = [vp]
    lib.pdf_mlp_destroy.restype = None
    lib.pdf_mlp_set_params.argtypes = [vp, i32, vp, vp, vp]
    lib.pdf_mlp_set_params.restype = ctypes.c_int
    lib.pdf_mlp_get_params.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    lib.pdf_mlp_get_params.restype = ctypes.c_int
    lib.pdf_mlp_forward.argtypes = [vp, vp, vp, i32, vp]
    lib.pdf_mlp_forward.restype = ctypes.c_int
    lib.pdf_mlp_loss_grad.argtypes = [vp, vp, vp, i32, vp, vp]
    lib.pdf_mlp_loss_grad.restype = ctypes.c_int
    lib.pdf_mlp_train_step.argtypes = [vp, vp, vp, i32, dbl, vp, vp]
    lib.pdf_mlp_train_step.restype = ctypes.c_int
    lib.pdf_mlp_error_flag.argtypes = [vp]
    lib.pdf_mlp_error_flag.restype = i32
    lib.pdf_mlp_features.argtypes = [vp, i32, i32, vp, vp]
    lib.pdf_mlp_features.restype = ctypes.c_int
    lib.pdf_last_error.argtypes = []
    lib.pdf_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(st: int):
    if st != PDF_OK:
        raise PDFError(st, load().pdf_last_error().decode(errors="replace"))


def _ptr(t) -> Optional[int]:
    """Device (torch CUDA tensor) or host (numpy) pointer; None stays None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


# ---------------------------------------------------------------------------
# C-named entry points
# ---------------------------------------------------------------------------

def make_config(nx, ny, side_x, side_y, k0, tx, rx, kx, ky, beta=6.0 + 0j, inc_kind=0, precision=0,
                lambda_bound=1e-3, lambda_tv=1e-5, lambda_bridge=1e-5, tau_b=0.5, eps_tv=1e-8, eps_abs=1e-12,
                q_min=1e-6, fft_path=0, fold_gs=1, cco_in_loss=0, cco_radius=2, cco_eps=1e-2, cco_eta_max=0.1,
                cco_tau=3.0, cco_delta=0.5):
    """Returns (pdf_config, keep-alive antenna arrays)."""
    lib = load()
    c = pdf_config()
    lib.pdf_config_default(ctypes.byref(c))
    tx = np.ascontiguousarray(tx, dtype=np.float64)
    rx = np.ascontiguousarray(rx, dtype=np.float64)
    c.nx, c.ny, c.side_x, c.side_y, c.k0 = nx, ny, side_x, side_y, k0
    c.ni, c.nr = tx.shape[0], rx.shape[0]
    c.tx_xy = tx.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    c.rx_xy = rx.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    c.inc_kind, c.kx, c.ky = inc_kind, kx, ky
    beta = complex(beta)
    c.beta_re, c.beta_im = beta.real, beta.imag
    c.lambda_bound, c.lambda_tv, c.lambda_bridge = lambda_bound, lambda_tv, lambda_bridge
    c.tau_b, c.eps_tv, c.eps_abs, c.q_min = tau_b, eps_tv, eps_abs, q_min
    c.precision = precision
    c.fft_path = fft_path
    c.fold_gs = fold_gs
    c.cco_in_loss, c.cco_radius = int(cco_in_loss), cco_radius
    c.cco_eps, c.cco_eta_max, c.cco_tau, c.cco_delta = cco_eps, cco_eta_max, cco_tau, cco_delta
    return c, (tx, rx)


def pdf_setup(cfg: pdf_config, esca=None, stream=None) -> int:
    """esca: host numpy complex64 [ni][nr], a CUDA tensor, or None."""
    lib = load()
    h = ctypes.c_void_p()
    on_dev = 0 if (esca is None or isinstance(esca, np.ndarray)) else 1
    if isinstance(esca, np.ndarray):
        esca = np.ascontiguousarray(esca, dtype=np.complex64)
    _check(lib.pdf_setup(ctypes.byref(cfg), _ptr(esca), on_dev, _stream(stream), ctypes.byref(h)))
    return h.value


def pdf_set_data(h: int, esca, stream=None):
    on_dev = 0 if isinstance(esca, np.ndarray) else 1
    if isinstance(esca, np.ndarray):
        esca = np.ascontiguousarray(esca, dtype=np.complex64)
    _check(load().pdf_set_data(h, _ptr(esca), on_dev, _stream(stream)))


def pdf_loss_grad(h: int, alpha, grad=None, terms=None, stream=None):
    _check(load().pdf_loss_grad(h, _ptr(alpha), _ptr(grad), _ptr(terms), _stream(stream)))


def pdf_apply_op(h: int, op: int, x, out, stream=None):
    _check(load().pdf_apply_op(h, op, _ptr(x), _ptr(out), _stream(stream)))


def pdf_cluster_plan(h: int):
    """[(C, smem bytes, co-resident clusters, usable)] the cluster loop would consider for handle h."""
    buf = (ctypes.c_int32 * 20)()
    n = load().pdf_cluster_plan(h, buf, 5)
    if n < 0:
        _check(n)
    return [tuple(buf[4 * i: 4 * i + 4]) for i in range(n)]


def pdf_solve(h: int, opts: pdf_solve_opts, chi_out=None, chi_raw_out=None, alpha_out=None, report=True,
              stream=None) -> Optional[pdf_solve_report]:
    rep = pdf_solve_report() if report else None
    _check(load().pdf_solve(h, ctypes.byref(opts), _ptr(chi_out), _ptr(chi_raw_out), _ptr(alpha_out),
                            ctypes.byref(rep) if rep is not None else None, _stream(stream)))
    return rep


def pdf_forward(h: int, chi, esca_out, j_out=None, tol=1e-6, max_iter=2000, stream=None) -> int:
    it = ctypes.c_int32(0)
    _check(load().pdf_forward(h, _ptr(chi), _ptr(esca_out), _ptr(j_out), tol, max_iter, ctypes.byref(it),
                              _stream(stream)))
    return it.value


def pdf_gs_apply_static(gs, x, out, stream=None):
    """out[p][r] = sum_n gs[r][n] x[p][n] with no device allocation (static library scratch).

    gs [nr][m...], x [ni][m...] and out [ni][nr] must be contiguous CUDA complex64 tensors without
    a pending lazy conjugation (the library reads their raw device memory); anything else raises
    ValueError before the library is called."""
    import torch
    for name, t in (("gs", gs), ("x", x), ("out", out)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor on the GPU, not {type(t).__name__}")
        if t.dim() < 2 or t.dtype != torch.complex64:
            raise ValueError(f"{name} must be a complex64 tensor of at least two dimensions")
    nr = gs.shape[0]
    m = gs.numel() // max(nr, 1)
    ni = x.shape[0]
    if nr < 1 or m < 1 or ni < 1 or gs.numel() != nr * m or x.numel() != ni * m or out.numel() != ni * nr:
        raise ValueError(f"sizes do not match: gs {tuple(gs.shape)} ([nr][m]), x {tuple(x.shape)} ([ni][m]), "
                         f"out {tuple(out.shape)} ([ni][nr])")
    for name, t in (("gs", gs), ("x", x), ("out", out)):
        if not t.is_cuda:
            raise ValueError(f"{name} must be on the GPU")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.is_conj():
            raise ValueError(f"{name} carries a lazy conjugation: pass torch.conj_physical(...)")
    _check(load().pdf_gs_apply_static(gs.data_ptr(), x.data_ptr(), out.data_ptr(), ni, nr, m, _stream(stream)))


def pdf_destroy(h: int):
    if h:
        load().pdf_destroy(h)


def pdf_launch_count() -> int:
    return int(load().pdf_launch_count())


def pdf_fp32_fma_peak(reps: int = 10, stream=None) -> float:
    """Measured FP32 FMA throughput of the current device, TFLOP/s."""
    out = ctypes.c_double(0.0)
    _check(load().pdf_fp32_fma_peak(reps, ctypes.byref(out), _stream(stream)))
    return out.value


def pdf_profile_loss_grad(h: int, alpha, reps: int = 20, stream=None):
    """{kernel name: mean ms per launch} for the kernels of one pdf_loss_grad (CUDA events)."""
    lib = load()
    buf = (ctypes.c_float * 64)()
    k = lib.pdf_profile_loss_grad(h, _ptr(alpha), reps, buf, 64, _stream(stream))
    if k < 0:
        _check(k)
    return [(lib.pdf_stage_name(h, i).decode(), float(buf[i])) for i in range(k)]


def solve_opts(**kw) -> pdf_solve_opts:
    o = pdf_solve_opts()
    load().pdf_solve_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k in ("alpha0", "chi_true", "history", "fcnn_params0"):
            v = _ptr(v)
        setattr(o, k, v)
    return o


# ---------------------------------------------------------------------------
# convenience handle + autograd
# ---------------------------------------------------------------------------

class Problem:
    """A pdf_problem handle with its sizes (device tensors are torch complex64 on CUDA)."""

    def __init__(self, nx, ny, side_x, side_y, k0, tx, rx, kx, ky, esca=None, stream=None, **kw):
        self.cfg, self._keep = make_config(nx, ny, side_x, side_y, k0, tx, rx, kx, ky, **kw)
        self.nx, self.ny, self.kx, self.ky = nx, ny, kx, ky
        self.ni, self.nr = self.cfg.ni, self.cfg.nr
        self.h = pdf_setup(self.cfg, esca, stream)

    @classmethod
    def from_workload(cls, w, tx=None, rx=None, esca=None, **kw):
        import scenes
        if tx is None or rx is None:
            t, r = scenes.geometry(w)
            tx = t if tx is None else tx
            rx = r if rx is None else rx
        return cls(w.nx, w.ny, w.side, w.side, w.k0, tx, rx, w.kx, w.ky, esca=esca, beta=w.beta,
                   inc_kind=w.inc_kind, **kw)

    def close(self):
        if getattr(self, "h", None):
            pdf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _t(self, *shape):
        import torch
        return torch.empty(shape, dtype=torch.complex64, device="cuda")

    def set_data(self, esca, stream=None):
        pdf_set_data(self.h, esca, stream)

    def loss_grad(self, alpha, stream=None):
        import torch
        grad = torch.empty_like(alpha)
        terms = torch.empty(6, dtype=torch.float64, device=alpha.device)
        pdf_loss_grad(self.h, alpha, grad, terms, stream)
        return terms, grad

    def op(self, op, x, stream=None):
        out_shape = {OP_GD: (self.ni, self.ny, self.nx), OP_GDH: (self.ni, self.ny, self.nx),
                     OP_GS: (self.ni, self.nr), OP_GSH: (self.ni, self.ny, self.nx),
                     OP_SYN: (self.ni, self.ny, self.nx), OP_ANA: (self.ni, self.ky, self.kx),
                     OP_CCO: (self.ny, self.nx), OP_CHI: (self.ny, self.nx),
                     OP_EINC: (self.ni, self.ny, self.nx)}[op]
        out = self._t(*out_shape)
        pdf_apply_op(self.h, op, x, out, stream)
        return out

    def solve(self, iters=300, lr=1e-2, init=0, alpha0=None, chi_true=None, apply_cco=True, use_graph=3,
              history_every=0, stream=None, **kw):
        import torch
        hist = None
        if history_every > 0:
            hist = torch.full((math.ceil(iters / history_every), 8), float("nan"), dtype=torch.float64, device="cuda")
        o = solve_opts(iters=iters, lr=lr, init=init, alpha0=alpha0, chi_true=chi_true, apply_cco=int(apply_cco),
                       use_graph=int(use_graph), history_every=history_every, history=hist, **kw)
        chi = self._t(self.ny, self.nx)
        chi_raw = self._t(self.ny, self.nx)
        alpha = self._t(self.ni, self.ky, self.kx)
        rep = pdf_solve(self.h, o, chi, chi_raw, alpha, True, stream)
        return dict(chi=chi, chi_raw=chi_raw, alpha=alpha, terms=np.array(rep.terms[:]), relerr=rep.relerr,
                    relerr_cco=rep.relerr_cco, history=hist, used_warm_start=rep.used_warm_start,
                    loop_mode=rep.loop_mode)

    def forward(self, chi, tol=1e-6, max_iter=2000, stream=None):
        esca = self._t(self.ni, self.nr)
        J = self._t(self.ni, self.ny, self.nx)
        it = pdf_forward(self.h, chi, esca, J, tol, max_iter, stream)
        return esca, J, it


def _autograd():
    import torch

    class PDFLossGrad(torch.autograd.Function):
        """L(alpha) of Eq. (13) with the library's hand-written adjoint as the backward."""

        @staticmethod
        def forward(ctx, alpha, problem):
            a = alpha.detach().contiguous()
            terms, grad = problem.loss_grad(a)
            ctx.save_for_backward(grad)
            return terms[0].to(torch.float32) if alpha.dtype == torch.complex64 else terms[0]

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            return grad * gout.to(grad.real.dtype), None

    return PDFLossGrad


_PDFLossGrad = None


def pdf_loss(alpha, problem: Problem):
    """Differentiable loss: PDFLossGrad.apply(alpha, problem)."""
    global _PDFLossGrad
    if _PDFLossGrad is None:
        _PDFLossGrad = _autograd()
    return _PDFLossGrad.apply(alpha, problem)


def PDFLossGrad():
    global _PDFLossGrad
    if _PDFLossGrad is None:
        _PDFLossGrad = _autograd()
    return _PDFLossGrad
