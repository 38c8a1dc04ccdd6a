"""The allocation-free entry point pdf_gs_apply_static against the handle path's PDF_OP_GS.

pdf_gs_apply_static serves callers that cannot call cudaMalloc (their device memory is owned
by another allocator, or their loop cannot afford an allocation's device synchronisation); it
keeps its split-K partial sums in a fixed 4 MiB device array inside the library.  This file
runs last so that a failure here does not hide the other GPU tests; it passes alone or after
them (it builds its own inputs).
"""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5          # the FP32 parity tolerance used by the other GPU tests (norm-wise relative)


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_static_scratch_gs_matches_handle_path_twice():
    from paper_2602_13805_gb300 import build, pdf
    build.build()
    w = scenes.workload("c2", ni=32, nr=32)          # ni == nr: G_S is recoverable from G_S^H of the identity
    esca = np.ones((w.ni, w.nr), np.complex64)
    prob = pdf.Problem.from_workload(w, esca=esca)
    m = w.nx * w.ny
    eye = torch.eye(w.nr, dtype=torch.complex64, device="cuda").contiguous()
    # conj_physical: torch.conj only sets a lazy flag, and the library reads raw memory
    gs = torch.conj_physical(prob.op(pdf.OP_GSH, eye)).reshape(w.nr, m).contiguous()   # the handle's G_S
    rng = np.random.default_rng(0)
    for call in range(2):                          # two calls in a row share the static scratch
        x = torch.from_numpy((rng.standard_normal((w.ni, w.ny, w.nx)) +
                              1j * rng.standard_normal((w.ni, w.ny, w.nx))).astype(np.complex64)).cuda()
        ref = prob.op(pdf.OP_GS, x)
        out = torch.full((w.ni, w.nr), float("nan"), dtype=torch.complex64, device="cuda")
        pdf.pdf_gs_apply_static(gs, x.reshape(w.ni, m).contiguous(), out)
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(out)).all()
        assert _rel(out, ref) < TOL, f"call {call}: rel err {_rel(out, ref):.2e}"
    prob.close()


def test_static_scratch_rejects_oversize():
    import ctypes
    from paper_2602_13805_gb300 import pdf
    lib = pdf.load()
    dummy = torch.zeros(1, dtype=torch.complex64, device="cuda")
    p = dummy.data_ptr()
    st = lib.pdf_gs_apply_static(p, p, p, 1024, 1024, 16, None)
    assert st == pdf.PDF_EINVAL
    assert b"static scratch" in lib.pdf_last_error()
