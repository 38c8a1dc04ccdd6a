"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports every
symbol include/pdf.h declares, and rejects invalid configurations before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_13805_gb300 import build, pdf
    build.build()
    return pdf.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pdf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pdf_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert "pdf_loss_grad" in syms and "pdf_setup" in syms and "pdf_solve" in syms
    for s in syms:
        assert hasattr(lib, s), f"{s} not exported"


def test_binding_names_match_header():
    from paper_2602_13805_gb300 import pdf
    for s in declared_symbols():
        assert s in pdf.EXPORTS


def test_struct_layouts_match_header(lib):
    # pdf_config_default writes the paper's defaults through the binding's struct layout
    from paper_2602_13805_gb300 import pdf
    c = pdf.pdf_config()
    lib.pdf_config_default(ctypes.byref(c))
    assert c.beta_re == 6.0 and c.lambda_bound == 1e-3 and c.lambda_tv == 1e-5 and c.tau_b == 0.5
    assert abs(c.k0 - 2 * np.pi) < 1e-15
    o = pdf.pdf_solve_opts()
    lib.pdf_solve_opts_default(ctypes.byref(o))
    assert o.iters == 300 and o.lr == 1e-2 and o.adam_b2 == 0.999 and o.cco_radius == 2 and o.use_graph == 3


@pytest.mark.parametrize("field,value,status", [
    ("nx", 1, -1), ("nx", 300, -6), ("kx", 0, -1), ("kx", 40, -1), ("ni", 0, -1),
    ("beta_re", -1.0, -1), ("side_x", 0.0, -1), ("inc_kind", 3, -1), ("precision", 5, -1),
])
def test_invalid_config_rejected_without_gpu(lib, field, value, status):
    from paper_2602_13805_gb300 import pdf
    tx = np.zeros((4, 2))
    rx = np.zeros((8, 2))
    c, keep = pdf.make_config(32, 32, 2.0, 2.0, 2 * np.pi, tx, rx, 11, 11)
    setattr(c, field, value)
    h = ctypes.c_void_p()
    st = lib.pdf_setup(ctypes.byref(c), None, 0, None, ctypes.byref(h))
    assert st == status
    assert h.value is None
    assert len(lib.pdf_last_error()) > 0


def test_null_arguments_rejected(lib):
    assert lib.pdf_loss_grad(None, None, None, None, None) == -1
    assert lib.pdf_solve(None, None, None, None, None, None, None) == -1
    assert lib.pdf_apply_op(None, 0, None, None, None) == -1
    lib.pdf_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2602_13805_gb300 import pdf
    with pytest.raises(pdf.PDFError):
        pdf.load.__wrapped__(str(tmp_path / "nope.so")) if hasattr(pdf.load, "__wrapped__") else \
            _load_fresh(pdf, str(tmp_path / "nope.so"))


def _load_fresh(pdf, path):
    saved = pdf._lib
    pdf._lib = None
    try:
        pdf.load(path)
    finally:
        pdf._lib = saved


def test_fma_peak_rejects_bad_arguments_without_gpu(lib):
    out = ctypes.c_double(0.0)
    assert lib.pdf_fp32_fma_peak(0, ctypes.byref(out), None) == -1
    assert lib.pdf_fp32_fma_peak(3, None, None) == -1


def test_static_gs_wrapper_rejects_host_and_missized_arguments():
    # checked before the library is called: a host pointer or a short array would reach the device
    torch = pytest.importorskip("torch")
    from paper_2602_13805_gb300 import pdf
    gs = torch.zeros((4, 6), dtype=torch.complex64)
    x = torch.zeros((3, 6), dtype=torch.complex64)
    out = torch.zeros((3, 4), dtype=torch.complex64)
    with pytest.raises(ValueError, match="torch tensor"):
        pdf.pdf_gs_apply_static(gs.numpy(), x, out)
    with pytest.raises(ValueError, match="complex64"):
        pdf.pdf_gs_apply_static(gs.to(torch.complex128), x, out)
    with pytest.raises(ValueError, match="sizes"):
        pdf.pdf_gs_apply_static(gs, torch.zeros((3, 5), dtype=torch.complex64), out)
    with pytest.raises(ValueError, match="sizes"):
        pdf.pdf_gs_apply_static(gs, x, torch.zeros((3, 3), dtype=torch.complex64))
    with pytest.raises(ValueError, match="GPU"):
        pdf.pdf_gs_apply_static(gs, x, out)              # right sizes, host memory
