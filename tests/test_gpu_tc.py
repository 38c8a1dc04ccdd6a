"""Split-BF16 tensor-core path (precision = 1) against the FP64 oracle.

The contractions (Fourier synthesis/analysis, G_S and G_S^H) run as tcgen05 GEMMs on
hi/lo BF16 pairs with FP32 accumulation.  The contract's bound for this path is 1e-2;
the three-product split keeps ~16 mantissa bits, so the tests ask for 1e-4 and report.
"""
import numpy as np
import pytest

import scenes
from oracle import fbe, loss, solve
from tests.gpu_common import Case, assert_close, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_TC = 1e-4


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# fold 0: G_S and G_S^H as tensor-core GEMMs on the synthesised currents; fold 1 (default): the
# data term through the folded operator, the tensor cores then carry synthesis and analysis
@pytest.fixture(scope="module", params=[("g24x20", dict(nx=24, ny=20, ni=5, nr=7, kx=7, ky=5), 0),
                                        ("c1", dict(), 0), ("c2", None, 0), ("c1-fold", dict(), 1),
                                        ("c2-fold", None, 1)], ids=lambda c: c[0])
def case(request):
    name, over, fold = request.param
    w = scenes.workload("c2") if over is None else scenes.workload("c1", **over)
    c = Case(w)
    c.prob = c.problem(precision=1, fold_gs=fold)
    yield c
    c.prob.close()


def test_tc_operators(case):
    from paper_2602_13805_gb300 import pdf
    p, ops, prob = case.p, case.ops, case.prob
    rng = np.random.default_rng(3)
    x = (rng.standard_normal((p.ni, p.ny, p.nx)) + 1j * rng.standard_normal((p.ni, p.ny, p.nx))).astype(np.complex64)
    d = (rng.standard_normal((p.ni, p.nr)) + 1j * rng.standard_normal((p.ni, p.nr))).astype(np.complex64)
    a = case.alpha()
    checks = {
        "GS": (prob.op(pdf.OP_GS, _dev(x)), ops.gs(x.astype(complex))),
        "GSH": (prob.op(pdf.OP_GSH, _dev(d)), ops.gsh(d.astype(complex))),
        "SYN": (prob.op(pdf.OP_SYN, _dev(a)), fbe.synth(a.astype(complex), p.ny, p.nx)),
        "ANA": (prob.op(pdf.OP_ANA, _dev(x)), fbe.analysis(x.astype(complex), p.ky, p.kx)),
    }
    for k, (gpu, ref) in checks.items():
        assert_close(k, gpu, ref, TOL_TC)


def test_tc_loss_and_gradient(case):
    p, ops, prob = case.p, case.ops, case.prob
    a = case.alpha(scale=0.3, seed=7)
    terms, grad = prob.loss_grad(_dev(a))
    t_ref, g_ref = loss.loss_grad(ops, case.esca, a.astype(complex))
    t = terms.cpu().numpy()
    el = abs(t[0] - t_ref[0]) / abs(t_ref[0])
    print(f"loss rel {el:.2e}")
    assert el < TOL_TC
    assert_close("gradient", grad, g_ref, TOL_TC)


def test_tc_solve_relerr_close_to_oracle():
    w = scenes.workload("c1", iters=60)
    c = Case(w)
    prob = c.problem(precision=1)
    out = prob.solve(iters=w.iters, chi_true=_dev(c.chi.astype(np.complex64)))
    ref = solve.pdf_solve(c.ops, c.esca, w.iters, chi_true=c.chi)
    print("relerr tc", out["relerr_cco"], "oracle", ref["relerr_cco"])
    assert abs(out["relerr_cco"] - ref["relerr_cco"]) < 1e-3
    prob.close()
