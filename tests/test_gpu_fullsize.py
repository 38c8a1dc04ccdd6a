"""Parity at the full sizes of the large workloads, in the configuration bench.py times.

128x128 / Ni=36 / Nr=72 / K=21 and 192x192 / Ni=64 / Nr=128 / K=31: loss terms and the whole
gradient against the FP64 oracle, for the FP32 path and the split-BF16 tensor-core path.  The
measured data are seeded random complex values (any E_sca is a valid input of Eq. 16), so no
oracle input comes from the CUDA path and the oracle needs no forward solve at these sizes.
"""
import numpy as np
import pytest

import scenes
from oracle import loss
from oracle.green import Operators
from oracle.problem import from_workload
from tests.gpu_common import TOL_FP32, assert_close, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["c3", "c5"])
def big(request):
    w = scenes.workload(request.param)
    p = from_workload(w)
    ops = Operators(p)
    rng = np.random.default_rng(42)
    esca = (rng.standard_normal((w.ni, w.nr)) + 1j * rng.standard_normal((w.ni, w.nr))).astype(np.complex64)
    a = scenes.random_coeffs(w.ni, w.ky, w.kx, 0.3, rng).astype(np.complex64)
    t_ref, g_ref = loss.loss_grad(ops, esca.astype(complex), a.astype(complex))
    return w, esca, a, t_ref, g_ref


@pytest.mark.parametrize("precision,fold", [(0, 1), (1, 1), (0, 0), (1, 0)])
def test_fullsize_loss_gradient(big, precision, fold):
    from paper_2602_13805_gb300 import pdf
    w, esca, a, t_ref, g_ref = big
    prob = pdf.Problem.from_workload(w, esca=esca, precision=precision, fold_gs=fold)
    terms, grad = prob.loss_grad(torch.from_numpy(a).cuda())
    t = terms.cpu().numpy()
    eg = rel(grad.cpu().numpy(), g_ref)
    print(w.name, precision, fold, "loss rel", abs(t[0] - t_ref[0]) / abs(t_ref[0]), "grad rel", eg)
    for k in range(3):
        assert abs(t[k] - t_ref[k]) <= TOL_FP32 * abs(t_ref[k])
    assert_close(f"{w.name} gradient", grad, g_ref, TOL_FP32)
    prob.close()
