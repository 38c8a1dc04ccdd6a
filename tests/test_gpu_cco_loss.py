"""The CCO inside the loss (pdf_config.cco_in_loss, Sec. 2.4 Eq. 10-11 in the regularisers) on the
GPU against the FP64 oracle: loss terms and gradient element by element, and whole solves.

Two weightings: the paper's (lambda 1e-3 / 1e-5 / 1e-5, CCO gain centred at |chi| = 3), where the
regulariser path is a small share of the gradient, and a heavy one (lambdas 1 / 0.3 / 0.5, gain
centred on the contrast present), where the CCO's adjoint carries a large share of it.
"""
import numpy as np
import pytest

import scenes
from oracle import loss, solve
from tests.gpu_common import TOL_FP32, Case, assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HEAVY = dict(lambda_bound=1.0, lambda_tv=0.3, lambda_bridge=0.5, cco_tau=0.3, cco_delta=0.2)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _case(name, over, weights):
    w = scenes.workload(name, **over)
    c = Case(w)
    kw = dict(cco_in_loss=1, **weights)
    prob = c.problem(**kw)
    p = c.p
    p.cco_in_loss = True
    p.lam_bound = kw.get("lambda_bound", p.lam_bound)
    p.lam_tv = kw.get("lambda_tv", p.lam_tv)
    p.lam_bridge = kw.get("lambda_bridge", p.lam_bridge)
    p.cco_tau = kw.get("cco_tau", p.cco_tau)
    p.cco_delta = kw.get("cco_delta", p.cco_delta)
    return c, prob


CASES = [("g24x20", "c1", dict(nx=24, ny=20, ni=5, nr=7, kx=7, ky=5)), ("c1", "c1", {}), ("c2", "c2", {}),
         ("g256", "c1", dict(nx=256, ny=256, ni=2, nr=8, kx=9, ky=9))]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
@pytest.mark.parametrize("weights", ["paper", "heavy"])
def test_cco_in_loss_loss_and_gradient(case, weights):
    name, base, over = case
    c, prob = _case(base, over, HEAVY if weights == "heavy" else {})
    a = c.alpha(scale=0.3, seed=7)
    terms, grad = prob.loss_grad(_dev(a))
    t_ref, g_ref = loss.loss_grad(c.ops, c.esca, a.astype(complex))
    t = terms.cpu().numpy()
    print(name, weights, "terms", t, "oracle", t_ref)
    for k in range(3):
        assert abs(t[k] - t_ref[k]) <= TOL_FP32 * abs(t_ref[k]), (k, t[k], t_ref[k])
    for k in (3, 4, 5):
        assert abs(t[k] - t_ref[k]) <= 1e-4 * max(abs(t_ref[k]), 1e-6), (k, t[k], t_ref[k])
    # the heavy weighting puts the regularisers' chi-hat amplification (1 / |1 - R|^2) into the
    # gradient, as in the plain heavy-regulariser test: 1e-4 there
    assert_close(f"{name} {weights} gradient", grad, g_ref, TOL_FP32 if weights == "paper" else 1e-4)
    prob.close()


def test_cco_in_loss_changes_the_gradient():
    c, prob = _case("c1", dict(nx=24, ny=20, ni=5, nr=7, kx=7, ky=5), HEAVY)
    plain = c.problem(**{k: v for k, v in HEAVY.items()})
    a = _dev(c.alpha(scale=0.3, seed=7))
    _, g1 = prob.loss_grad(a)
    _, g0 = plain.loss_grad(a)
    assert (g1 - g0).abs().max().item() > 1e-3 * g1.abs().max().item()
    prob.close()
    plain.close()


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_cco_in_loss_solve_matches_oracle(name):
    w = scenes.workload(name, iters=40)
    c, prob = _case(name, dict(iters=40), {})
    chi_t = _dev(c.chi.astype(np.complex64))
    out = prob.solve(iters=w.iters, chi_true=chi_t, use_graph=3)
    assert out["loop_mode"] == 1                     # the one-launch loops do not carry the CCO
    ref = solve.pdf_solve(c.ops, c.esca, w.iters, chi_true=c.chi)
    print(name, "RelErr (CCO)", out["relerr_cco"], "oracle", ref["relerr_cco"])
    assert abs(out["relerr"] - ref["relerr"]) < 1e-3
    assert abs(out["relerr_cco"] - ref["relerr_cco"]) < 1e-3
    prob.close()
