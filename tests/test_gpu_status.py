"""The solve's device-side status on the GPU, with failures made on the host side only.

- A grid-barrier wait cap of one clock cycle (pdf_solve_opts.barrier_wait_cycles) makes the first
  CTA to reach a grid barrier of the one-launch loops give up at once: every wait ends, the kernel
  runs to its end, and pdf_solve returns PDF_ETIMEOUT with or without a report.  The next solve on
  the same handle starts clean.
- Coefficients with a NaN, handed in by the caller as alpha_(0), give PDF_ENONFINITE.
- A cluster launch whose kernel does not find the cluster shape it expects returns at its entry
  check without touching any state (forced through the library's PDF_TEST_CLUSTER_SHAPE hook);
  the solve then runs the same iterations as the CUDA graph and matches a graph solve exactly.
"""
import numpy as np
import pytest

import scenes
from tests.gpu_common import Case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module")
def c1():
    w = scenes.workload("c1", iters=20)
    return Case(w)


@pytest.mark.parametrize("loop,fold", [(3, 1), (2, 0)])
@pytest.mark.parametrize("report", [False, True])
def test_forced_barrier_timeout(c1, loop, fold, report):
    from paper_2602_13805_gb300 import pdf
    prob = c1.problem(fold_gs=fold)
    chi_t = _dev(c1.chi.astype(np.complex64))
    ref = prob.solve(iters=20, chi_true=chi_t, use_graph=loop)
    assert ref["loop_mode"] == loop
    opts = pdf.solve_opts(iters=20, chi_true=chi_t, use_graph=loop, barrier_wait_cycles=1)
    chi = torch.empty((c1.p.ny, c1.p.nx), dtype=torch.complex64, device="cuda")
    with pytest.raises(pdf.PDFError) as e:
        pdf.pdf_solve(prob.h, opts, chi, None, None, report=report)
    assert e.value.status == pdf.PDF_ETIMEOUT
    assert "timed out" in str(e.value)
    # no stale flag: the next solve on this handle runs and reproduces the first one
    again = prob.solve(iters=20, chi_true=chi_t, use_graph=loop)
    assert again["loop_mode"] == loop
    assert torch.equal(again["alpha"], ref["alpha"])
    prob.close()


@pytest.mark.parametrize("loop", [1, 3])
@pytest.mark.parametrize("report", [False, True])
def test_nonfinite_alpha0(c1, loop, report):
    from paper_2602_13805_gb300 import pdf
    prob = c1.problem()
    a = c1.alpha(scale=0.2, seed=3)
    a[1, 2, 3] = np.nan
    opts = pdf.solve_opts(iters=20, init=1, alpha0=_dev(a), use_graph=loop)
    chi = torch.empty((c1.p.ny, c1.p.nx), dtype=torch.complex64, device="cuda")
    with pytest.raises(pdf.PDFError) as e:
        pdf.pdf_solve(prob.h, opts, chi, None, None, report=report)
    assert e.value.status == pdf.PDF_ENONFINITE
    # a finite start afterwards is fine
    ok = prob.solve(iters=20, init=1, alpha0=_dev(c1.alpha(scale=0.2, seed=3)), use_graph=loop)
    assert np.all(np.isfinite(ok["terms"]))
    prob.close()


def test_loss_terms_of_nonfinite_alpha_are_nan(c1):
    prob = c1.problem()
    a = c1.alpha(scale=0.2, seed=3)
    a[0, 0, 0] = np.inf
    terms, _ = prob.loss_grad(_dev(a))
    assert not np.isfinite(terms.cpu().numpy()[0])
    prob.close()


@pytest.mark.parametrize("report", [False, True])
def test_cluster_shape_mismatch_falls_back_to_the_graph(c1, monkeypatch, report):
    from paper_2602_13805_gb300 import pdf
    prob = c1.problem()
    chi_t = _dev(c1.chi.astype(np.complex64))
    graph = prob.solve(iters=20, chi_true=chi_t, use_graph=1)
    monkeypatch.setenv("PDF_TEST_CLUSTER_SHAPE", "mismatch")
    alpha = torch.empty((c1.p.ni, c1.p.ky, c1.p.kx), dtype=torch.complex64, device="cuda")
    opts = pdf.solve_opts(iters=20, chi_true=chi_t, use_graph=3)
    rep = pdf.pdf_solve(prob.h, opts, None, None, alpha, report=report)
    monkeypatch.delenv("PDF_TEST_CLUSTER_SHAPE")
    if report:
        assert rep.loop_mode == 1
    # the fallback ran the graph loop from the same start: identical iterates
    assert torch.equal(alpha, graph["alpha"])
    # and the cluster form runs again once the hook is gone
    assert prob.solve(iters=20, chi_true=chi_t, use_graph=3)["loop_mode"] == 3
    prob.close()
