"""Failure paths of the solvers, driven from the host: no GPU fault, trap or hang is used.

A right-hand side poisoned with NaN, an iteration cap below what the tolerance needs, and a tolerance below
the FP64 rounding floor (so that a restart cycle stops reducing the residual) each return their status
(FDA_E_NAN, FDA_E_NOT_CONVERGED, FDA_E_BREAKDOWN) with a message in fda_last_error, and the context and the
plan stay usable: a clean solve right after each one converges.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1311_5202_gb300 import fdbem, inputs  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def c1():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mesh = inputs.icosphere(4, 0.5)
    S = fdbem.Solver(mesh.nodes, mesh.elems, 10.0, eps=1e-6, leaf_max=64, precision=fdbem.FDA_PREC_FP32,
                     nrhs_max=2)
    b = torch.empty((2, S.N), dtype=torch.complex128, device=DEV)
    fdbem.bm_rhs_plane_wave(S.prob, np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]]), b)
    yield S, b
    S.close()


def _clean_solve_still_works(S, b):
    x = torch.zeros_like(b[0])
    st = S.solve(b[0].contiguous(), x, tol=1e-6, restart=50, max_iter=300)
    assert st["status"] == fdbem.FDA_OK and st["rel_residual"] <= 1e-6
    assert fdbem.fda_plan_check(S.plan) == fdbem.FDA_OK


@pytest.mark.parametrize("mode", ["fp64", "refine", "block", "block_refine"])
def test_nan_right_hand_side_returns_nan_status(c1, mode):
    S, b = c1
    bb = b.clone() if mode.startswith("block") else b[0].clone()
    flat = bb.view(-1)
    flat[S.N + 17 if mode.startswith("block") else 17] = complex(float("nan"), 0.0)
    x = torch.zeros_like(bb)
    st = S.solve(bb, x, tol=1e-6, restart=30, max_iter=100, refine=mode.endswith("refine"), inner_tol=1e-3,
                 raise_on_error=False)
    assert st["status"] == fdbem.FDA_E_NAN, st
    msg = fdbem.fda_last_error()
    assert "NaN" in msg, msg
    _clean_solve_still_works(S, b)


@pytest.mark.parametrize("mode", ["fp64", "refine", "block"])
def test_iteration_cap_returns_not_converged(c1, mode):
    S, b = c1
    bb = b.clone() if mode == "block" else b[0].clone()
    x = torch.zeros_like(bb)
    st = S.solve(bb, x, tol=1e-12, restart=30, max_iter=5, refine=mode == "refine", inner_tol=1e-3,
                 raise_on_error=False)
    assert st["status"] == fdbem.FDA_E_NOT_CONVERGED, st
    assert "reached" in fdbem.fda_last_error()
    assert st["iterations"] <= 5
    # the partial solution is finite and better than x = 0
    assert torch.isfinite(torch.view_as_real(x)).all()
    assert 0 < st["rel_residual"] < 1.0
    _clean_solve_still_works(S, b)


def test_tolerance_below_rounding_returns_breakdown(c1):
    """GMRES(10) in FP64 with tol = 1e-20: once the residual sits on the rounding floor a restart cycle no
    longer reduces it, and the solver reports the stagnation instead of running to the iteration cap."""
    S, b = c1
    x = torch.zeros_like(b[0])
    st = S.solve(b[0].contiguous(), x, tol=1e-20, restart=10, max_iter=5000, raise_on_error=False)
    assert st["status"] == fdbem.FDA_E_BREAKDOWN, st
    assert "stagnated" in fdbem.fda_last_error()
    assert st["rel_residual"] < 1e-11 and st["iterations"] < 5000
    _clean_solve_still_works(S, b)
