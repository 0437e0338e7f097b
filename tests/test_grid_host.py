"""Host logic of the torch layer (no GPU): StencilFn refuses a backward whose
forward record was overwritten, and VarCoefProblem's record bookkeeping."""
import types

import pytest
import torch

from paper_2512_19851_gb300.grid import StencilFn, VarCoefProblem


def fake_problem(coeff_generation=0):
    p = object.__new__(VarCoefProblem)
    p.grid = types.SimpleNamespace(coeff_generation=coeff_generation)
    p.generation = 0
    p.recorded = None
    return p


def test_record_follows_forward_runs_and_coefficients():
    p = fake_problem()
    assert not p.record_valid(None)
    # what forward() does after enqueueing the checkpointed run
    p.generation += 1
    p.recorded = (p.generation, p.grid.coeff_generation)
    first = p.recorded
    assert p.record_valid(first)
    p.generation += 1
    p.recorded = (p.generation, p.grid.coeff_generation)
    assert not p.record_valid(first) and p.record_valid(p.recorded)
    p.grid.coeff_generation += 1  # set_coeff after the run
    assert not p.record_valid(p.recorded)


def test_backward_of_an_overwritten_record_raises_before_any_library_call():
    p = fake_problem()
    p.generation, p.recorded = 2, (2, 0)

    def no_call(**kw):  # pragma: no cover - must not be reached
        raise AssertionError("backward_from called on a stale record")

    p.backward_from = no_call
    ctx = types.SimpleNamespace(problem=p, record=(1, 0), u0_dtype=torch.float64, kappa_dtype=torch.float64)
    with pytest.raises(RuntimeError, match="overwritten"):
        StencilFn.backward(ctx, torch.zeros(2))
