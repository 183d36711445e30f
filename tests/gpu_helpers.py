"""Shared helpers of the GPU parity tests: tolerance checks against the oracle."""
import numpy as np

# Objective: 1e-12 relative.  Gradient: 1e-10 relative per component, plus a round-off floor
# of 1e-13 of the largest component (a component that cancels to far below the others carries
# the absolute rounding error of its O(1e3..1e5)-term sum; see the design notes).
OBJ_RTOL = 1e-12
GRAD_RTOL = 1e-10
GRAD_FLOOR = 1e-13


def assert_objective_close(got, want, rtol=OBJ_RTOL):
    assert abs(got - want) <= rtol * abs(want), (got, want, abs(got - want) / abs(want))


def grad_mismatch(got, want, rtol=GRAD_RTOL, floor=GRAD_FLOOR):
    got, want = np.asarray(got), np.asarray(want)
    scale = np.max(np.abs(want)) if want.size else 0.0
    tol = rtol * np.abs(want) + floor * scale
    bad = np.abs(got - want) > tol
    worst = float(np.max(np.abs(got - want) / np.maximum(np.abs(want), 1e-300))) if want.size else 0.0
    return int(bad.sum()), worst


def assert_grad_close(got, want, rtol=GRAD_RTOL, floor=GRAD_FLOOR, what="gradient"):
    nbad, worst = grad_mismatch(got, want, rtol, floor)
    assert nbad == 0, f"{what}: {nbad} components outside tolerance (worst rel {worst:.3e})"
