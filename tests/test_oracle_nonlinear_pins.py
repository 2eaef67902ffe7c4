"""Pins for the oracle's temperature-dependent diffusivity (Section 3.3:
chi_par proportional to T^(5/2), harmonic face average of the two cells'
values, taken from each update's input).  Checked against:
- the linear step, bit for bit, when the exponent is zero;
- the linear step with chi scaled by T0^alpha, to second order in a small
  perturbation of a uniform T0 (a missing factor on either the normal or the
  transverse part of the face flux shows up at first order);
- the steady state of (T^alpha T')' = 0 between fixed ends, whose exact
  solution has T^(alpha+1) linear in x, at second order in the grid spacing;
- conservation, and the harmonic mean's property that a cell at T = 0 passes
  no heat."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _co(bx, by, bc):
    return O.face_coeffs(bx, by, bc)


def test_zero_exponent_is_the_linear_step_bit_for_bit():
    inst = W.random_instance(64, 48, seed=2, dt_factor=100.0)
    co = _co(inst.bx, inst.by, inst.bc)
    lin = O.step(inst.T0, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=3)
    nl = O.step_nl(inst.T0, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, 0.0, nsteps=3)
    assert np.array_equal(lin, nl)


@pytest.mark.parametrize("limiter", [O.LIM_VANLEER, O.LIM_ARITH])
def test_small_perturbation_is_the_scaled_linear_step(limiter):
    # T = T0 (1 + eps g): to first order every face factor is T0^alpha, so the
    # step equals the linear one with chi_par T0^alpha; the difference is
    # O(eps^2), i.e. it falls 100x when eps falls 10x.
    rng = np.random.default_rng(3)
    ny, nx = 24, 32
    b = rng.normal(size=(2, ny, nx))
    b /= np.linalg.norm(b, axis=0)
    co = _co(b[0], b[1], O.BC_PERIODIC)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    g = np.cos(2 * np.pi * (2 * x / nx + y / ny)) + 0.5 * np.sin(2 * np.pi * 3 * y / ny)
    T0, alpha, chi, dt = 2.0, 2.5, 1.0, 5.0
    diffs = []
    for eps in (1e-3, 1e-4):
        T = T0 * (1 + eps * g)
        nl = O.step_nl(T, co, O.BC_PERIODIC, dt, 1.0, 1.0, chi, alpha, t_ref=1.0, limiter=limiter)
        lin = O.step(T, co, O.BC_PERIODIC, dt, 1.0, 1.0, chi * T0 ** alpha, limiter=limiter)
        diffs.append(np.max(np.abs(nl - lin)) / (T0 * eps))
    assert diffs[0] < 0.2            # small against the perturbation itself
    assert 50 < diffs[0] / diffs[1] * 10 < 200 or diffs[1] < 1e-12


def _kirchhoff_error(n, alpha, Ta=1.0, Tb=3.0):
    s = np.arange(n) / (n - 1)
    exact = (Ta ** (alpha + 1) + (Tb ** (alpha + 1) - Ta ** (alpha + 1)) * s) ** (1 / (alpha + 1))
    T = np.tile(Ta + (Tb - Ta) * s, (5, 1))      # interior rows start linear
    T[0], T[-1] = exact, exact                     # fixed edge rows: the exact profile
    bx, by = np.ones_like(T), np.zeros_like(T)     # b along x: rows are independent
    co = _co(bx, by, O.BC_DIRICHLET)
    dx = 1.0 / (n - 1)
    prev = None
    for _ in range(400):
        T = O.step_nl(T, co, O.BC_DIRICHLET, 1e6, dx, dx, 1.0, alpha, t_ref=1.0)
        if prev is not None and np.max(np.abs(T - prev)) < 1e-14:
            break
        prev = T
    assert np.max(np.abs(T - prev)) < 1e-12      # converged to the steady state
    return np.max(np.abs(T[2] - exact))


@pytest.mark.parametrize("alpha", [1.0, 2.5])
def test_steady_state_between_fixed_ends_converges_at_second_order(alpha):
    errs = [_kirchhoff_error(n, alpha) for n in (17, 33, 65)]
    orders = [np.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(1.8 < o < 2.2 for o in orders), (errs, orders)


@pytest.mark.parametrize("bc", [O.BC_ZEROFLUX, O.BC_PERIODIC])
def test_conservation_with_temperature_dependent_chi(bc):
    inst = W.random_instance(40, 56, seed=6, dt_factor=10.0)
    co = _co(inst.bx, inst.by, bc)
    T = O.step_nl(inst.T0, co, bc, inst.dt, inst.dx, inst.dy, inst.chi_par, 2.5, nsteps=4)
    assert abs(T.sum() - inst.T0.sum()) <= 1e-12 * inst.T0.sum()


def test_a_cell_at_zero_passes_no_heat():
    # chi(0) = 0 and the harmonic mean with it is 0, so with b along x the
    # faces of a cold cell carry nothing and it stays at exactly zero.
    ny, nx = 6, 16
    T = np.full((ny, nx), 2.0)
    T[:, 7] = 0.0
    co = _co(np.ones((ny, nx)), np.zeros((ny, nx)), O.BC_PERIODIC)
    out = O.step_nl(T, co, O.BC_PERIODIC, 10.0, 1.0, 1.0, 1.0, 2.5, nsteps=5)
    assert np.all(out[:, 7] == 0.0)
    assert np.allclose(out[:, :7], 2.0) and np.allclose(out[:, 8:], 2.0)
