"""The oracle's pins are sensitive: a plausible mistake planted in the oracle
(on the CPU, by wrapping its Python entry points) makes at least one of the
pin tests fail.

Planted mistakes: the nearest cell instead of the one below, an unwrapped cell
index, an unstable order among equal keys, swapped key axes, offsets off by
one in the split and binning; a transposed node order, a flipped sign, a
dropped term, a mirrored or shifted cell offset in the weights; swapped axes, swapped
components, a one-cell index shift in the triple sum; a wrong step size, a
flipped velocity sign, a reversed Adams-Bashforth history in the steppers; a
missing Jacobian term, transposed axes, a scaled cotangent in the adjoint.
Nothing here runs the library."""
import numpy as np
import pytest

import oracle
import test_golden as G
import test_oracle_adjoint as PA
import test_oracle_interp as PI
import test_oracle_steppers as PS
import test_oracle_weights as PW

L = 2 * np.pi


def fails(pin, *args):
    try:
        pin(*args)
    except AssertionError:
        return True
    return False


def any_pin_fails(pins):
    return sum(fails(pin, *args) for pin, args in pins)


# ---- weights ---------------------------------------------------------------
WEIGHT_MUTATIONS = {
    "transposed node order": lambda w, t, f: w[::-1].copy(),
    "flipped sign of one term": lambda w, t, f: w * np.where(np.arange(len(w)) == 1, -1.0, 1.0),
    "dropped term": lambda w, t, f: np.where(np.arange(len(w)) == 0, 0.0, w),
    "mirrored offset t -> 1 - t": lambda w, t, f: f(1.0 - t),
    "index shifted by one node": lambda w, t, f: np.roll(w, 1),
}


def weight_pins():
    pins = []
    for fam, I, m in [(oracle.LAGRANGE, 4, 0), (oracle.LAGRANGE, 6, 0), (oracle.SPLINE, 4, 1), (oracle.SPLINE, 6, 2)]:
        pins += [(PW.test_partition_of_unity, (fam, I, m)), (PW.test_interpolates_nodes, (fam, I, m)),
                 (PW.test_polynomial_reproduction_degree, (fam, I, m))]
    pins += [(G.test_lagrange_midpoint_weights, (r,)) for r in G.rows("lagrange_midpoint_weights.txt")]
    pins += [(G.test_spline_I4_m1_is_the_cubic_convolution_kernel, (r,)) for r in G.rows("keys_cubic_convolution.txt")]
    return pins


@pytest.mark.parametrize("name", list(WEIGHT_MUTATIONS))
def test_weight_mistakes_are_caught(monkeypatch, name):
    orig = oracle.weights
    mut = WEIGHT_MUTATIONS[name]

    def planted(family, I, m, t, deriv=False):
        if deriv:   # the pins used here read the values only
            return orig(family, I, m, t, deriv)
        return mut(orig(family, I, m, t), t, lambda s: orig(family, I, m, s))

    monkeypatch.setattr(oracle, "weights", planted)
    assert any_pin_fails(weight_pins()) > 0


# ---- split and binning --------------------------------------------------------
def unstable_ties(orig, pos, *a, **k):
    keys, perm, offsets = orig(pos, *a, **k)
    perm = perm.copy()
    for b in range(len(offsets) - 1):          # reverse the order inside every block
        perm[offsets[b]:offsets[b + 1]] = perm[offsets[b]:offsets[b + 1]][::-1]
    return keys, perm, offsets


def offsets_off_by_one(orig, pos, *a, **k):
    keys, perm, offsets = orig(pos, *a, **k)
    offsets = offsets.copy()
    offsets[1:-1] += 1
    return keys, perm, offsets


BIN_MUTATIONS = {
    "unstable order among equal keys": unstable_ties,
    "key axes x1 and x2 swapped": lambda orig, pos, *a, **k: orig(pos[[1, 0, 2]], *a, **k),
    "offsets off by one": offsets_off_by_one,
}


def round_to_nearest_cell(orig, pos, N, *a, **k):
    c, t = orig(pos, N, *a, **k)
    up = t >= 0.5
    return np.where(up, (c + 1) % N, c).astype(c.dtype), np.where(up, t - 1.0, t)


def no_periodic_wrap(orig, pos, N, *a, **k):
    c, t = orig(pos, N, *a, **k)
    L_ = k.get("L", L)
    return (c + N * np.floor(pos / L_).astype(c.dtype)), t


SPLIT_MUTATIONS = {
    "nearest cell instead of the cell below": round_to_nearest_cell,
    "cell index not wrapped": no_periodic_wrap,
}


def bin_pins():
    return [(PI.test_split_geometry_and_ranges, ()), (PI.test_binning_slices_like_the_paper, ())] + [
        (PI.test_binning_is_stable_sort_by_block, (B,)) for B in [(2, 2, 2), (4, 2, 8)]]


@pytest.mark.parametrize("name", list(BIN_MUTATIONS))
def test_binning_mistakes_are_caught(monkeypatch, name):
    orig = oracle.bin_particles
    mut = BIN_MUTATIONS[name]
    monkeypatch.setattr(oracle, "bin_particles", lambda pos, *a, **k: mut(orig, pos, *a, **k))
    assert any_pin_fails(bin_pins()) > 0


@pytest.mark.parametrize("name", list(SPLIT_MUTATIONS))
def test_split_mistakes_are_caught(monkeypatch, name):
    orig = oracle.split
    mut = SPLIT_MUTATIONS[name]
    monkeypatch.setattr(oracle, "split", lambda pos, N, *a, **k: mut(orig, pos, N, *a, **k))
    assert any_pin_fails(bin_pins()) > 0


# ---- triple sum --------------------------------------------------------------
def shift_one_cell(orig, field, pos, *a, **k):
    N = field.shape[-1]
    return orig(field, pos + L / N, *a, **k)


INTERP_MUTATIONS = {
    "axes x1 and x2 swapped": lambda orig, field, pos, *a, **k: orig(field, pos[[1, 0, 2]], *a, **k),
    "components swapped": lambda orig, field, pos, *a, **k: orig(field, pos, *a, **k)[[1, 0, 2] if field.shape[0] == 3
                                                                                       else slice(None)],
    "one-cell index shift": shift_one_cell,
}


def interp_pins():
    pins = []
    for fam, I, m in [(oracle.LAGRANGE, 4, 0), (oracle.SPLINE, 6, 2)]:
        pins += [(PI.test_constant_field, (fam, I, m)), (PI.test_polynomial_field_reproduced_on_local_window, (fam, I, m))]
    pins += [(PI.test_lagrange_separable_field_vs_scipy, (4,))]
    return pins


@pytest.mark.parametrize("name", list(INTERP_MUTATIONS))
def test_interpolation_mistakes_are_caught(monkeypatch, name):
    orig = oracle.interp
    mut = INTERP_MUTATIONS[name]
    monkeypatch.setattr(oracle, "interp", lambda field, pos, *a, **k: mut(orig, field, pos, *a, **k))
    assert any_pin_fails(interp_pins()) > 0


# ---- time steppers -------------------------------------------------------------
def reversed_history(orig, field, pos, dt, steps, *a, **k):
    rhs = k.get("rhs")
    if rhs is not None and np.asarray(rhs).shape[0] > 1:
        k = dict(k, rhs=np.asarray(rhs)[::-1].copy())
    return orig(field, pos, dt, steps, *a, **k)


STEP_MUTATIONS = {
    "step size off by 0.1%": lambda orig, field, pos, dt, steps, *a, **k: orig(field, pos, dt * 1.001, steps, *a, **k),
    "velocity sign flipped": lambda orig, field, pos, dt, steps, *a, **k: orig(-field, pos, dt, steps, *a, **k),
    "history entries reversed": reversed_history,
}


def step_pins():
    pins = [(PS.test_uniform_flow_is_exact, (oracle.RK2,)), (PS.test_uniform_flow_is_exact, (oracle.AB2,)),
            (PS.test_rk2_rotation_closed_form, (oracle.SPLINE, 6, 2)), (PS.test_ab2_rotation_recurrence, ())]
    pins += [(PS.test_ab_weights_match_their_definition, (s, k)) for s, k in [(oracle.AB3, 3), (oracle.AB4, 4)]]
    pins += [(G.test_adams_bashforth_coefficients, (r,)) for r in G.rows("adams_bashforth_coefficients.txt")]
    return pins


@pytest.mark.parametrize("name", list(STEP_MUTATIONS))
def test_stepper_mistakes_are_caught(monkeypatch, name):
    orig = oracle.advance
    mut = STEP_MUTATIONS[name]
    monkeypatch.setattr(oracle, "advance", lambda field, pos, dt, steps, *a, **k: mut(orig, field, pos, dt, steps, *a, **k))
    assert any_pin_fails(step_pins()) > 0


# ---- adjoint ----------------------------------------------------------------------
def adjoint_transposed_axes(orig, field, pos0, lam, *a, **k):
    gpos, gf = orig(field, pos0, lam, *a, **k)
    return gpos, (gf.transpose(0, 1, 3, 2).copy() if gf is not None else gf)


ADJOINT_MUTATIONS = {
    "position gradient missing the J^T term": lambda orig, field, pos0, lam, *a, **k:
        (lam.copy(), orig(field, pos0, lam, *a, **k)[1]),
    "field gradient with x1, x2 transposed": adjoint_transposed_axes,
    "lambda scaled by 1.001": lambda orig, field, pos0, lam, *a, **k: orig(field, pos0, lam * 1.001, *a, **k),
}


def adjoint_pins():
    return [(PA.test_position_gradient_matches_central_differences, ()),
            (PA.test_field_gradient_matches_central_differences, ()),
            (PA.test_interpolation_transpose_identity, ())]


@pytest.mark.parametrize("name", list(ADJOINT_MUTATIONS))
def test_adjoint_mistakes_are_caught(monkeypatch, name):
    orig = oracle.adjoint_rk2
    mut = ADJOINT_MUTATIONS[name]
    monkeypatch.setattr(oracle, "adjoint_rk2", lambda field, pos0, lam, *a, **k: mut(orig, field, pos0, lam, *a, **k))
    assert any_pin_fails(adjoint_pins()) > 0


def test_unmutated_oracle_passes_every_pin_used_here():
    for pin, args in weight_pins() + bin_pins() + interp_pins() + step_pins() + adjoint_pins():
        pin(*args)
