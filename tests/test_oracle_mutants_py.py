"""The pins of the oracle's NumPy functions have teeth: plausible mistakes planted in them (on
the CPU, by replacing the function for the duration of the check) must each fail at least one
of the pins in test_oracle.py."""
import numpy as np
import pytest

import oracle
import test_oracle as pins


def _norm_abs_not_squared(c, w):
    c = np.asarray(c, dtype=np.complex128)
    return float(np.sum(np.asarray(w) * np.abs(c)))


def _norm_real_part_only(c, w):
    c = np.asarray(c, dtype=np.complex128)
    return float(np.sum(np.asarray(w) * c.real * c.real))


def _grad_without_two(c, w, g=1.0):
    return (g * np.asarray(w, dtype=np.float64)) * np.asarray(c, dtype=np.complex128)


def _grad_conjugated(c, w, g=1.0):
    return (2.0 * g * np.asarray(w, dtype=np.float64)) * np.conj(np.asarray(c, dtype=np.complex128))


def _real_parity_swapped(G_real, idx):
    G = np.asarray(G_real, dtype=np.float64)
    N = G.shape[0].bit_length() - 1
    c = oracle.decompose_at(G.astype(np.complex128), idx)
    k = oracle.y_count(idx, N)
    return np.where(k % 2 == 0, (c * -1j).real, c.real)


def _real_sign_flipped(G_real, idx):
    G = np.asarray(G_real, dtype=np.float64)
    N = G.shape[0].bit_length() - 1
    c = oracle.decompose_at(G.astype(np.complex128), idx)
    k = oracle.y_count(idx, N)
    return np.where(k % 2 == 1, (c * 1j).real, c.real)


NORM_PINS = [lambda: pins.test_weighted_norm_unit_weights_is_parseval(3), pins.test_weighted_norm_one_hot_and_batch,
             pins.test_weighted_norm_grad_by_finite_differences]
GRAD_PINS = [pins.test_weighted_norm_grad_by_finite_differences, pins.test_gradient_of_weighted_norm_by_finite_differences]
REAL_PINS = [pins.test_real_matrix_coefficients]

MUTANTS = {
    "norm_abs_not_squared": ("weighted_norm", _norm_abs_not_squared, NORM_PINS),
    "norm_real_part_only": ("weighted_norm", _norm_real_part_only, NORM_PINS),
    "grad_without_two": ("weighted_norm_grad", _grad_without_two, GRAD_PINS),
    "grad_conjugated": ("weighted_norm_grad", _grad_conjugated, GRAD_PINS),
    "real_parity_swapped": ("real_coefficients_at", _real_parity_swapped, REAL_PINS),
    "real_sign_flipped": ("real_coefficients_at", _real_sign_flipped, REAL_PINS),
}


def _some_pin_fails(checks):
    for check in checks:
        try:
            check()
        except AssertionError:
            return True
    return False


def test_pins_pass_on_the_real_functions():
    assert not _some_pin_fails(NORM_PINS + REAL_PINS)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, monkeypatch):
    attr, fn, checks = MUTANTS[name]
    monkeypatch.setattr(oracle, attr, fn)
    assert _some_pin_fails(checks), f"mutant {name} passed every pin"
