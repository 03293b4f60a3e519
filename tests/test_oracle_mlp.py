"""The pins of tests/mlp_pins.py on the FP64 reference of the learned seed
(oracle/mlp.py), and on copies of it with one planted mistake each, every one
of which some pin must catch."""
import importlib.util
import os
import types

import pytest

torch = pytest.importorskip("torch")

import mlp_pins  # noqa: E402
from oracle import mlp as om  # noqa: E402

MUTANTS = {
    "bf16_truncates": ("r = ((u + 0x7FFF + lsb) & 0xFFFF0000)", "r = (u & 0xFFFF0000)"),
    "input_lo_half_dropped": ("    return hi + lo\n", "    return hi\n"),
    "relu_mask_dropped_in_backward": ('dz2 = np.outer(dy, c["W3r"]) * (c["z2"] > 0)',
                                      'dz2 = np.outer(dy, c["W3r"])'),
    "dW2_transposed": ('dW2 = dz2r.T @ c["a1"]', 'dW2 = c["a1"].T @ dz2r'),
    "db1_from_unmasked_signal": ("db1 = dz1.sum(axis=0)", "db1 = da1.sum(axis=0)"),
    "adam_without_bias_correction": ("mhat = m / (1.0 - beta1 ** t)", "mhat = m"),
    "sin_psi_sign": ("np.cos(psi), np.sin(psi)", "np.cos(psi), -np.sin(psi)"),
    "target_without_half": ("g = (np.asarray(h, np.float64) - hl) / (0.5 * k * hl * hl)",
                            "g = (np.asarray(h, np.float64) - hl) / (k * hl * hl)"),
}


def _mutant(name):
    old, new = MUTANTS[name]
    src = open(om.__file__).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mod = types.ModuleType(f"mlp_mutant_{name}")
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("pin", mlp_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin_holds(pin):
    pin(om)


@pytest.mark.parametrize("name", list(MUTANTS))
def test_mutant_is_caught(name):
    m = _mutant(name)
    caught = []
    for pin in mlp_pins.ALL_PINS:
        try:
            pin(m)
        except Exception:
            caught.append(pin.__name__)
    assert caught, f"no pin catches the planted mistake {name}"
