"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins
in test_oracle_pins.py catch each one."""
import cmath
import math

import pytest

import test_oracle_pins as pins
from oracle import basis, brute, proa, substate


def _fails(fn, *args):
    try:
        fn(*args)
    except (AssertionError, basis.PatternError, ValueError):
        return True
    return False


def test_eq1_literal_sign_is_caught(monkeypatch):
    """Taking Eq. 1 literally (e^{-ia} in |+-a>) conjugates the phase."""
    orig = basis.resolved_phase
    monkeypatch.setattr(substate, "resolved_phase", lambda a, s, t: orig(a, s, t).conjugate())
    assert _fails(pins.test_j_alpha_closed_form, 0.7)


def test_dropped_t_signal_is_caught(monkeypatch):
    orig = basis.resolved_phase
    monkeypatch.setattr(substate, "resolved_phase", lambda a, s, t: orig(a, s, 0))
    assert _fails(pins.test_textbook_reduction_jcz_circuits)


def test_dropped_s_signal_is_caught(monkeypatch):
    orig = basis.resolved_phase
    monkeypatch.setattr(substate, "resolved_phase", lambda a, s, t: orig(a, 0, t))
    assert _fails(pins.test_textbook_reduction_jcz_circuits)


def test_swapped_outcome_rows_are_caught(monkeypatch):
    """Outcome 0 taking the minus row of Eq. 12 instead of Eq. 11."""
    orig = basis.resolved_phase
    monkeypatch.setattr(substate, "resolved_phase", lambda a, s, t: -orig(a, s, t))
    assert _fails(pins.test_figure8_cnot_trace)


def test_missing_sqrt2_is_caught(monkeypatch):
    monkeypatch.setattr(substate, "SQRT2", 1.0)
    assert _fails(pins.test_measurement_compaction_eq21)


def test_brute_force_wrong_projector_is_caught(monkeypatch):
    orig = basis.ket_pm
    monkeypatch.setattr(brute, "ket_pm", lambda a, s: orig(-a, s))
    assert _fails(pins.test_bruteforce_agrees_with_substate)


def test_proa_flag_inverted_is_caught(monkeypatch):
    orig = proa.greedy

    def bad(pattern, a, b, g, d, eowqs=False, product_input=False, stages=None):
        # swapping the two branches of Eq. 18 by exchanging a*MS with a*(MS+1)*d
        return orig(pattern, a * d, b, g, 1.0 / d, eowqs, product_input, stages)

    monkeypatch.setattr(proa, "greedy", bad)
    assert _fails(pins.test_table1_proa_trace)


def test_eowqs_sampling_against_computed_probability_is_caught(monkeypatch):
    """EOWQS drawing a sampled outcome against the computed probability
    instead of the 1/2 of Section 4.5."""
    orig = substate.outcome_probabilities
    monkeypatch.setattr(substate, "outcome_probabilities", lambda mode, t, half: orig("owqs", t, half))
    assert _fails(pins.test_eowqs_sampled_draws_fair_coins)
