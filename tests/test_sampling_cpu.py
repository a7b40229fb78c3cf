"""The checked guess of sampled OWQS runs, on the CPU model of the pass
contract (no GPU).

A sampled OWQS run first takes outcome k = (u_k > 1/2), u_k the k-th
splitmix64 uniform in execution order, runs those outcomes as forced ones,
and keeps that run iff every draw u_k <= prob_0 against the probabilities it
computed gives back its guess; otherwise it draws one measurement at a time.
Here the forced run is the host schedule compiler's passes run through the
pass-contract model, and the one-at-a-time draw is the oracle's.  When the
check holds the guesses are the oracle's outcomes (by induction over k); when
it fails they are not, so falling back is needed.  Both cases occur: flow
patterns (every probability 1/2, Section 4.5) keep the guess, patterns that
measure an unentangled input with prob_0 != 1/2 fail it for some seeds."""
import numpy as np
import pytest

from oracle import substate
from owqs_inputs.patterns import E, M, N, Pattern, circuit_to_pattern, random_jcz_circuit
from owqs_inputs.rng import SplitMix64, random_state

import pass_emulator


@pytest.fixture(scope="module")
def owqs():
    from paper_1604_05659_gb300 import build, owqs as mod
    build.ensure_built()
    mod.library()
    return mod


def _patterns():
    rng = SplitMix64(4100)
    pats = [circuit_to_pattern(n, random_jcz_circuit(n, 4, rng, cz_per_layer=1), f"flow{n}") for n in (2, 3, 4)]
    # qubit 0: an input measured without entanglement (prob_0 = |<+_a|psi_0>|^2);
    # qubit 1: entangled with the output, its angle depending on qubit 0
    pats.append(Pattern(3, [0, 1], [2], [N(2), E(1, 2), M(0, 0.3), M(1, 0.7, sdom=(0,))], "input_measured"))
    pats.append(Pattern(2, [0], [1], [N(1), M(0, 1.2)], "lone_input"))
    return pats


def test_checked_guess_reproduces_the_one_at_a_time_draw(owqs):
    kept_n = failed_n = 0
    for p in _patterns():
        h = owqs.load(p)
        order = h.order()                       # execution order (labels)
        load = p.measured()                     # outcome buffer order (labels)
        rng = SplitMix64(4200 + p.nqubits)
        psi = random_state(rng, len(p.inputs))
        if p.name == "lone_input":
            psi = np.array([0.8, 0.6j])
        for seed in range(30):
            stream = SplitMix64(seed)
            u = {q: stream.uniform() for q in order}
            guess = {q: 0 if u[q] <= 0.5 else 1 for q in order}
            descs = h.describe_passes([guess[q] for q in load])
            _, probs = pass_emulator.emulate(descs, psi)
            pk = dict(zip(order, probs))        # probability of each guessed outcome
            kept = all((0 if u[q] <= (pk[q] if guess[q] == 0 else 1.0 - pk[q]) else 1) == guess[q] for q in order)
            ref = substate.run(p, psi, policy="sampled", seed=seed)
            if kept:
                kept_n += 1
                assert all(ref.outcomes[q] == guess[q] for q in order), (p.name, seed)
                assert all(abs(ref.probs[q] - pk[q]) < 1e-12 for q in order), (p.name, seed)
            else:
                failed_n += 1
                assert any(ref.outcomes[q] != guess[q] for q in order), (p.name, seed)
        if p.name.startswith("flow"):
            assert all(abs(v - 0.5) < 1e-12 for v in probs)
    assert kept_n >= 60 and failed_n >= 5, (kept_n, failed_n)


def test_checked_launches_reproduce_the_one_at_a_time_draw(owqs):
    """Checked launches (patterns without a gflow): run the forced schedule
    of the current outcome vector, take the measurements in execution order,
    and at the first draw u_k <= prob_0 that decides the other outcome
    correct it and run again from that measurement (its input is the same,
    since every earlier outcome is unchanged).  The outcomes end equal to the
    oracle's one-at-a-time draw, and the corrections are exactly the
    measurements whose drawn outcome differs from its guess u_k > 1/2, each
    corrected once."""
    from owqs_inputs import workloads
    pats = [(w.pattern, w.psi_in) for w in (workloads.measured_inputs(6), workloads.brickwork_readout(3, 4, kept=1,
                                                                                                  with_input=True))]
    pats += [(p, None) for p in _patterns()[-2:]]
    corrected_total = 0
    for p, psi in pats:
        h = owqs.load(p)
        if p.is_standard():
            h.reorder()
        order = h.order()
        load = p.measured()
        if psi is None:
            psi = random_state(SplitMix64(4300 + p.nqubits), len(p.inputs))
        op_cmds = p
        if p.is_standard():
            from oracle import proa
            op_cmds = proa.reorder_commands(p, order)
        for seed in range(12):
            stream = SplitMix64(seed)
            u = {q: stream.uniform() for q in order}
            oc = {q: 0 if u[q] <= 0.5 else 1 for q in order}
            guess = dict(oc)
            decided = set()
            corrections = 0
            while True:
                _, probs = pass_emulator.emulate(h.describe_passes([oc[q] for q in load]), psi)
                bad = None
                for q, pv in zip(order, probs):
                    if q in decided:
                        continue
                    decided.add(q)
                    p0 = pv if oc[q] == 0 else 1.0 - pv
                    drawn = 0 if u[q] <= p0 else 1
                    if drawn != oc[q]:
                        bad = q
                        oc[q] = drawn
                        break
                if bad is None:
                    break
                corrections += 1
            ref = substate.run(op_cmds, psi, policy="sampled", seed=seed)
            assert all(ref.outcomes[q] == oc[q] for q in order), (p.name, seed)
            assert corrections == sum(ref.outcomes[q] != guess[q] for q in order), (p.name, seed)
            corrected_total += corrections
    assert corrected_total >= 10
