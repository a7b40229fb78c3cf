"""C-ABI library on the CPU: it loads, exports every declared symbol, and its
host logic (validation D0-D3, PROA, schedule compiler, index maps) agrees
with the oracle.  No kernel is launched here."""
import math
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import basis, counting, proa, substate
from owqs_inputs import workloads
from owqs_inputs.patterns import E, M, N, Pattern, X, Z, circuit_to_pattern, random_jcz_circuit
from owqs_inputs.rng import SplitMix64, random_state

import pass_emulator
from helpers import outcomes_by_label
from test_oracle_pins import _wild_patterns, cnot_eq22, swap_graph_pattern

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def owqs():
    from paper_1604_05659_gb300 import build, owqs as mod
    build.ensure_built()
    mod.library()
    return mod


def test_exports_every_declared_symbol(owqs):
    header = open(os.path.join(ROOT, "include", "owqs.h")).read()
    declared = set(re.findall(r"\b(owqs_[a-z_]+)\s*\(", header))
    assert "owqs_run" in declared and "owqs_reorder" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", owqs.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (owqs_[a-z_]+)\b", out))
    assert declared <= exported, declared - exported
    lib = owqs.library()
    assert lib.owqs_abi_version() == 2


def test_binding_constants_match_the_header(owqs):
    """Every enum value the binding passes or decodes is the header's: status
    codes, command kinds, modes, dtypes, outcome policies, run flags, flow
    kinds, and the kernel kinds owqs_profile_run documents."""
    header = open(os.path.join(ROOT, "include", "owqs.h")).read()
    enum = {k: int(v) for k, v in re.findall(r"\b(OWQS_[A-Z0-9_]+)\s*=\s*(\d+)", header)}
    assert [enum["OWQS_" + n] for n in owqs.STATUS_NAMES] == list(range(len(owqs.STATUS_NAMES)))
    assert enum["OWQS_ERR_UNSUPPORTED"] == owqs.ERR_UNSUPPORTED and enum["OWQS_ERR_CUDA"] == owqs.ERR_CUDA
    assert {k: enum["OWQS_CMD_" + k] for k in owqs.CMD_KIND} == owqs.CMD_KIND
    assert {k: enum["OWQS_MODE_" + k.upper()] for k in owqs.MODE} == owqs.MODE
    assert {k: enum["OWQS_" + k.upper()] for k in owqs.DTYPE} == owqs.DTYPE
    assert {k: enum["OWQS_OUTCOME_" + k.upper()] for k in owqs.POLICY} == owqs.POLICY
    for flag in ("HOST_SAMPLING", "PER_PASS", "SEQUENTIAL_SAMPLING"):
        assert enum["OWQS_RUN_" + flag] == getattr(owqs, "RUN_" + flag)
    assert (enum["OWQS_FLOW_CAUSAL"], enum["OWQS_FLOW_GFLOW"]) == (owqs.FLOW_CAUSAL, owqs.FLOW_GFLOW)
    doc = header[header.index("kind[i] its"):header.index("owqs_status owqs_profile_run")]
    documented = {int(k) for k in re.findall(r"\b(\d+) [a-z]", doc.replace("\n *", " ")) if int(k) < 32}
    assert documented == set(owqs.KERNEL_KIND), (documented, set(owqs.KERNEL_KIND))


def test_validation_errors(owqs):
    bad = {
        "D0": Pattern(3, [0], [2], [E(0, 1), E(1, 2), M(0, 0.0, [1]), M(1, 0.0)]),
        "D1": Pattern(2, [0], [1], [E(0, 1), M(0, 0.0), Z(0)]),
        "D2": Pattern(2, [0], [1], [E(0, 1), N(1), M(0, 0.0)]),
        "D3": Pattern(2, [0], [1], [E(0, 1), M(0, 0.0), M(1, 0.0)]),
        "EUU": Pattern(2, [0], [1], [E(1, 1), M(0, 0.0)]),
    }
    for name, p in bad.items():
        with pytest.raises(owqs.OwqsError) as ei:
            owqs.load(p)
        assert ei.value.status == owqs.ERR_PATTERN, name
    with pytest.raises(owqs.OwqsError) as ei:
        owqs.load(Pattern(2, [5], [1], [E(0, 1), M(0, 0.0)]))
    assert ei.value.status == owqs.ERR_ARG
    h = owqs.load(cnot_eq22())
    assert h.info()["nmeas"] == 2 and h.info()["standard"] == 1
    # not standard form -> reorder refuses
    wild = _wild_patterns()[0]
    hw = owqs.load(wild)
    if not wild.is_standard():
        with pytest.raises(owqs.OwqsError) as ei:
            hw.reorder()
        assert ei.value.status == owqs.ERR_NOT_STANDARD


def _cases():
    cases = [("cnot", cnot_eq22(), False), ("small", workloads.small_random().pattern, False),
             ("brick6x10", workloads.brickwork(6, 10).pattern, False),
             ("qft5", workloads.qft(5, with_input=False).pattern, False)]
    for wl in workloads.random_batch(count=6, wmin=3, wmax=8, dmin=3, dmax=9):
        cases.append((wl.name, wl.pattern, False))
    _, sw = swap_graph_pattern()
    cases.append(("swap", sw, True))
    return cases


@pytest.mark.parametrize("eowqs", [False, True])
def test_reorder_matches_oracle_proa(owqs, eowqs):
    """C++ PROA gives the oracle's order bit for bit, with the same peak m,
    live width and amplitude-update count."""
    for name, p, product in _cases():
        h = owqs.load(p)
        order, info = h.reorder(mode="eowqs" if eowqs else "owqs", product_input=product)
        o_order, o_ms, o_a = proa.proa(p, eowqs=eowqs, product_input=product)
        assert order == o_order, name
        assert info["peak_m"] == max(o_ms), name
        assert info["alpha_used"] == o_a, name
        rp = proa.reorder_commands(p, o_order)
        assert info["peak_live"] == proa.single_array_peak(rp), name
        assert info["amp_updates"] == counting.amplitude_updates(rp), name
        assert h.order() == o_order


def test_reorder_full_size_brickwork_and_qft(owqs):
    for wl, peak in [(workloads.brickwork(28, 40), 29), (workloads.qft(24, with_input=False), 25)]:
        h = owqs.load(wl.pattern)
        order, info = h.reorder()
        o_order, o_ms, _ = proa.proa(wl.pattern)
        assert order == o_order
        assert info["peak_m"] == max(o_ms) == peak
        assert info["peak_live"] == peak


def test_table1_through_abi(owqs):
    g, p = swap_graph_pattern()
    h = owqs.load(p)
    order, info = h.reorder(mode="eowqs", product_input=True, sweep=False, weights=(2, 2, 0.5, 2))
    assert [v + 1 for v in order] == [s["measure"] for s in g["stages"]]
    assert info["peak_m"] == 3


def _model_index_maps(p):
    """Independent model of the bit convention: inputs at bits 0..|I|-1; a
    qubit is appended as the new top bit when first touched; eliminating a
    qubit shifts the bits above it down."""
    live = list(p.inputs)
    maps = []

    def snap():
        m = [-1] * p.nqubits
        for i, q in enumerate(live):
            m[q] = i
        maps.append(m)

    snap()
    for c in p.cmds:
        if c.kind == "N":
            continue
        for q in [c.q0] + ([c.q1] if c.kind == "E" else []):
            if q not in live:
                live.append(q)
        if c.kind == "M":
            live.remove(c.q0)
            snap()
    return maps


def test_index_maps_bit_exact(owqs):
    for name, p, product in _cases():
        h = owqs.load(p)
        order, _ = h.reorder(product_input=product)
        rp = proa.reorder_commands(p, order)
        want = _model_index_maps(rp)
        for i, m in enumerate(want):
            assert h.index_map(i) == m, (name, i)


def _check_emulated(owqs, p, psi, bits, mode, reorder=True, atol=1e-12):
    h = owqs.load(p)
    if reorder:
        order, _ = h.reorder(mode="owqs")
        op = proa.reorder_commands(p, order)
    else:
        op = p
    descs = h.describe_passes(bits, mode=mode)
    out, probs = pass_emulator.emulate(descs, psi, mode=mode)
    r = substate.run(op, psi, outcomes=outcomes_by_label(p, bits), mode=mode)
    assert np.allclose(out, r.psi_out, atol=atol, rtol=0)
    if mode == "owqs":
        o_probs = [r.probs[q] for q in op.measured()]
        assert np.allclose(probs, o_probs, atol=atol, rtol=0)
    return descs


@pytest.mark.parametrize("mode", ["owqs", "eowqs"])
def test_schedule_compiler_against_oracle(owqs, mode):
    """The host schedule compiler's passes, run through the CPU model of the
    kernel contract, reproduce the oracle exactly (no phase freedom)."""
    rng = SplitMix64(77)
    for name, p, _ in _cases()[:-1]:
        psi = random_state(rng, len(p.inputs))
        bits = rng.bits(p.K)
        _check_emulated(owqs, p, psi, bits, mode)
        _check_emulated(owqs, p, None, bits, mode)


def test_schedule_compiler_wild_patterns(owqs):
    """Non-standard patterns with X and Z between measurements and all E
    commands up front (pattern order, no reordering)."""
    rng = SplitMix64(78)
    for p in _wild_patterns():
        psi = random_state(rng, len(p.inputs))
        for _ in range(3):
            bits = rng.bits(p.K)
            for mode in ("owqs", "eowqs"):
                _check_emulated(owqs, p, psi, bits, mode, reorder=False)
