"""The bounds-checked debug build (libowqs_checked.so, kernels compiled with
OWQS_BOUNDS_CHECK): every global access of the pass kernels is first checked
against the extent of the buffer it touches.

- Runs that take every launch kind (pass groups from a materialised and from
  the virtual input, exact-half and norm-summing groups, complex128 groups in
  FP64 and in double-float, bulk-copy and register-tiled single passes,
  generic and final passes, the input norm, factor joins and separate
  sub-states, unitaries, sampled outcomes by a whole-run guess, by checked
  launches and one measurement at a time on the device, EOWQS, asynchronous
  runs, the allocation-free entry point) finish with no failed check and
  give the release library's results.
- With every extent shortened through the test hook, the checked build
  reports the accesses beyond them (skipping them, so nothing outside a
  buffer is touched) and the run fails with OWQS_ERR_CUDA.

The checked library runs in a child process (one library per process)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
from paper_1604_05659_gb300 import owqs
from owqs_inputs import workloads
from owqs_inputs.patterns import circuit_to_pattern, random_jcz_circuit
from owqs_inputs.rng import SplitMix64, random_state


def run_cases(out_path):
    res = {{}}
    for dtype in ("c64", "c128"):
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        dev = lambda v: torch.from_numpy(np.asarray(v)).to(tdt).cuda()
        rng = SplitMix64(1201)
        cases = [("bw14x8", workloads.brickwork(14, 8).pattern, False),
                 ("bw14x8_in", workloads.brickwork(14, 8).pattern, True),
                 ("bw12x6", workloads.brickwork(12, 6).pattern, False),
                 ("qft10", workloads.qft(10, with_input=False).pattern, True),
                 ("small", workloads.small_random().pattern, True)]
        for n in (11, 13):
            cases.append((f"rand{{n}}", circuit_to_pattern(n, random_jcz_circuit(n, 6, rng, cz_per_layer=3), "r"), True))
        for name, p, real in cases:
            h = owqs.load(p)
            h.reorder()
            bits = workloads.forced_outcomes(p, SplitMix64(1300))
            psi = dev(random_state(SplitMix64(1301), len(p.inputs))) if real else None
            out, _, probs, st = h.run(psi, dtype=dtype, outcomes=bits, check=False)
            res[f"{{dtype}}:{{name}}:owqs"] = (st, out.cpu().numpy(), probs)
            out, _, probs, st = h.run(psi, dtype=dtype, mode="eowqs", outcomes=bits, check=False)
            res[f"{{dtype}}:{{name}}:eowqs"] = (st, out.cpu().numpy(), probs)
        p = workloads.brickwork(10, 6).pattern
        h = owqs.load(p)
        h.reorder()
        out, oc, probs, st = h.run(None, dtype=dtype, policy="sampled", seed=9, check=False)
        res[f"{{dtype}}:sampled"] = (st, out.cpu().numpy(), probs)
        out, oc, probs, st = h.run(None, dtype=dtype, policy="sampled", seed=9, check=False, sequential_sampling=True)
        res[f"{{dtype}}:sampled_seq"] = (st, out.cpu().numpy(), probs)
        p = circuit_to_pattern(6, random_jcz_circuit(6, 5, SplitMix64(1302), cz_per_layer=2), "r6")
        h = owqs.load(p)
        h.reorder()
        bits = workloads.forced_outcomes(p, SplitMix64(1303))
        factors = [(p.inputs[2 * f:2 * f + 2], dev(random_state(SplitMix64(1310 + f), 2))) for f in range(3)]
        out, _, probs, st = h.run_product(factors, dtype=dtype, outcomes=bits, check=False)
        res[f"{{dtype}}:product"] = (st, out.cpu().numpy(), probs)
        psi = dev(random_state(SplitMix64(1304), 6))
        out, _, probs, st = h.run_static(psi, dtype=dtype, outcomes=bits, check=False)
        res[f"{{dtype}}:static"] = (st, out.cpu().numpy(), probs)
        u, _ = h.unitary(dtype=dtype, outcomes=bits)
        res[f"{{dtype}}:unitary"] = (owqs.OK, u.cpu().numpy(), np.zeros(1))
        # separate sub-states (arena), double-float groups, groups that sum
        # every pass's norm, checked launches, an asynchronous run
        wl = workloads.brickwork(10, 6)
        h = owqs.load(wl.pattern)
        h.reorder()
        out, _, probs, st = h.run(None, dtype=dtype, outcomes=wl.outcomes, layout="substates", check=False)
        res[f"{{dtype}}:substates"] = (st, out.cpu().numpy(), probs)
        o = torch.empty(1 << 10, dtype=tdt, device="cuda")
        h.run_async(None, o, dtype=dtype, outcomes=wl.outcomes)
        _, probs, st = h.wait(check=False)
        res[f"{{dtype}}:async"] = (st, o.cpu().numpy(), probs)
        wl = workloads.brickwork(14, 8)
        h = owqs.load(wl.pattern)
        h.reorder()
        psi = dev(random_state(SplitMix64(1305), 14))
        out, _, probs, st = h.run(psi, dtype=dtype, outcomes=wl.outcomes, double_float=True, check=False)
        res[f"{{dtype}}:df"] = (st, out.cpu().numpy(), probs)
        wl = workloads.chain_measurements(14, 9, joined_every=0)
        h = owqs.load(wl.pattern)
        out, _, probs, st = h.run(dev(wl.psi_in), dtype=dtype, outcomes=wl.outcomes, layout="one_array", check=False)
        res[f"{{dtype}}:chain"] = (st, out.cpu().numpy(), probs)
        wl = workloads.brickwork_readout(7, 8, kept=2, with_input=True)
        h = owqs.load(wl.pattern)
        h.reorder()
        out, _, probs, st = h.run(dev(wl.psi_in), dtype=dtype, policy="sampled", seed=3, check=False)
        res[f"{{dtype}}:checked"] = (st, out.cpu().numpy(), probs)
    np.savez(out_path, **{{k + "|st": np.array(v[0]) for k, v in res.items()}},
             **{{k + "|out": v[1] for k, v in res.items()}}, **{{k + "|p": v[2] for k, v in res.items()}})


def shrunk(out_path):
    wl = workloads.brickwork(14, 8)
    h = owqs.load(wl.pattern)
    h.reorder()
    owqs.test_shrink_extents(1, 64)
    _, _, _, st = h.run(None, dtype="c64", outcomes=wl.outcomes, check=False)
    msg = owqs.last_error()
    out, _, _, st2 = h.run(None, dtype="c64", outcomes=wl.outcomes, check=False)   # the hook is spent
    np.savez(out_path, st=np.array(st), st2=np.array(st2), msg=np.array(msg), out=out.cpu().numpy())


if __name__ == "__main__":
    owqs.library(sys.argv[1])
    {{"cases": run_cases, "shrunk": shrunk}}[sys.argv[2]](sys.argv[3])
'''


@pytest.fixture(scope="module")
def libs(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_05659_gb300 import build
    build.ensure_built()
    checked = build.ensure_built(bounds_check=True)
    d = tmp_path_factory.mktemp("bounds")
    script = d / "cases.py"
    script.write_text(CASES.format(root=ROOT))
    return build, checked, d, script


def _child(script, lib, what, out):
    r = subprocess.run([sys.executable, str(script), lib, what, str(out)], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    return np.load(out)


def test_every_launch_kind_passes_the_checks_and_matches_release(libs):
    build, checked, d, script = libs
    rel = _child(script, build.LIB, "cases", d / "release.npz")
    chk = _child(script, checked, "cases", d / "checked.npz")
    keys = sorted(k[:-3] for k in rel.files if k.endswith("|st"))
    assert len(keys) == 2 * (7 * 2 + 5 + 5)
    for k in keys:
        assert int(chk[k + "|st"]) == 0, (k, int(chk[k + "|st"]))
        assert int(rel[k + "|st"]) == int(chk[k + "|st"]), k
        tol = 1e-6 if k.startswith("c64") else 1e-13
        assert np.max(np.abs(rel[k + "|out"] - chk[k + "|out"])) <= tol, k
        assert np.max(np.abs(rel[k + "|p"] - chk[k + "|p"])) <= tol, k


def test_shortened_extents_are_reported(libs):
    build, checked, d, script = libs
    r = _child(script, checked, "shrunk", d / "shrunk.npz")
    from paper_1604_05659_gb300 import owqs
    assert int(r["st"]) == owqs.ERR_CUDA and "outside its buffer" in str(r["msg"]), (int(r["st"]), str(r["msg"]))
    assert int(r["st2"]) == owqs.OK
    # the release build ignores extents: the same hook changes nothing there
    rr = _child(script, build.LIB, "shrunk", d / "shrunk_release.npz")
    assert int(rr["st"]) == owqs.OK and int(rr["st2"]) == owqs.OK
    assert np.max(np.abs(rr["out"] - r["out"])) <= 1e-6
