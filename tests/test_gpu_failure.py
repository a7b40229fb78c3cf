"""Failure detection without a GPU fault: every wait inside the bulk-copy
pass kernels is bounded.  The test hook makes one launch wait on a barrier
that nothing arrives at; the kernel gives up after a short limit, raises the
run's error flag and returns, the run reports OWQS_ERR_TIMEOUT, and the next
run on the same context is correct."""
import math

import numpy as np
import pytest

from owqs_inputs import workloads
from owqs_inputs.patterns import E, M, Pattern
from owqs_inputs.rng import SplitMix64, random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_05659_gb300 import build, owqs
    build.ensure_built()
    owqs.library()
    return torch, owqs


def _check_timeout_then_recovery(env, h, psi, outcomes, kind):
    torch, owqs = env
    ref_out, _, ref_p, st = h.run(psi, dtype="c64", outcomes=outcomes)
    assert st == owqs.OK
    ms, _, kd, _ = h.profile(psi, dtype="c64", outcomes=outcomes)
    assert kind in set(int(k) for k in kd)
    owqs.test_wait_timeout(1, 2_000_000)
    _, _, _, st = h.run(psi, dtype="c64", outcomes=outcomes, check=False)
    assert st == owqs.ERR_TIMEOUT
    assert "gave up" in owqs.last_error()
    out, _, p, st = h.run(psi, dtype="c64", outcomes=outcomes)  # the hook is spent
    torch.cuda.synchronize()
    assert st == owqs.OK
    assert torch.equal(out, ref_out) and np.array_equal(p, ref_p)


def test_group_kernel_wait_limit(env):
    torch, owqs = env
    wl = workloads.brickwork(14, 8)
    h = owqs.load(wl.pattern)
    h.reorder()
    _check_timeout_then_recovery(env, h, None, wl.outcomes, 8)


def test_tma_pass_wait_limit(env):
    """A single measurement on a 14-qubit input: one bulk-copy pass."""
    torch, owqs = env
    n = 14
    p = Pattern(n, list(range(n)), list(range(1, n)), [E(0, 1), E(0, 5), M(0, 0.7)], "one-measurement")
    h = owqs.load(p)
    psi = torch.from_numpy(random_state(SplitMix64(31), n).astype(np.complex64)).cuda()
    _check_timeout_then_recovery(env, h, psi, [1], 5)
