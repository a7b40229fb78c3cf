"""Pins of the reference network (oracle/mlp.py) on the CPU: its analytic
backward pass against central finite differences of its own loss (without
bfloat16 rounding, where the loss is smooth), and its bfloat16 rounding
against hand-checked bit patterns."""
import numpy as np

from oracle import mlp
from owqs_inputs.rng import SplitMix64


def _data(seed, steps=7, width=5):
    rng = SplitMix64(seed)
    params = (rng.uniform_block(mlp.NPARAM) * 2 - 1) * 0.3
    first = [0]
    target = []
    for s in range(steps):
        n = 2 + rng.randint(width)
        target.append(first[-1] + rng.randint(n))
        first.append(first[-1] + n)
    X = rng.uniform_block(first[-1] * mlp.NF).reshape(-1, mlp.NF) * 2
    return params, X, np.array(first), np.array(target)


def test_backward_matches_finite_differences():
    params, X, first, target = _data(1)
    loss, g = mlp.loss_and_grad(params, X, first, target, bf=False)
    rng = SplitMix64(2)
    idx = sorted({rng.randint(mlp.NPARAM) for _ in range(60)} | {mlp.P_B3, mlp.P_W3, mlp.P_B1, mlp.P_W2 + 5})
    h = 1e-6
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, X, first, target, bf=False)[0] -
              mlp.loss_and_grad(pm, X, first, target, bf=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])
    # the loss is a mean of cross-entropies: positive, and log(n) for equal scores
    zero = np.zeros(mlp.NPARAM)
    l0, _ = mlp.loss_and_grad(zero, X, first, target, bf=False)
    want = np.mean([np.log(first[s + 1] - first[s]) for s in range(len(target))])
    assert abs(l0 - want) < 1e-12 and loss > 0


def test_bf16_rounding_bits():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to even (1.0)
    assert mlp.bf16(1.0 + 2 ** -8) == 1.0
    assert mlp.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6
    assert mlp.bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7
    assert mlp.bf16(-3.14159) == -3.140625
    x = np.linspace(-5, 5, 1001)
    r = mlp.bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8 + 1e-30)
