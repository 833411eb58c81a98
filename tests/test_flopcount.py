"""The FLOP counter's restated step computes the FP64 oracle's step (so the
count is of the method's arithmetic), and the counting scalar tallies what it
should: one per arithmetic operation on a per-drone value, none for
parameter-only constants."""
import numpy as np
import pytest
import torch

import flopcount as fc
import workloads as W
from oracle import physics as ph


def test_counting_scalar():
    c = fc._count(lambda: (fc.Num(2.0) * 3.0 + 1.0) / fc.Num(4.0) - 2.0 * 3.0)
    assert c == {"flop": 4, "mufu": 0, "cmp": 0}
    c = fc._count(lambda: fc.sqrt(fc.clip(fc.Num(5.0) * 0.5, 0.0, 1.0)))
    assert c == {"flop": 1, "mufu": 1, "cmp": 2}


def _oracle_step(x, a, P, rk4, model):
    Pb = ph.param_batch([P], [0])
    return ph.step(torch.tensor(np.asarray(x)[None], dtype=torch.float64),
                   torch.tensor(np.asarray(a)[None], dtype=torch.float64), Pb, 1 / 500,
                   ph.RK4 if rk4 else ph.EULER, ph.CTRL_ATTITUDE, model)[0].numpy()


@pytest.mark.parametrize("rk4", [False, True])
def test_restated_first_principles_step_is_the_oracles(rk4):
    rng = np.random.default_rng(4)
    P = W.crazyflie_params()
    for _ in range(5):
        x = W.fp_state(rng.uniform(-1, 1, (1, 3)), rng.uniform(-0.5, 0.5, (1, 3)), rng.uniform(-1, 1, (1, 3)),
                       rng.uniform(-2, 2, (1, 3)), rng.uniform(12000, 17000, (1, 4)))[0]
        a = rng.uniform(-1.2, 1.2, 4)  # some actions beyond the clip
        got = fc.step_fp([fc.Num(v) for v in x], [fc.Num(v) for v in a], P, 1 / 500, rk4, fc.mixer_inverse(P))
        got = np.array([fc._v(v) for v in got])
        np.testing.assert_allclose(got, _oracle_step(x, a, P, rk4, ph.FIRST_PRINCIPLES), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("rk4", [False, True])
def test_restated_abstracted_step_is_the_oracles(rk4):
    rng = np.random.default_rng(5)
    P = W.crazyflie_params()
    for _ in range(5):
        x = np.zeros(20)
        x[:13] = W.abs_state(rng.uniform(-1, 1, (1, 3)), rng.uniform(-0.5, 0.5, (1, 3)), rng.uniform(-1, 1, (1, 3)),
                             rng.uniform(-1, 1, (1, 3)), np.array([0.3]))[0, :13]
        a = rng.uniform(-1, 1, 4)
        got = fc.step_abs([fc.Num(v) for v in x], [fc.Num(v) for v in a], P, 1 / 500, rk4)
        got = np.array([fc._v(v) for v in got])
        np.testing.assert_allclose(got, _oracle_step(x, a, P, rk4, ph.ABSTRACTED), rtol=1e-12, atol=1e-12)


def test_counts_of_the_benchmark_steps():
    """RK4 = controller + 4 derivatives + the stage and final combinations
    (3 x 17 x 2 + 17 x 7 = 221) + the renormalisation (11); Euler replaces the
    three stage evaluations and the combination by 17 x 2."""
    t = fc.table()
    fp4, fp1 = t[("fp", "rk4")]["step_without_decode"], t[("fp", "euler")]["step_without_decode"]
    deriv = (fp4["flop"] - fp1["flop"] - (221 - 34)) / 3
    assert deriv == int(deriv) and deriv > 0
    ctrl = fp1["flop"] - deriv - 34 - 11
    assert fp4["flop"] == ctrl + 4 * deriv + 221 + 11
    assert t[("abs", "euler")]["step_without_decode"]["mufu"] == 6
    assert t[("fp", "rk4")]["mufu"] == pytest.approx(5 + 6 / 50)
