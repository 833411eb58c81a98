"""GPU parity of the MPPI elite selection (sim_mppi_select_elites, the same
device code the MPPI update runs) against the oracle's stable argsort: the
selected sample indices must be identical, on rows with ties, NaN, +-inf,
+-0, negative costs and fewer valid costs than elites, on both kernels: one
warp per row (up to 2048 costs and 32 elites) and one thread block per row
(beyond that, up to SIM_MAX_ELITES elites)."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import mppi as om
from paper_2606_01478_b300 import _lib as L
from paper_2606_01478_b300 import select_elites

pytestmark = pytest.mark.gpu


def _select(cost: np.ndarray, n_e: int):
    idx, jmin = select_elites(torch.tensor(cost, dtype=torch.float32, device="cuda"), n_e)
    return idx.cpu().numpy(), jmin.cpu().numpy()


def _expected(row: np.ndarray, n_e: int):
    valid = np.count_nonzero(~np.isnan(row))
    el = om.select_elites(row, n_e)[:min(n_e, valid)]
    jmin = row[el[0]] if len(el) else np.inf
    return np.sort(el), jmin


def _check(cost, n_e):
    cost = np.asarray(cost, np.float32)
    idx, jmin = _select(cost, n_e)
    for r in range(cost.shape[0]):
        el, jm = _expected(cost[r].astype(np.float64), n_e)
        got = idx[r]
        assert np.array_equal(got[:len(el)], el), (r, got[:len(el)], el)  # increasing index order
        assert np.all(got[len(el):] == -1)
        assert (jmin[r] == jm) or (np.isinf(jm) and np.isinf(jmin[r]))


@pytest.mark.parametrize("S_c", [1, 5, 31, 32, 33, 100, 1600, 2048, 2049, 100_000])
@pytest.mark.parametrize("n_e", [1, 16, 32, 33, 1000, 4096])
def test_random_rows(S_c, n_e):
    rng = np.random.default_rng(S_c * 100 + n_e)
    _check(rng.uniform(0.0, 1e4, (37, S_c)), n_e)


@pytest.mark.parametrize("S_c", [64, 1600, 2048, 2049, 5000, 60_000])
def test_ties_nan_inf_signed_zero(S_c):
    rng = np.random.default_rng(S_c)
    rows = []
    # heavy ties: costs from a handful of values
    rows.append(rng.integers(0, 4, S_c).astype(np.float64))
    # all equal
    rows.append(np.full(S_c, 3.5))
    # ties exactly at the threshold among distinct smaller values
    r = rng.uniform(10, 20, S_c)
    r[rng.choice(S_c, min(S_c, 40), replace=False)] = 5.0
    r[rng.choice(S_c, 5, replace=False)] = 1.0
    rows.append(r)
    # NaN, +-inf, negative values and both zeros
    r = rng.normal(0.0, 1.0, S_c)
    r[rng.choice(S_c, S_c // 3, replace=False)] = np.nan
    r[rng.choice(S_c, 7, replace=False)] = -np.inf
    r[rng.choice(S_c, 7, replace=False)] = np.inf
    r[rng.choice(S_c, 5, replace=False)] = -0.0
    r[rng.choice(S_c, 5, replace=False)] = 0.0
    rows.append(r)
    # fewer valid costs than elites, and none at all
    r = np.full(S_c, np.nan)
    r[rng.choice(S_c, 3, replace=False)] = rng.uniform(0, 1, 3)
    rows.append(r)
    rows.append(np.full(S_c, np.nan))
    # only infinities
    rows.append(np.where(rng.uniform(size=S_c) < 0.5, np.inf, -np.inf))
    for n_e in (1, 8, 32, 33, 500, 4096):
        _check(np.stack(rows), n_e)


def test_zero_rows_and_bad_arguments():
    lib = L.load()
    c = torch.zeros(4, 8, device="cuda")
    idx = torch.zeros(4, 2, dtype=torch.int32, device="cuda")
    assert lib.sim_mppi_select_elites(ctypes.c_void_p(c.data_ptr()), 0, 8, 2,
                                      ctypes.c_void_p(idx.data_ptr()), None, None) == L.SIM_OK
    for rows, S_c, n_e in ((-1, 8, 2), (4, 0, 2), (4, 8, 0), (4, 8, L.MAX_ELITES + 1), (1 << 27, 8, 2)):
        assert lib.sim_mppi_select_elites(ctypes.c_void_p(c.data_ptr()), rows, S_c, n_e,
                                          ctypes.c_void_p(idx.data_ptr()), None,
                                          None) == L.SIM_EINVAL


def test_binding_reports_rejected_arguments_with_their_code():
    """A rejected call surfaces as SimError carrying the library's code."""
    from paper_2606_01478_b300 import SimError
    c = torch.zeros(3, 10, device="cuda")
    with pytest.raises(SimError) as ei:
        select_elites(c, 0)
    assert ei.value.code == L.SIM_EINVAL
