"""Full-size parity: the d = 729 chain over all 2000 intervals (the bench.py launch
configuration) against sampled entries of the oracle's U(T) stored in tests/golden/
(written by tests/golden/make_golden.py, which runs only the CPU oracle)."""
import json
import os

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09982_gb300 import magnus as M  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "chain_d729_N2000_propagator.json")


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def ctx():
    c = M.Context(0)
    yield c
    c.close()


def check(U, golden, tol):
    e = np.array(golden["entries"])
    i, j = e[:, 0].astype(int), e[:, 1].astype(int)
    ref = e[:, 2] + 1j * e[:, 3]
    err = np.abs(U[i, j] - ref).max()
    assert err <= tol, err
    assert abs(np.linalg.norm(U) - golden["frobenius_norm"]) <= 50 * tol
    return err


@pytest.mark.parametrize("L", [6])
def test_chain_d729_full_split(ctx, golden, L):
    wl = W.config(1)
    U, rep = M.evolve_workload(ctx, wl, M.MG_PREC_SPLIT, L)
    check(U.cpu().numpy(), golden, 1e-6)
    assert rep["unitarity_defect"] < 1e-6


@pytest.mark.slow
def test_chain_d729_full_fp64(ctx, golden):
    wl = W.config(1)
    U, rep = M.evolve_workload(ctx, wl, M.MG_PREC_FP64)
    check(U.cpu().numpy(), golden, 1e-11)


GOLDEN_4096 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "alltoall_d4096_N500_first2_propagator.json")


@pytest.mark.parametrize("prec,L,tol", [(M.MG_PREC_SPLIT, 6, 1e-6), (M.MG_PREC_FP64, 6, 1e-11)])
def test_alltoall_d4096_first_intervals(ctx, prec, L, tol):
    """d = 4096 (4 transmons x 8 levels, all-to-all, two-tone drives): the first 2 of its 500
    intervals against the oracle's sampled entries (one 4096 x 4096 eigendecomposition each)."""
    with open(GOLDEN_4096) as f:
        g = json.load(f)
    wl = W.config(3)
    U, rep = M.evolve_workload(ctx, wl, prec, L, N=g["workload"]["intervals_applied"])
    check(U.cpu().numpy(), g, tol)
