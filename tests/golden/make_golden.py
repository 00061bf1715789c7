"""Write the stored expected values of the full-size parity tests.

Runs ONLY the CPU FP64 oracle (oracle/) on the seeded workloads (workloads/)
and stores sampled entries, so that GPU tests can check full-size runs whose
oracle would take minutes.  Usage:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def sample_indices(d, count, seed):
    rng = np.random.default_rng(seed)
    idx = {(i, i) for i in rng.integers(0, d, count // 4)}       # diagonal entries (large)
    while len(idx) < count:
        idx.add((int(rng.integers(0, d)), int(rng.integers(0, d))))
    return sorted((int(i), int(j)) for i, j in idx)


def write_propagator_samples(wl, name, count=256, n_intervals=None):
    t0 = time.time()
    U = oracle.evolve_workload(wl, n_intervals=n_intervals)
    secs = time.time() - t0
    idx = sample_indices(wl.d, count, seed=12345)
    rec = {
        "what": f"sampled entries of the full propagator U(T) = U_(N-1)...U_0 of workloads.{name}",
        "source": "oracle.evolve_workload (CPU FP64: Gauss-Legendre quadrature, eigh exponentials, plain products)",
        "workload": {"name": wl.name, "d": wl.d, "K": wl.K, "N": wl.N, "P": wl.P, "T": wl.T,
                     "intervals_applied": wl.N if n_intervals is None else n_intervals},
        "oracle_seconds": secs,
        "unitarity_defect": oracle.unitarity_defect(U),
        "frobenius_norm": float(np.linalg.norm(U)),
        "trace": [float(np.trace(U).real), float(np.trace(U).imag)],
        "entries": [[i, j, float(U[i, j].real), float(U[i, j].imag)] for i, j in idx],
    }
    path = os.path.join(HERE, f"{name}.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    print(f"wrote {path} ({secs:.0f} s)")


if __name__ == "__main__":
    which = sys.argv[1:] or ["chain", "alltoall"]
    if "chain" in which:
        write_propagator_samples(W.config(1), "chain_d729_N2000_propagator")
    if "alltoall" in which:
        # the first 2 of the 500 intervals of the d = 4096 workload (one 4096 x 4096
        # eigendecomposition per interval on the CPU)
        write_propagator_samples(W.config(3), "alltoall_d4096_N500_first2_propagator", n_intervals=2)
