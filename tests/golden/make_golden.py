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


def write_propagator_samples(wl, name, count=256, n_intervals=None, streamed=False):
    t0 = time.time()
    if streamed:   # one interval at a time: the d = 4096 matrices of every interval do not fit in memory
        U, _ = oracle.evolve_workload_streamed(wl, n_intervals=n_intervals)
    else:
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


def _result_record(wl, out, count, seed):
    """psi in full (d <= 512) or sampled entries; U by sampled entries."""
    if wl.psi0 is not None:
        if wl.d <= 512:
            return {"kind": "state", "psi": [[float(v.real), float(v.imag)] for v in out]}
        idx = sorted(set(int(i) for i in np.random.default_rng(seed).integers(0, wl.d, count)))
        return {"kind": "state", "d": wl.d, "entries": [[i, float(out[i].real), float(out[i].imag)] for i in idx]}
    idx = sample_indices(wl.d, count, seed)
    return {"kind": "propagator", "unitarity_defect": oracle.unitarity_defect(out),
            "entries": [[i, j, float(out[i, j].real), float(out[i, j].imag)] for i, j in idx]}


def write_uneven_batch(name, stride=32):
    """Every stride-th instance of the 512-instance uneven batch (16 of them), psi(T) in full."""
    jobs = W.uneven_batch()
    t0 = time.time()
    recs = []
    for q in range(0, len(jobs), stride):
        wl = jobs[q]
        psi = oracle.evolve_workload(wl)
        recs.append({"index": q, "d": wl.d, "N": wl.N, **_result_record(wl, psi, 0, q)})
    rec = {"what": "psi(T) of every 32nd instance of workloads.uneven_batch() (512 instances, seed 2)",
           "source": "oracle.evolve_workload (CPU FP64)", "oracle_seconds": time.time() - t0, "jobs": recs}
    path = os.path.join(HERE, f"{name}.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=0)
    print(f"wrote {path} ({rec['oracle_seconds']:.0f} s)")


def write_serving_prefix(name, requests=24, n_cap=200, count=256):
    """The first `requests` requests of workloads.serving_stream(), each with its interval
    count capped at n_cap (the oracle of a d = 1388 request of 4126 intervals takes over an hour)."""
    stream = W.serving_stream()[:requests]
    t0 = time.time()
    recs = []
    for q, (arrival, spec) in enumerate(stream):
        spec = dict(spec, N=min(spec["N"], n_cap))
        wl = W.serving_job(spec)
        out = oracle.evolve_workload(wl)
        recs.append({"request": q, "arrival_s": arrival, "spec": spec, **_result_record(wl, out, count, 1000 + q)})
    rec = {"what": f"results of the first {requests} requests of workloads.serving_stream() (rate 200/s, seed 4), "
                   f"interval counts capped at {n_cap}",
           "source": "oracle.evolve_workload (CPU FP64)", "oracle_seconds": time.time() - t0, "requests": recs}
    path = os.path.join(HERE, f"{name}.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=0)
    print(f"wrote {path} ({rec['oracle_seconds']:.0f} s)")


if __name__ == "__main__":
    which = sys.argv[1:] or ["chain", "alltoall"]
    if "chain" in which:
        write_propagator_samples(W.config(1), "chain_d729_N2000_propagator")
    if "alltoall" in which:
        # the first 2 of the 500 intervals of the d = 4096 workload (one 4096 x 4096
        # eigendecomposition per interval on the CPU)
        write_propagator_samples(W.config(3), "alltoall_d4096_N500_first2_propagator", n_intervals=2)
    if "uneven" in which:
        write_uneven_batch("uneven_batch512_every32nd_state")
    if "serving" in which:
        write_serving_prefix("serving_stream_first24_Ncap200")
    if "alltoall130" in which:
        # the first 130 of the 500 intervals: two re-orthonormalisation boundaries at
        # R = 64 and a tree product across chunks
        write_propagator_samples(W.config(3), "alltoall_d4096_N500_first130_propagator", n_intervals=130,
                                 streamed=True)
