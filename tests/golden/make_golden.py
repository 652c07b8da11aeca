"""Write full-grid oracle results for a workload to tests/golden/<name>_oracle.json
and its full-grid density (float64, node order) to tests/golden/<name>_oracle_rho.npy.

Calls only oracle/ and synth/: every node's Lanczos bounds and Chebyshev
moments are computed by the CPU oracle (spread over spawned worker
processes; each node is independent, so the split does not change any
value), then the oracle's weights, Fermi-level bisection and
density/energy run over the whole grid in node order.

    python tests/golden/make_golden.py al108_48 [--procs N]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

_S = {}


def _init(name):
    s = synth.make_system(name)
    _S["wl"] = s.wl
    _S["osys"] = oracle.OracleSystem.from_synth(s)


def _chunk(nodes):
    wl, osys = _S["wl"], _S["osys"]
    chi, zeta = osys.bounds(nodes, wl.n_lanczos, wl.margin)
    mom = osys.moments(nodes, chi, zeta, wl.npl)
    return nodes, chi, zeta, mom


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name")
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--sample", type=int, default=512)
    a = ap.parse_args()
    oracle.build()
    wl = synth.WORKLOADS[a.name]
    N = wl.n_nodes
    chi = np.zeros(N)
    zeta = np.zeros(N)
    mom = np.zeros((N, wl.npl + 1))
    chunks = np.array_split(np.arange(N, dtype=np.int64), max(1, N // 256))
    t0 = time.time()
    with mp.get_context("spawn").Pool(a.procs, initializer=_init, initargs=(a.name,)) as pool:
        for i, (nodes, c, z, m) in enumerate(pool.imap_unordered(_chunk, chunks)):
            chi[nodes], zeta[nodes], mom[nodes] = c, z, m
            if i % 50 == 0:
                print(f"{i}/{len(chunks)} chunks, {time.time() - t0:.0f} s", flush=True)
    W = oracle.cc_weights(mom)
    mu, steps = oracle.fermi_level(W, chi, zeta, wl.n_electrons, wl.kT)
    rho, eb, es, ne = oracle.density_energy(W, chi, zeta, mu, wl.kT, wl.h)
    sample = synth.sample_nodes(N, a.sample, seed=2024)
    out = {
        "workload": a.name, "n_nodes": N, "npl": wl.npl, "kT": wl.kT, "n_electrons": wl.n_electrons,
        "n_lanczos": wl.n_lanczos, "margin": wl.margin,
        "mu": mu, "bisection_steps": steps, "e_band": eb, "e_ent": es, "n_elec": ne,
        "rho_norm2": float(np.linalg.norm(rho)), "rho_max": float(rho.max()), "rho_sum": float(rho.sum()),
        "moments_abs_max": float(np.abs(mom).max()),
        "sample_nodes": sample.tolist(), "sample_rho": rho[sample].tolist(),
        "sample_chi": chi[sample].tolist(), "sample_zeta": zeta[sample].tolist(),
        "sample_moments": mom[sample].tolist(),
        "source": "oracle/sq_oracle.c via tests/golden/make_golden.py (full grid, FP64)",
    }
    path = os.path.join(ROOT, "tests", "golden", f"{a.name}_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f)
    np.save(os.path.join(ROOT, "tests", "golden", f"{a.name}_oracle_rho.npy"), rho)
    print(f"wrote {path} in {time.time() - t0:.0f} s: mu={mu} e_band={eb} e_ent={es} N={ne}")


if __name__ == "__main__":
    main()
