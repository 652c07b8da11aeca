"""The learned SCF warm start on a workload, end to end:

1. training pairs: for seeded geometries of a small training cell, SCF
   iterations of the SQ path, keeping every (V_in, rho = SQ(V_in)) pair;
2. training: Adam on random minibatches of those pairs (SQCNN.train_step);
3. comparison: the SCF of the target system from V_loc and from the
   network's starting potential (warm_start_potential), iterations counted
   to the same residual.

Every step runs in libsq (the SQ path, Poisson, effective potential, mixer
and the network's kernels); this module sequences calls and keeps the pairs
on the device.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

import synth

from . import SQ_FP32, SQ_FP64, SQCNN, SQSCF, SQSolver, warm_start_potential


def pair_collector(solver, kT, pairs, mu_offsets=(0.0,)):
    """An ``on_step`` callback for SQSCF.run that appends (shape, V_in, rho,
    mu', offset) to ``pairs`` for every mu' = mu + offset.  The densities at shifted
    Fermi levels come from the same SQ solve: the moments do not depend on
    mu (Section 3.2), so each is one sq_density_energy call at mu'.  They
    teach a network fed V - mu how the density moves with the Fermi level.
    The solver's own density (the SCF's) is restored before returning."""
    shape = solver.shape

    def on_step(V, rho, mu):
        keep = rho.clone()
        for d in mu_offsets:
            if d == 0.0:
                pairs.append((shape, V.clone(), keep.clone(), float(mu), 0.0))
            else:
                solver.density_energy(float(mu) + d, kT)
                pairs.append((shape, V.clone(), solver.rho.clone(), float(mu) + d, float(d)))
        rho.copy_(keep)
    return on_step


def training_pairs(template, n_geometries, iters, seed, precision=SQ_FP32, device="cuda:0", mu_offsets=(0.0,)):
    """(shape, V_in, rho, mu, offset) device pairs (mu: the SQ Fermi level
    of that solve plus one of ``mu_offsets``; see pair_collector) from ``iters`` SCF
    iterations on each of ``n_geometries`` geometries of ``template`` (a
    synth.Workload), seeds seed, seed + 1, ...  Returns (pairs, seconds)."""
    import torch
    pairs = []
    t0 = time.perf_counter()
    for g in range(n_geometries):
        wl = dataclasses.replace(template, name=f"{template.name}-g{g}", seed=seed + g)
        s = synth.make_system(wl)
        solver = SQSolver.from_workload(wl, s.positions, precision=precision, device=device)
        V_loc = torch.from_numpy(s.V.ravel().copy()).to(device)
        scf = SQSCF(solver, V_loc, wl.n_electrons, wl.kT, margin=wl.margin)
        scf.run(tol=0.0, max_iter=iters, on_step=pair_collector(solver, wl.kT, pairs, mu_offsets))
        scf.close()
        solver.close()
    torch.cuda.synchronize()
    return pairs, time.perf_counter() - t0


def scf_pairs(pairs):
    """The pairs at the SCF's own Fermi level (offset 0): the only ones a
    network fed V itself (not V - mu) can learn from."""
    return [p for p in pairs if len(p) < 5 or p[4] == 0.0]


def input_scales(pairs, fermi_referenced=True):
    """(v_shift, v_scale, rho_scale) from the training pairs: mean and
    standard deviation of the network's input (V - mu, or V), mean of rho
    (host reductions of copies)."""
    some = pairs[: min(len(pairs), 64)]
    V = np.concatenate([p[1].cpu().numpy() - (p[3] if fermi_referenced else 0.0) for p in some])
    rho = np.concatenate([p[2].cpu().numpy() for p in some])
    return float(V.mean()), float(V.std()), float(rho.mean())


def train(net, pairs, steps, batch=8, lr=2e-3, lr_final=2e-4, seed=0, log_every=0, fermi_referenced=True):
    """Adam on random minibatches, learning rate decayed geometrically from
    lr to lr_final; with ``fermi_referenced`` the network learns V - mu -> rho.
    Returns (losses, seconds)."""
    import torch
    rng = np.random.default_rng(seed)
    losses = []
    t0 = time.perf_counter()
    for k in range(steps):
        r = lr * (lr_final / lr) ** (k / max(1, steps - 1))
        idx = rng.choice(len(pairs), size=min(batch, len(pairs)), replace=False)
        losses.append(net.train_step([pairs[i] if fermi_referenced else pairs[i][:3] for i in idx], r))
        if log_every and k % log_every == 0:
            print(f"step {k} loss {losses[-1]:.4e}", flush=True)
    torch.cuda.synchronize()
    return losses, time.perf_counter() - t0


def compare(nets, wl, tol=1e-6, max_iter=100, precision=SQ_FP32, device="cuda:0", beta=0.3, history=16,
            kerker=(0.5, 0.1), reuse_bounds=None, fresh_below=None, refine_at=None):
    """SCF iterations of ``wl`` from V_loc and from the warm start of each
    network in ``nets`` = {label: (net, fermi_referenced)}, all with the same
    mixer (Kerker-preconditioned unless ``kerker`` is None).  Returns
    {"plain": {...}, label: {...}} with iterations, convergence, residual
    histories, times, and for the warm starts the surrogate's steps and
    residual, whether the network's potential was kept, and the largest
    density difference to the plain SCF's fixed point.  ``reuse_bounds``,
    ``fresh_below`` and ``refine_at`` (an FP64 context takes over at that
    residual) are passed to SQSCF."""
    import torch
    s = synth.make_system(wl)
    solver = SQSolver.from_workload(wl, s.positions, precision=precision, device=device)
    fine = None
    if refine_at is not None:
        fine = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=device)
    V_loc = torch.from_numpy(s.V.ravel().copy()).to(device)
    scf = SQSCF(solver, V_loc, wl.n_electrons, wl.kT, beta=beta, history=history, margin=wl.margin, kerker=kerker,
                reuse_bounds=reuse_bounds, fresh_below=fresh_below,
                refine=None if fine is None else (fine, refine_at))
    t0 = time.perf_counter()
    plain = scf.run(tol=tol, max_iter=max_iter)
    out = {"plain": dict(iterations=plain["iterations"], converged=plain["converged"],
                         residuals=[float(r) for r in plain["residuals"]], seconds=time.perf_counter() - t0,
                         refined_at=plain["refined_at"], lanczos_runs=plain["lanczos_runs"])}
    rho_plain = plain["rho"].clone()
    for label, (net, fermi) in nets.items():
        t0 = time.perf_counter()
        V0, surrogate, used = warm_start_potential(net, solver, V_loc, history=history, kerker=kerker,
                                                   n_electrons=wl.n_electrons if fermi else None)
        t_surr = time.perf_counter() - t0
        t0 = time.perf_counter()
        warm = scf.run(V0=V0, tol=tol, max_iter=max_iter)
        drho = float((warm["rho"] - rho_plain).abs().max().item() / rho_plain.abs().max().item())
        out[label] = dict(iterations=warm["iterations"], converged=warm["converged"],
                          residuals=[float(r) for r in warm["residuals"]], seconds=time.perf_counter() - t0,
                          surrogate_steps=len(surrogate), surrogate_residual=float(surrogate[-1]),
                          surrogate_seconds=t_surr, network_used=used, rho_rel_diff=drho,
                          refined_at=warm["refined_at"], lanczos_runs=warm["lanczos_runs"])
    scf.close()
    solver.close()
    if fine is not None:
        fine.close()
    return out
