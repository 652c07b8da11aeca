"""GB300-native Spectral Quadrature hot path (arXiv:1708.07913, Section 3).

``sq`` is the ctypes binding of libsq.so (the C ABI in include/sq.h);
``SQSolver`` strings its calls together for one grid/geometry:

    bounds (Lanczos) -> Chebyshev moments -> Fermi level -> density/energy

Device memory and streams come from PyTorch; all arithmetic of the path runs
in libsq's CUDA kernels.
"""
from __future__ import annotations

from . import sq
from .sq import SQ_FP32, SQ_FP64, SQError

__all__ = ["sq", "SQSolver", "SQBatch", "SQSCF", "SQCNN", "warm_start_potential", "SQ_FP32", "SQ_FP64",
           "SQError", "build"]


def build(force: bool = False) -> str:
    from .builder import build as _build
    return _build(force=force)


class SQSolver:
    """One context (grid, region, projectors, precision) and its device buffers."""

    def __init__(self, shape, h, r_cut, npl, precision=SQ_FP64, positions=None, proj_types=(), fd_half_order=6,
                 device="cuda:0"):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.shape = tuple(int(s) for s in shape)          # (n1, n2, n3)
        self.npl = int(npl)
        self.h = float(h)
        n1, n2, n3 = self.shape
        self.n_nodes = n1 * n2 * n3
        self.n_atoms = len(positions) if (positions is not None and len(proj_types)) else 0
        with torch.cuda.device(self.device):
            self.ctx = sq.sq_setup_grid(n1, n2, n3, h, fd_half_order, r_cut, npl, precision, positions,
                                        list(proj_types))
            f64 = dict(dtype=torch.float64, device=self.device)
            self.chi = torch.empty(self.n_nodes, **f64)
            self.zeta = torch.empty(self.n_nodes, **f64)
            self.moments = torch.empty(self.n_nodes, self.npl + 1, **f64)
            self.rho = torch.empty(self.n_nodes, **f64)

    @classmethod
    def from_workload(cls, wl, positions, precision=SQ_FP64, device="cuda:0"):
        import synth
        return cls((wl.n, wl.n, wl.n), wl.h, wl.r_cut, wl.npl, precision, positions,
                   synth.projector_types(wl.nonlocal_), wl.fd_half_order, device)

    def close(self):
        if getattr(self, "ctx", None):
            sq.sq_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bounds(self, V, n_lanczos=40, margin=0.01):
        sq.sq_set_stream(self.ctx)
        sq.sq_spectral_bounds(self.ctx, V, self.chi, self.zeta, n_lanczos, margin)
        return self.chi, self.zeta

    def widen_bounds(self, V, V_ref, chi_ref, zeta_ref):
        """Bounds for V from bounds computed for V_ref, widened by w = max|V - V_ref|
        (Weyl's inequality; sq_widen_bounds) into self.chi, self.zeta; returns w."""
        sq.sq_set_stream(self.ctx)
        return sq.sq_widen_bounds(self.ctx, V, V_ref, chi_ref, zeta_ref, self.chi, self.zeta)

    def compute_moments(self, V, chi=None, zeta=None):
        sq.sq_set_stream(self.ctx)
        sq.sq_moments(self.ctx, V, self.chi if chi is None else chi, self.zeta if zeta is None else zeta,
                      self.moments)
        return self.moments

    def fermi_level(self, n_electrons, kT, chi=None, zeta=None):
        sq.sq_set_stream(self.ctx)
        return sq.sq_fermi_level(self.ctx, self.moments, self.chi if chi is None else chi,
                                 self.zeta if zeta is None else zeta, n_electrons, kT)

    def density_energy(self, mu, kT, chi=None, zeta=None):
        sq.sq_set_stream(self.ctx)
        return sq.sq_density_energy(self.ctx, self.moments, self.chi if chi is None else chi,
                                    self.zeta if zeta is None else zeta, mu, kT, self.rho)

    def nl_forces(self, V, mu, kT, chi=None, zeta=None, nodes=None):
        """Nonlocal atomic forces (n_atoms, 3), Ha/bohr, at Fermi level mu;
        ``nodes`` (int64 device tensor) restricts the sum to those nodes."""
        F = self.torch.zeros(max(self.n_atoms, 1) * 3, dtype=self.torch.float64, device=self.device)
        sq.sq_set_stream(self.ctx)
        chi = self.chi if chi is None else chi
        zeta = self.zeta if zeta is None else zeta
        if nodes is None:
            sq.sq_nl_forces(self.ctx, V, chi, zeta, mu, kT, F if self.n_atoms else None)
        else:
            sq.sq_nl_forces_nodes(self.ctx, V, chi, zeta, mu, kT, nodes, F if self.n_atoms else None)
        return F[:3 * self.n_atoms].view(self.n_atoms, 3)

    def solve(self, V, n_electrons, kT, n_lanczos=40, margin=0.01, bounds=None):
        """The whole path on a device potential V (float64, N_d).  ``bounds``
        = (chi, zeta) device tensors skips the Lanczos step."""
        if bounds is None:
            chi, zeta = self.bounds(V, n_lanczos, margin)
        else:
            chi, zeta = bounds
        self.compute_moments(V, chi, zeta)
        mu = self.fermi_level(n_electrons, kT, chi, zeta)
        eb, es, ne = self.density_energy(mu, kT, chi, zeta)
        return dict(mu=mu, e_band=eb, e_ent=es, n_elec=ne, rho=self.rho, moments=self.moments, chi=chi,
                    zeta=zeta)

    @property
    def launches(self):
        return sq.sq_launch_count(self.ctx)


class SQBatch:
    """Several SQSolver systems run as one batch: the whole step (bounds,
    moments, Fermi level, density/energies) of every system is one CUDA graph
    launch (sq_batch_* in include/sq.h): per-system streams, or persistent
    queue kernels per group of systems with one region size, whichever the
    autotuner measures faster unless a plan is set.  Results land in each
    solver's own buffers (chi, zeta, moments, rho)."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.batch = sq.sq_batch_create([s.ctx for s in self.solvers])

    def run(self, V, n_electrons, kT, n_lanczos=40, margin=0.01):
        """Enqueue the step for every system (V: list of device tensors)."""
        S = self.solvers
        sq.sq_batch_run(self.batch, list(V), [s.chi for s in S], [s.zeta for s in S], [s.moments for s in S],
                        [s.rho for s in S], list(n_electrons), list(kT), n_lanczos, margin)

    def results(self):
        """Wait; per system a dict with mu, e_band, e_ent, n_elec."""
        mu, eb, es, ne = sq.sq_batch_results(self.batch, len(self.solvers))
        return [dict(mu=a, e_band=b, e_ent=c, n_elec=d) for a, b, c, d in zip(mu, eb, es, ne)]

    def blocks(self):
        """Region-kernel grid chosen per system by the autotuner (0 = the full persistent grid)."""
        return sq.sq_batch_blocks(self.batch, len(self.solvers))

    def set_plan(self, plan, nodes_per_item=1):
        """sq.SQ_BATCH_AUTO, SQ_BATCH_STREAMS, SQ_BATCH_STREAMS_SHARE or SQ_BATCH_QUEUE."""
        sq.sq_batch_set_plan(self.batch, plan, nodes_per_item)

    def plan(self):
        """(plan, nodes_per_item) in use (after the first run)."""
        return sq.sq_batch_plan(self.batch)

    def set_wait(self, budget_cycles, wait_on_unset=False):
        """Wait budget of the queue plan (SM clock cycles); wait_on_unset makes every wait run out."""
        sq.sq_batch_set_wait(self.batch, budget_cycles, 1 if wait_on_unset else 0)

    def close(self):
        if getattr(self, "batch", None):
            sq.sq_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SQSCF:
    """The SCF loop around the path for one SQSolver: the effective potential
    is the fixed-point variable (V_in -> SQ density -> V_out = V_loc + phi +
    v_x, Anderson-mixed), stopped when ||V_out - V_in|| <= tol ||V_out||.
    Every step runs in libsq (sq_* calls, include/sq.h); this class only
    sequences them."""

    def __init__(self, solver, V_loc, n_electrons, kT, alpha=2.0 / 3.0, beta=0.3, history=7, n_lanczos=40,
                 margin=0.01, kerker=None, period=1, reuse_bounds=None, fresh_below=None, refine=None):
        """``kerker`` = (k0, amin): mix the Kerker-preconditioned residual
        (sq_kerker) in place of V_out - V_in; the stopping test stays on the
        unpreconditioned residual.  ``period`` = p > 1: Periodic Pulay
        mixing (extrapolation on every p-th step, simple mixing between).
        ``reuse_bounds`` = w_max (Ha): an iteration takes the Lanczos bounds
        of the last potential V_ref they were computed for, widened by
        w = max|V_in - V_ref| (sq_widen_bounds; by Weyl's inequality they
        still enclose every nodal spectrum), instead of running Lanczos, as
        long as w <= w_max.  Near convergence the bounds then stay fixed, so
        the SQ map the mixer iterates no longer changes with the rounding of
        fresh bounds (in FP32 that rounding moves zeta by ~1e-5 relative and
        puts a floor under the residual); the fixed point is that of SQ with
        those enclosing bounds, at most w_max wider than fresh ones -- and at
        low degree the SQ density moves noticeably with the bounds, so
        ``fresh_below`` = r ends the reuse once the residual is at or below
        r: from then on every iteration takes fresh bounds, and the loop ends
        on the fixed point of SQ with bounds of (nearly) its own potential.
        That changes the map the mixer iterates, so the mixing history is
        dropped at the switch (its differences belong to the old map; kept,
        they stalled Anderson mixing at the jump in the residual).
        ``refine`` = (solver_fp64, r_switch): once the residual is at or below
        r_switch, the remaining iterations run on solver_fp64 (an FP64
        context of the same grid and atoms), starting from the current bounds
        with a fresh mixing history (the FP32 map's differences in the
        history kept the loop wandering at the FP32 noise level for as many
        iterations as the history is long); they reuse the last Lanczos
        bounds widened by the potential change while that stays within 1e-3
        Ha (an FP64 Lanczos run costs about two FP64 SQ steps).  The FP32 recurrence
        leaves rounding noise of ~1e-6 relative in the density, which stalls
        the residual near that level; the FP64 iterations converge past it."""
        torch = solver.torch
        self.solver, self.V_loc = solver, V_loc
        self.kerker = None if kerker is None else (float(kerker[0]), float(kerker[1]))
        self.period = int(period)
        self.reuse = None if reuse_bounds is None else float(reuse_bounds)
        self.fresh_below = None if fresh_below is None else float(fresh_below)
        self.refine = None if refine is None else (refine[0], float(refine[1]))
        self.n_electrons, self.kT, self.alpha = float(n_electrons), float(kT), float(alpha)
        self.n_lanczos, self.margin = int(n_lanczos), float(margin)
        f64 = dict(dtype=torch.float64, device=solver.device)
        self.phi = torch.empty(solver.n_nodes, **f64)
        self.V_out = torch.empty(solver.n_nodes, **f64)
        self.V_pre = torch.empty(solver.n_nodes, **f64) if kerker is not None else None
        self._V = [torch.empty(solver.n_nodes, **f64), torch.empty(solver.n_nodes, **f64)]
        with torch.cuda.device(solver.device):
            self.mixer = sq.sq_mixer_create(solver.n_nodes, history, beta)

    def run(self, V0=None, tol=1e-6, max_iter=60, poisson_tol=1e-12, checkpoint=None, resume=None, on_step=None):
        """Returns a dict: V (the converged input potential), rho, mu,
        e_band, e_ent, n_elec, residuals, iterations, converged, poisson
        iterations per SCF step.  ``checkpoint``: a path; after every
        iteration the next input potential and the mixing history are saved
        there (.npz of .npy arrays).  ``resume``: such a file; the loop
        continues from it (V0 is then ignored).  ``on_step(V_in, rho, mu)`` is
        called after every SQ solve (e.g. to collect training pairs; the
        tensors are reused by the next iteration)."""
        import numpy as np
        sv = self.solver
        sq.sq_mixer_reset(self.mixer)
        V_in, V_next = self._V
        res, pit, out = [], [], None
        if resume is not None:
            ck = np.load(resume)
            V_in.copy_(self.solver.torch.from_numpy(ck["V"]))
            sq.sq_mixer_import(self.mixer, ck["X"], ck["F"])
            res = list(ck["residuals"])
        else:
            V_in.copy_(self.V_loc if V0 is None else V0)
        sq.sq_mixer_set_period(self.mixer, self.period, len(res))
        ref = None                                   # (V_ref, chi_ref, zeta_ref) of the last Lanczos run
        lanczos = 0
        refined_at = None
        reusing = self.reuse is not None             # still in the bound-reuse phase
        for it in range(len(res), max_iter):
            switched = False
            if self.refine is not None and refined_at is None and res and res[-1] <= self.refine[1]:
                fine = self.refine[0]
                fine.chi.copy_(sv.chi)
                fine.zeta.copy_(sv.zeta)
                sv, refined_at, switched = fine, it, True
            if reusing and self.fresh_below is not None and res and res[-1] <= self.fresh_below:
                reusing, switched = False, True      # the reuse ends for good
            if refined_at is not None:
                w_max = 1e-3
            elif reusing:
                w_max = self.reuse
            else:
                w_max = None                         # fresh bounds this iteration
            widened = False
            if ref is not None and w_max is not None:
                w = sv.widen_bounds(V_in, *ref)
                widened = w <= w_max
            if widened:
                out = sv.solve(V_in, self.n_electrons, self.kT, bounds=(sv.chi, sv.zeta))
            else:
                out = sv.solve(V_in, self.n_electrons, self.kT, self.n_lanczos, self.margin)
                lanczos += 1
                if self.reuse is not None or self.refine is not None:
                    ref = (V_in.clone(), sv.chi.clone(), sv.zeta.clone())
            if on_step is not None:
                on_step(V_in, sv.rho, out["mu"])
            sq.sq_set_stream(sv.ctx)
            k, _ = sq.sq_poisson(sv.ctx, sv.rho, self.phi, poisson_tol)
            pit.append(k)
            sq.sq_effective_potential(sv.ctx, self.V_loc, self.phi, sv.rho, self.alpha, self.V_out)
            if switched:
                sq.sq_mixer_reset(self.mixer)
            if self.kerker is None:
                res.append(sq.sq_mixer_step(self.mixer, V_in, self.V_out, V_next))
            else:
                r, _ = sq.sq_kerker(sv.ctx, V_in, self.V_out, self.kerker[0], self.kerker[1], self.V_pre)
                sq.sq_mixer_step(self.mixer, V_in, self.V_pre, V_next)
                res.append(r)
            if res[-1] <= tol:
                return dict(V=V_in, rho=sv.rho, mu=out["mu"], e_band=out["e_band"], e_ent=out["e_ent"],
                            n_elec=out["n_elec"], residuals=res, iterations=it + 1, converged=True,
                            poisson_iterations=pit, lanczos_runs=lanczos, refined_at=refined_at)
            V_in, V_next = V_next, V_in
            if checkpoint is not None:
                X, F = sq.sq_mixer_export(self.mixer, sv.n_nodes)
                np.savez(checkpoint, V=V_in.cpu().numpy(), X=X, F=F, residuals=np.array(res))
        return dict(V=V_in, rho=sv.rho, mu=out["mu"], e_band=out["e_band"], e_ent=out["e_ent"],
                    n_elec=out["n_elec"], residuals=res, iterations=max_iter, converged=False,
                    poisson_iterations=pit, lanczos_runs=lanczos, refined_at=refined_at)

    def close(self):
        if getattr(self, "mixer", None):
            sq.sq_mixer_destroy(self.mixer)
            self.mixer = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SQCNN:
    """The learned warm start's network (sq_cnn_*, include/sq.h): a 3-D CNN
    on the periodic grid mapping the 9^3 patch of the effective potential
    around each node to the node's SQ density.  Weights and activations in
    bfloat16 (or FP32), FP32 accumulation, FP32 master weights and Adam
    state; every step runs in libsq."""

    CHANNELS = 32
    KERNELS = (5, 3, 3)

    def __init__(self, bf16=True, seed=0, v_shift=-1.0, v_scale=1.0, rho_scale=0.03, device="cuda:0"):
        import numpy as np
        import torch
        self.torch, self.device, self.bf16 = torch, torch.device(device), bool(bf16)
        with torch.cuda.device(self.device):
            self.net = sq.sq_cnn_create(self.CHANNELS, self.bf16)
        C, (k1, k2, k3) = self.CHANNELS, self.KERNELS
        rng = np.random.default_rng(seed)            # variance 1/fan-in, zero biases
        parts = [rng.standard_normal(C * k1 ** 3) / np.sqrt(k1 ** 3), np.zeros(C),
                 rng.standard_normal(C * C * k2 ** 3) / np.sqrt(C * k2 ** 3), np.zeros(C),
                 rng.standard_normal(C * k3 ** 3) / np.sqrt(C * k3 ** 3), np.zeros(1)]
        self.set_params(np.concatenate(parts), v_shift, v_scale, rho_scale)

    def set_params(self, flat, v_shift, v_scale, rho_scale):
        self.scales = (float(v_shift), float(v_scale), float(rho_scale))
        sq.sq_cnn_set_params(self.net, flat, *self.scales)

    def params(self):
        return sq.sq_cnn_get_params(self.net)

    def predict(self, shape, V, out=None):
        """Density (float64, N) of the potential V (device float64, N) on the periodic grid ``shape`` = (n1, n2, n3)."""
        rho = out if out is not None else self.torch.empty(V.numel(), dtype=self.torch.float64, device=self.device)
        sq.sq_cnn_forward(self.net, shape, V, rho)
        return rho

    def train_step(self, batch, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        """One Adam step on the mean loss over ``batch`` = [(shape, V,
        rho_ref[, mu]), ...]; with mu the sample is seen as V - mu (the
        Fermi-level-referenced map).  Returns that mean loss."""
        total = 0.0
        try:
            for i, item in enumerate(batch):
                shape, V, ref = item[:3]
                if len(item) > 3:
                    lo, hi = getattr(self, "mu_seen", (item[3], item[3]))
                    self.mu_seen = (min(lo, item[3]), max(hi, item[3]))
                sq.sq_cnn_set_shift(self.net, item[3] if len(item) > 3 else 0.0)
                rho = self.torch.empty(V.numel(), dtype=self.torch.float64, device=self.device)
                total += sq.sq_cnn_backward(self.net, shape, V, ref, rho, accumulate=i > 0)
        finally:
            sq.sq_cnn_set_shift(self.net, 0.0)
        sq.sq_cnn_adam_step(self.net, lr, beta1, beta2, eps, grad_scale=1.0 / len(batch))
        return total / len(batch)

    def predict_electrons(self, shape, V, n_electrons, h, out=None, steps=50, center=None, half_width=None,
                          points=33):
        """Density of V for a network trained on V - mu: the shift mu with
        h^3 sum rho = n_electrons.  N(mu) is evaluated on ``points`` shifts
        evenly spread over center +- half_width (default: the middle of the
        Fermi levels seen in training, and the larger of 2 v_scale and the
        training range), the sign change of N - n_electrons nearest the
        centre is kept, and bisection narrows it in ``steps`` halvings (a
        trained network need not be monotone in mu far from its training
        range, so no direction is assumed).  Returns (rho, mu), or
        (None, None) when N never crosses n_electrons on the scan; the scan
        is kept in ``self.last_scan`` = (shifts, counts) for diagnosis."""
        rho = out if out is not None else self.torch.empty(V.numel(), dtype=self.torch.float64, device=self.device)
        h3 = float(h) ** 3
        lo_seen, hi_seen = getattr(self, "mu_seen", (0.0, 0.0))
        c = 0.5 * (lo_seen + hi_seen) if center is None else float(center)
        w = max(2.0 * self.scales[1], hi_seen - lo_seen) if half_width is None else float(half_width)

        def count(mu):
            sq.sq_cnn_set_shift(self.net, mu)
            return h3 * sq.sq_cnn_forward_sum(self.net, shape, V, rho)

        try:
            shifts = [c - w + 2.0 * w * k / (points - 1) for k in range(points)]
            counts = [count(m) for m in shifts]
            self.last_scan = (shifts, counts)
            f = [n - n_electrons for n in counts]
            best = None
            for k in range(points - 1):
                if f[k] == 0.0 or (f[k] < 0.0) != (f[k + 1] < 0.0):
                    d = abs(0.5 * (shifts[k] + shifts[k + 1]) - c)
                    if best is None or d < best[0]:
                        best = (d, k)
            if best is None:
                return None, None
            k = best[1]
            lo, hi, f_lo = shifts[k], shifts[k + 1], f[k]
            if f_lo == 0.0:
                hi = lo
            for _ in range(steps):
                if hi == lo:
                    break
                mid = 0.5 * (lo + hi)
                fm = count(mid) - n_electrons
                if (fm < 0.0) == (f_lo < 0.0):
                    lo, f_lo = mid, fm
                else:
                    hi = mid
            mu = 0.5 * (lo + hi)
            count(mu)                              # rho at the final shift
            return rho, mu
        finally:
            sq.sq_cnn_set_shift(self.net, 0.0)

    def save(self, path):
        import numpy as np
        np.savez(path, params=self.params(), scales=np.array(self.scales), bf16=np.array(self.bf16),
                 mu_seen=np.array(getattr(self, "mu_seen", (0.0, 0.0))))

    @classmethod
    def load(cls, path, device="cuda:0"):
        import numpy as np
        d = np.load(path)
        net = cls(bool(d["bf16"]), 0, *d["scales"], device=device)
        net.set_params(d["params"], *d["scales"])
        if "mu_seen" in d:
            net.mu_seen = tuple(float(x) for x in d["mu_seen"])
        return net

    def close(self):
        if getattr(self, "net", None):
            sq.sq_cnn_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def warm_start_potential(net, solver, V_loc, alpha=2.0 / 3.0, iters=30, tol=1e-4, beta=0.3, history=7,
                         poisson_tol=1e-10, kerker=None, accept=0.1, n_electrons=None):
    """The SCF's starting potential from the learned network: the fixed
    point of V_in -> rho = net(V_in) -> V_out = V_loc + phi[rho] + v_x(rho)
    (the SCF map with the network in place of the SQ solve, Anderson-mixed,
    Kerker-preconditioned if ``kerker`` = (k0, amin) is given, at most
    ``iters`` steps or until ||V_out - V_in|| <= tol ||V_out||).
    Plain SQ is the fallback: if the surrogate's last residual is not finite
    or above ``accept``, V_loc is returned instead.  The SCF that follows
    always runs the SQ path, which judges the result.  Returns (V_in,
    residuals, used): ``used`` tells whether the network's potential was
    kept.  With ``n_electrons`` the network is the Fermi-level-referenced
    map (trained on V - mu): each surrogate step finds mu so that the
    predicted density holds n_electrons (SQCNN.predict_electrons).  Every
    step runs in libsq."""
    import math
    torch = solver.torch
    shape = solver.shape
    f64 = dict(dtype=torch.float64, device=solver.device)
    V_in, V_next = V_loc.clone(), torch.empty(solver.n_nodes, **f64)
    rho, phi, V_out, V_pre = (torch.empty(solver.n_nodes, **f64) for _ in range(4))
    with torch.cuda.device(solver.device):
        mixer = sq.sq_mixer_create(solver.n_nodes, history, beta)
    res = []
    try:
        sq.sq_set_stream(solver.ctx)
        for _ in range(iters):
            try:
                if n_electrons is None:
                    net.predict(shape, V_in, out=rho)
                elif net.predict_electrons(shape, V_in, n_electrons, solver.h, out=rho)[0] is None:
                    res.append(float("nan"))
                    break
                sq.sq_poisson(solver.ctx, rho, phi, poisson_tol)
                sq.sq_effective_potential(solver.ctx, V_loc, phi, rho, alpha, V_out)
                if kerker is None:
                    res.append(sq.sq_mixer_step(mixer, V_in, V_out, V_next))
                else:
                    r, _ = sq.sq_kerker(solver.ctx, V_in, V_out, kerker[0], kerker[1], V_pre)
                    sq.sq_mixer_step(mixer, V_in, V_pre, V_next)
                    res.append(r)
            except SQError:                   # e.g. a non-finite prediction: fall back to plain SQ
                res.append(float("nan"))
                break
            V_in, V_next = V_next, V_in
            if not math.isfinite(res[-1]) or res[-1] <= tol:   # not finite, or converged
                break
    finally:
        sq.sq_mixer_destroy(mixer)
    used = bool(res) and math.isfinite(res[-1]) and res[-1] <= accept
    return (V_in if used else V_loc.clone()), res, used
