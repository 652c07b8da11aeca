"""CPU oracle for the Spectral Quadrature hot path (plain serial FP64 C).

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The CUDA library never
imports, links or calls anything here, and this package imports nothing from
the CUDA package; the two share only the seeded input generator ``synth``.

``sq_oracle.c`` (the SQ path) and ``scf_oracle.c`` (Poisson, exchange and
mixing of the SCF loop around it) hold the arithmetic (each function cites
the passage of the paper it follows); this module only compiles them with
gcc, marshals numpy arrays through ctypes, and strings the SCF loop together
from those calls.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sq_oracle.c")
_SRC_SCF = os.path.join(_HERE, "scf_oracle.c")
_LIB = os.path.join(_HERE, "libsq_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_SCF))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-std=gnu11", "-o", tmp, _SRC, _SRC_SCF, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Sys(C.Structure):
    _fields_ = [("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int), ("h", C.c_double),
                ("no", C.c_int), ("m", C.c_int), ("periodic", C.c_int),
                ("V", C.POINTER(C.c_double)), ("n_atoms", C.c_int), ("R", C.POINTER(C.c_double)),
                ("n_ptypes", C.c_int), ("pl", C.POINTER(C.c_int)),
                ("pgamma", C.POINTER(C.c_double)), ("prc", C.POINTER(C.c_double)),
                ("prnl", C.POINTER(C.c_double))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp, lp, ip = C.POINTER(C.c_double), C.POINTER(C.c_long), C.POINTER(C.c_int)
            sp = C.POINTER(_Sys)
            lib.or_fd_weights.argtypes = [C.c_int, C.c_double, dp]
            lib.or_region_size.argtypes = [sp]; lib.or_region_size.restype = C.c_long
            lib.or_apply_H.argtypes = [sp, C.c_long, dp, dp]
            lib.or_dense_H.argtypes = [sp, C.c_long, dp]
            lib.or_num_projectors.argtypes = [sp, C.c_long]
            lib.or_tridiag_extremes.argtypes = [C.c_int, dp, dp, dp, dp]
            lib.or_lanczos_tridiag.argtypes = [sp, C.c_long, C.c_int, dp, dp, ip]
            lib.or_bounds.argtypes = [sp, C.c_long, lp, C.c_int, C.c_double, dp, dp]
            lib.or_moments.argtypes = [sp, C.c_long, lp, dp, dp, C.c_int, C.c_int, dp]
            lib.or_cheb_node.argtypes = [C.c_int, C.c_int]; lib.or_cheb_node.restype = C.c_double
            lib.or_cc_weights.argtypes = [C.c_long, C.c_int, dp, dp]
            lib.or_electron_count.argtypes = [C.c_long, C.c_int, dp, dp, dp, C.c_double, C.c_double]
            lib.or_electron_count.restype = C.c_double
            lib.or_fermi_level.argtypes = [C.c_long, C.c_int, dp, dp, dp, C.c_double, C.c_double, dp, ip]
            lib.or_density_energy.argtypes = [C.c_long, C.c_int, dp, dp, dp, C.c_double, C.c_double,
                                              C.c_double, dp, dp, dp, dp]
            lib.or_nl_force.argtypes = [sp, C.c_long, lp, dp, dp, C.c_int, C.c_double, C.c_double, dp]
            lib.or_grad_weights.argtypes = [C.c_int, C.c_double, dp]
            lib.or_laplacian_periodic.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, dp, dp]
            lib.or_poisson_cg.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, dp, dp, C.c_double,
                                          C.c_int, ip, dp]
            lib.or_xalpha.argtypes = [C.c_long, dp, C.c_double, dp]
            lib.or_xalpha.restype = None
            lib.or_anderson_step.argtypes = [C.c_long, C.c_int, dp, dp, C.c_double, dp]
            lib.or_kerker.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_double, C.c_double, dp, dp,
                                      C.c_double, C.c_int, ip]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def grad_weights(no: int, h: float) -> np.ndarray:
    """Central first-derivative weights of Eq. (FD:Gradient), index d = 0..no (wt[0] = 0)."""
    wt = np.zeros(no + 1)
    if _load().or_grad_weights(int(no), float(h), _dp(wt)) != 0:
        raise ValueError("bad FD parameters")
    return wt


def fd_weights(no: int, h: float) -> np.ndarray:
    """w_0..w_no of Eq. (FD:Laplacian)."""
    w = np.zeros(no + 1)
    if _load().or_fd_weights(no, h, _dp(w)) != 0:
        raise ValueError("bad FD parameters")
    return w


class OracleSystem:
    """A grid + potential + projectors, in the oracle's own representation.

    ``V`` has shape (n3, n2, n1) (x fastest).  ``proj_types`` is a list of
    (l, gamma, rc, r_nl).  ``periodic=True`` makes every region the whole
    periodic cell (used to compare against dense diagonalisation of the
    periodic Hamiltonian)."""

    def __init__(self, V, h, m, positions=None, proj_types=(), fd_half_order=6, periodic=False):
        self.V = _f64(V)
        n3, n2, n1 = self.V.shape
        self.shape = (n1, n2, n3)
        self.h, self.m, self.no, self.periodic = float(h), int(m), int(fd_half_order), bool(periodic)
        self.R = _f64(positions if positions is not None else np.zeros((0, 3))).reshape(-1, 3)
        pt = list(proj_types)
        self._pl = np.array([p[0] for p in pt] or [0], dtype=np.int32)
        self._pg = np.array([p[1] for p in pt] or [0.0])
        self._prc = np.array([p[2] for p in pt] or [1.0])
        self._prnl = np.array([p[3] for p in pt] or [0.0])
        self._s = _Sys(n1, n2, n3, self.h, self.no, self.m, int(self.periodic), _dp(self.V),
                       self.R.shape[0], _dp(self.R), len(pt),
                       self._pl.ctypes.data_as(C.POINTER(C.c_int)),
                       _dp(self._pg), _dp(self._prc), _dp(self._prnl))
        self.lib = _load()

    @classmethod
    def from_synth(cls, sysm, periodic=False):
        wl = sysm.wl
        return cls(sysm.V, wl.h, wl.m, sysm.positions, sysm.proj_types, wl.fd_half_order, periodic)

    @property
    def n_nodes(self):
        return int(np.prod(self.shape))

    @property
    def region_size(self):
        return int(self.lib.or_region_size(C.byref(self._s)))

    def apply_H(self, q, x):
        x = _f64(x).ravel()
        y = np.zeros_like(x)
        self.lib.or_apply_H(C.byref(self._s), int(q), _dp(x), _dp(y))
        return y

    def dense_H(self, q):
        N = self.region_size
        H = np.zeros((N, N))
        self.lib.or_dense_H(C.byref(self._s), int(q), _dp(H))
        return H

    def num_projectors(self, q):
        return int(self.lib.or_num_projectors(C.byref(self._s), int(q)))

    def lanczos_tridiag(self, q, nsteps):
        a, b, k = np.zeros(nsteps), np.zeros(nsteps), C.c_int(0)
        self.lib.or_lanczos_tridiag(C.byref(self._s), int(q), int(nsteps), _dp(a), _dp(b), C.byref(k))
        return a[:k.value], b[:max(k.value - 1, 0)]

    def bounds(self, nodes, n_lanczos=40, margin=0.01):
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        chi, zeta = np.zeros(len(nodes)), np.zeros(len(nodes))
        rc = self.lib.or_bounds(C.byref(self._s), len(nodes), nodes.ctypes.data_as(C.POINTER(C.c_long)),
                                int(n_lanczos), float(margin), _dp(chi), _dp(zeta))
        if rc:
            raise ValueError("or_bounds failed")
        return chi, zeta

    def nl_force(self, nodes, chi, zeta, npl, mu, kT):
        """Nonlocal atomic forces (n_atoms x 3) summed over the given nodes
        (Eq. Discrete:NLforce with the recurrence of Eq. Rec:FD1 to n_pl)."""
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        chi, zeta = _f64(chi), _f64(zeta)
        F = np.zeros((max(self.R.shape[0], 1), 3))
        if _load().or_nl_force(C.byref(self._s), nodes.size, nodes.ctypes.data_as(C.POINTER(C.c_long)), _dp(chi),
                               _dp(zeta), int(npl), float(mu), float(kT), _dp(F)) != 0:
            raise ValueError("bad arguments")
        return F[:self.R.shape[0]]

    def moments(self, nodes, chi, zeta, npl, product_rule=True):
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        chi, zeta = _f64(chi), _f64(zeta)
        mom = np.zeros((len(nodes), npl + 1))
        rc = self.lib.or_moments(C.byref(self._s), len(nodes), nodes.ctypes.data_as(C.POINTER(C.c_long)),
                                 _dp(chi), _dp(zeta), int(npl), int(bool(product_rule)), _dp(mom))
        if rc:
            raise ValueError("or_moments failed")
        return mom


def tridiag_extremes(a, b):
    a, b = _f64(a), _f64(np.append(b, 0.0))
    lo, hi = C.c_double(), C.c_double()
    _load().or_tridiag_extremes(len(a), _dp(a), _dp(b), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def cheb_nodes(npl):
    lib = _load()
    return np.array([lib.or_cheb_node(npl, k) for k in range(npl + 1)])


def cc_weights(mom):
    mom = _f64(mom)
    nq, K = mom.shape
    W = np.zeros_like(mom)
    _load().or_cc_weights(nq, K - 1, _dp(mom), _dp(W))
    return W


def electron_count(W, chi, zeta, mu, kT):
    W, chi, zeta = _f64(W), _f64(chi), _f64(zeta)
    return _load().or_electron_count(W.shape[0], W.shape[1] - 1, _dp(W), _dp(chi), _dp(zeta),
                                     float(mu), float(kT))


def fermi_level(W, chi, zeta, n_electrons, kT):
    """Returns (mu, bisection steps); raises if the bracket misses N_e."""
    W, chi, zeta = _f64(W), _f64(chi), _f64(zeta)
    mu, it = C.c_double(), C.c_int()
    rc = _load().or_fermi_level(W.shape[0], W.shape[1] - 1, _dp(W), _dp(chi), _dp(zeta),
                                float(n_electrons), float(kT), C.byref(mu), C.byref(it))
    if rc:
        raise ValueError("Fermi-level bracket does not straddle N_e")
    return mu.value, it.value


def density_energy(W, chi, zeta, mu, kT, h):
    """Returns (rho[nq], E_band, E_ent, N)."""
    W, chi, zeta = _f64(W), _f64(chi), _f64(zeta)
    rho = np.zeros(W.shape[0])
    eb, es, ne = C.c_double(), C.c_double(), C.c_double()
    _load().or_density_energy(W.shape[0], W.shape[1] - 1, _dp(W), _dp(chi), _dp(zeta), float(mu),
                              float(kT), float(h), _dp(rho), C.byref(eb), C.byref(es), C.byref(ne))
    return rho, eb.value, es.value, ne.value


def solve(osys: OracleSystem, npl, kT, n_electrons, n_lanczos=40, margin=0.01, nodes=None,
          bounds=None, product_rule=True):
    """The whole hot path on the CPU: bounds -> moments -> weights -> Fermi
    level -> density/energy.  ``nodes`` defaults to every node; ``bounds``
    (chi, zeta) may be given to skip the Lanczos step."""
    if nodes is None:
        nodes = np.arange(osys.n_nodes, dtype=np.int64)
    chi, zeta = bounds if bounds is not None else osys.bounds(nodes, n_lanczos, margin)
    mom = osys.moments(nodes, chi, zeta, npl, product_rule)
    W = cc_weights(mom)
    mu, it = fermi_level(W, chi, zeta, n_electrons, kT)
    rho, eb, es, ne = density_energy(W, chi, zeta, mu, kT, osys.h)
    return dict(chi=chi, zeta=zeta, moments=mom, W=W, mu=mu, bisection_steps=it, rho=rho,
                e_band=eb, e_ent=es, n_elec=ne)


# ---------------------------------------------------------------------------
# SCF loop pieces (scf_oracle.c) and the loop itself
# ---------------------------------------------------------------------------
def laplacian_periodic(x, h, no=6):
    """-lap_h x on the periodic grid; x has shape (n3, n2, n1)."""
    x = _f64(x)
    y = np.zeros_like(x)
    n3, n2, n1 = x.shape
    if _load().or_laplacian_periodic(n1, n2, n3, float(h), int(no), _dp(x), _dp(y)) != 0:
        raise ValueError("bad FD parameters")
    return y


def poisson(rho, h, no=6, tol=1e-12, max_iter=5000):
    """phi with -(1/4 pi) lap_h phi = rho - mean(rho), zero mean (periodic);
    returns (phi, iterations, relative residual)."""
    rho = _f64(rho)
    phi = np.zeros_like(rho)
    n3, n2, n1 = rho.shape
    it, res = C.c_int(), C.c_double()
    rc = _load().or_poisson_cg(n1, n2, n3, float(h), int(no), _dp(rho), _dp(phi), float(tol), int(max_iter),
                               C.byref(it), C.byref(res))
    if rc == 1:
        raise ValueError("bad arguments")
    return phi, it.value, res.value


def xalpha(rho, alpha=2.0 / 3.0):
    rho = _f64(rho)
    vx = np.zeros_like(rho)
    _load().or_xalpha(rho.size, _dp(rho), float(alpha), _dp(vx))
    return vx


def anderson_step(Xs, Fs, beta):
    """Xs, Fs: (mh + 1, n) iterates and residuals, oldest first."""
    Xs, Fs = _f64(Xs), _f64(Fs)
    out = np.zeros(Xs.shape[1])
    rc = _load().or_anderson_step(Xs.shape[1], Xs.shape[0] - 1, _dp(Xs), _dp(Fs), float(beta), _dp(out))
    if rc > 1:
        raise ValueError("bad history")
    return out


def kerker(f, h, k0, amin, no=6, tol=1e-12, max_iter=5000):
    """(-lap_h + amin k0^2)(-lap_h + k0^2)^{-1} f on the periodic grid; f has
    shape (n3, n2, n1).  Returns (y, CG iterations)."""
    f = _f64(f)
    y = np.zeros_like(f)
    n3, n2, n1 = f.shape
    it = C.c_int()
    rc = _load().or_kerker(n1, n2, n3, float(h), int(no), float(k0), float(amin), _dp(f), _dp(y), float(tol),
                           int(max_iter), C.byref(it))
    if rc == 1:
        raise ValueError("bad arguments")
    return y, it.value


_kerker = kerker      # the scf() argument of the same name shadows it there


def scf(V_loc, h, m, positions, proj_types, n_electrons, kT, npl, alpha=2.0 / 3.0, beta=0.3, history=7,
        tol=1e-6, max_iter=60, n_lanczos=40, margin=0.01, periodic=False, fd_half_order=6, poisson_tol=1e-12,
        kerker=None, period=1):
    """The SCF loop of Section 3 around the SQ path, with the effective
    potential as the fixed-point variable: V_in -> SQ density rho[V_in] ->
    V_out = V_loc + phi[rho] + v_x[rho] (phi: Eq. PoissonEqn with a
    neutralising background; v_x: Slater X-alpha), stopped when
    ||V_out - V_in|| <= tol ||V_out|| (2-norms); Anderson mixing with the last
    `history` differences.  Starts from V_in = V_loc.  ``kerker`` = (k0, amin)
    mixes the preconditioned residual P f (or_kerker) in place of f; the
    stopping test stays on f.  ``period`` = p > 1 is Periodic Pulay mixing
    (Section 3): the Anderson (Pulay) extrapolation on every p-th step
    (steps p-1, 2p-1, ... counting from 0), simple mixing x + beta f on the
    others, the history kept throughout.  Returns a dict with the converged
    V_in, rho, mu, energies, the residual history and iterations."""
    V_loc = _f64(V_loc)
    V_in = V_loc.copy()
    Xs, Fs, res = [], [], []
    out = None
    for it in range(max_iter):
        osys = OracleSystem(V_in, h, m, positions, proj_types, fd_half_order, periodic)
        out = solve(osys, npl, kT, n_electrons, n_lanczos, margin)
        rho = out["rho"].reshape(V_loc.shape)
        phi, _, _ = poisson(rho, h, fd_half_order, poisson_tol)
        V_out = V_loc + phi + xalpha(rho, alpha)
        f = (V_out - V_in).ravel()
        res.append(float(np.linalg.norm(f) / np.linalg.norm(V_out)))
        if res[-1] <= tol:
            return dict(V=V_in, V_out=V_out, rho=rho, mu=out["mu"], e_band=out["e_band"], e_ent=out["e_ent"],
                        n_elec=out["n_elec"], residuals=res, iterations=it + 1, converged=True)
        if kerker is not None:
            f = _kerker(f.reshape(V_loc.shape), h, kerker[0], kerker[1], fd_half_order)[0].ravel()
        Xs.append(V_in.ravel().copy())
        Fs.append(f.copy())
        Xs, Fs = Xs[-(history + 1):], Fs[-(history + 1):]
        if (it + 1) % period == 0:
            V_in = anderson_step(np.array(Xs), np.array(Fs), beta).reshape(V_loc.shape)
        else:
            V_in = anderson_step(np.array(Xs[-1:]), np.array(Fs[-1:]), beta).reshape(V_loc.shape)
    return dict(V=V_in, rho=out["rho"].reshape(V_loc.shape), mu=out["mu"], residuals=res, iterations=max_iter,
                converged=False)
