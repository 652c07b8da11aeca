"""ctypes binding of libsq (include/sq.h): argument marshalling only.

Each function has the name and meaning of the C entry point.  Device arrays
are ``torch.Tensor`` objects on a CUDA device (float64, contiguous); the
binding passes their data pointers and the current torch stream.  Every step
of the path runs in libsq's kernels: there is no CPU fallback, and a missing
or unloadable library raises immediately.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsq.so")

SQ_OK, SQ_EINVAL, SQ_ECUDA, SQ_EBOUNDS, SQ_ENOCONV, SQ_ETIMEOUT, SQ_ENOMEM, SQ_ECAPACITY, SQ_EUNSUPPORTED = range(9)
SQ_FP64, SQ_FP32 = 0, 1

# Every entry point declared in include/sq.h.
EXPORTS = ("sq_setup_grid", "sq_set_stream", "sq_spectral_bounds", "sq_moments", "sq_fermi_level",
           "sq_density_energy", "sq_density_energy_noalloc", "sq_sync", "sq_launch_count", "sq_context_info", "sq_destroy",
           "sq_strerror", "sq_batch_create", "sq_batch_run", "sq_batch_results", "sq_batch_blocks",
           "sq_batch_set_plan", "sq_batch_plan", "sq_batch_set_wait", "sq_batch_destroy", "sq_poisson", "sq_widen_bounds", "sq_effective_potential", "sq_mixer_create",
           "sq_mixer_step",
           "sq_mixer_set_period", "sq_mixer_history", "sq_mixer_export", "sq_mixer_import", "sq_mixer_reset", "sq_mixer_destroy",
           "sq_nl_forces", "sq_nl_forces_nodes", "sq_kerker", "sq_cnn_param_count", "sq_cnn_create",
           "sq_cnn_set_params", "sq_cnn_get_params", "sq_cnn_forward", "sq_cnn_set_shift", "sq_cnn_forward_sum",
           "sq_cnn_backward", "sq_cnn_get_grads", "sq_cnn_adam_step", "sq_cnn_destroy")


class SQError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {sq_strerror(code)} (status {code})")


class ProjType(C.Structure):
    _fields_ = [("l", C.c_int), ("gamma", C.c_double), ("rc", C.c_double), ("r_nl", C.c_double)]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libsq.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None and path == LIB_PATH:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libsq.so not built at {path}; run __graft_entry__.build()")
        lib = C.CDLL(path)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
        lib.sq_setup_grid.argtypes = [C.POINTER(vp), ip, ip, ip, C.c_double, ip, C.c_double, ip, ip, ip, dp, ip,
                                      C.POINTER(ProjType), vp]
        lib.sq_set_stream.argtypes = [vp, vp]
        lib.sq_spectral_bounds.argtypes = [vp, vp, vp, vp, ip, C.c_double]
        lib.sq_moments.argtypes = [vp, vp, vp, vp, vp]
        lib.sq_fermi_level.argtypes = [vp, vp, vp, vp, C.c_double, C.c_double, dp]
        lib.sq_density_energy.argtypes = [vp, vp, vp, vp, C.c_double, C.c_double, vp, dp, dp, dp]
        lib.sq_density_energy_noalloc.argtypes = [ip, ip, ip, C.c_double, ip, vp, vp, vp, C.c_double, C.c_double,
                                                  vp, dp, dp, dp, vp]
        lib.sq_sync.argtypes = [vp]
        lib.sq_launch_count.argtypes = [vp]
        lib.sq_launch_count.restype = C.c_longlong
        lib.sq_context_info.argtypes = [vp, C.POINTER(ip), ip]
        lib.sq_destroy.argtypes = [vp]
        lib.sq_destroy.restype = None
        lib.sq_strerror.argtypes = [ip]
        lib.sq_strerror.restype = C.c_char_p
        pp = C.POINTER(vp)
        lib.sq_batch_create.argtypes = [C.POINTER(vp), ip, pp, vp]
        lib.sq_batch_run.argtypes = [vp, pp, pp, pp, pp, pp, dp, dp, ip, C.c_double]
        lib.sq_batch_results.argtypes = [vp, dp, dp, dp, dp]
        lib.sq_batch_blocks.argtypes = [vp, C.POINTER(ip)]
        lib.sq_batch_set_plan.argtypes = [vp, ip, ip]
        lib.sq_batch_plan.argtypes = [vp, C.POINTER(ip), C.POINTER(ip)]
        lib.sq_batch_set_wait.argtypes = [vp, C.c_longlong, ip]
        lib.sq_batch_destroy.argtypes = [vp]
        lib.sq_batch_destroy.restype = None
        lib.sq_poisson.argtypes = [vp, vp, vp, C.c_double, ip, C.POINTER(ip), dp]
        lib.sq_effective_potential.argtypes = [vp, vp, vp, vp, C.c_double, vp]
        lib.sq_widen_bounds.argtypes = [vp, vp, vp, vp, vp, vp, vp, dp]
        lib.sq_nl_forces.argtypes = [vp, vp, vp, vp, C.c_double, C.c_double, vp]
        lib.sq_nl_forces_nodes.argtypes = [vp, vp, vp, vp, C.c_double, C.c_double, vp, C.c_longlong, vp]
        lib.sq_mixer_set_period.argtypes = [vp, ip, C.c_longlong]
        lib.sq_kerker.argtypes = [vp, vp, vp, C.c_double, C.c_double, C.c_double, ip, vp, dp, C.POINTER(ip)]
        lib.sq_cnn_param_count.argtypes = [ip]
        lib.sq_cnn_param_count.restype = C.c_longlong
        lib.sq_cnn_create.argtypes = [C.POINTER(vp), ip, ip, vp]
        lib.sq_cnn_set_params.argtypes = [vp, dp, C.c_double, C.c_double, C.c_double]
        lib.sq_cnn_get_params.argtypes = [vp, dp]
        lib.sq_cnn_forward.argtypes = [vp, ip, ip, ip, vp, vp]
        lib.sq_cnn_set_shift.argtypes = [vp, C.c_double]
        lib.sq_cnn_forward_sum.argtypes = [vp, ip, ip, ip, vp, vp, dp]
        lib.sq_cnn_backward.argtypes = [vp, ip, ip, ip, vp, vp, vp, ip, dp]
        lib.sq_cnn_get_grads.argtypes = [vp, dp]
        lib.sq_cnn_adam_step.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]
        lib.sq_cnn_destroy.argtypes = [vp]
        lib.sq_cnn_destroy.restype = None
        lib.sq_mixer_create.argtypes = [C.POINTER(vp), C.c_longlong, ip, C.c_double, vp]
        lib.sq_mixer_step.argtypes = [vp, vp, vp, vp, dp]
        lib.sq_mixer_history.argtypes = [vp, C.POINTER(ip)]
        lib.sq_mixer_export.argtypes = [vp, dp, dp]
        lib.sq_mixer_import.argtypes = [vp, ip, dp, dp]
        lib.sq_mixer_reset.argtypes = [vp]
        lib.sq_mixer_destroy.argtypes = [vp]
        lib.sq_mixer_destroy.restype = None
        if path == LIB_PATH:
            _lib = lib
        return lib


def sq_strerror(code: int) -> str:
    return load().sq_strerror(int(code)).decode()


def _check(rc: int, where: str):
    if rc != SQ_OK:
        raise SQError(rc, where)


def _dptr(t, name):
    """Device pointer of a contiguous float64 CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def sq_setup_grid(n1, n2, n3, h, fd_half_order, r_cut, npl, precision, positions=None, proj_types=(),
                  stream=None):
    """Returns an opaque context handle (int)."""
    lib = load()
    ctx = C.c_void_p()
    pos = np.ascontiguousarray(positions if positions is not None else np.zeros((0, 3)), dtype=np.float64)
    pt = (ProjType * max(len(proj_types), 1))(*[ProjType(*p) for p in proj_types])
    rc = lib.sq_setup_grid(C.byref(ctx), int(n1), int(n2), int(n3), float(h), int(fd_half_order), float(r_cut),
                           int(npl), int(precision), int(pos.shape[0]),
                           pos.ctypes.data_as(C.POINTER(C.c_double)) if pos.size else None,
                           len(proj_types), pt if len(proj_types) else None,
                           stream if stream is not None else _stream())
    _check(rc, "sq_setup_grid")
    return ctx.value


def sq_set_stream(ctx, stream=None):
    _check(load().sq_set_stream(C.c_void_p(ctx), stream if stream is not None else _stream()), "sq_set_stream")


def sq_spectral_bounds(ctx, V, chi, zeta, n_lanczos, margin):
    _check(load().sq_spectral_bounds(C.c_void_p(ctx), _dptr(V, "V"), _dptr(chi, "chi"), _dptr(zeta, "zeta"),
                                     int(n_lanczos), float(margin)), "sq_spectral_bounds")


def sq_moments(ctx, V, chi, zeta, moments):
    _check(load().sq_moments(C.c_void_p(ctx), _dptr(V, "V"), _dptr(chi, "chi"), _dptr(zeta, "zeta"),
                             _dptr(moments, "moments")), "sq_moments")


def sq_fermi_level(ctx, moments, chi, zeta, n_electrons, kT) -> float:
    mu = C.c_double()
    _check(load().sq_fermi_level(C.c_void_p(ctx), _dptr(moments, "moments"), _dptr(chi, "chi"),
                                 _dptr(zeta, "zeta"), float(n_electrons), float(kT), C.byref(mu)),
           "sq_fermi_level")
    return mu.value


def sq_density_energy(ctx, moments, chi, zeta, mu, kT, rho):
    """Fills rho; returns (E_band, E_ent, N)."""
    eb, es, ne = C.c_double(), C.c_double(), C.c_double()
    _check(load().sq_density_energy(C.c_void_p(ctx), _dptr(moments, "moments"), _dptr(chi, "chi"),
                                    _dptr(zeta, "zeta"), float(mu), float(kT), _dptr(rho, "rho"),
                                    C.byref(eb), C.byref(es), C.byref(ne)), "sq_density_energy")
    return eb.value, es.value, ne.value


def sq_nl_forces(ctx, V, chi, zeta, mu, kT, forces):
    """forces: float64 CUDA tensor of n_atoms*3 (None when there are no projectors)."""
    _check(load().sq_nl_forces(C.c_void_p(ctx), _dptr(V, "V"), _dptr(chi, "chi"), _dptr(zeta, "zeta"), float(mu),
                               float(kT), _dptr(forces, "forces")), "sq_nl_forces")


def sq_nl_forces_nodes(ctx, V, chi, zeta, mu, kT, nodes, forces):
    """nodes: int64 CUDA tensor of node indices."""
    import torch
    if not (isinstance(nodes, torch.Tensor) and nodes.is_cuda and nodes.dtype == torch.int64 and nodes.is_contiguous()):
        raise TypeError("nodes must be a contiguous int64 CUDA tensor")
    _check(load().sq_nl_forces_nodes(C.c_void_p(ctx), _dptr(V, "V"), _dptr(chi, "chi"), _dptr(zeta, "zeta"),
                                     float(mu), float(kT), C.c_void_p(nodes.data_ptr()), int(nodes.numel()),
                                     _dptr(forces, "forces")), "sq_nl_forces_nodes")


def sq_density_energy_noalloc(shape, h, npl, moments, chi, zeta, mu, kT, rho, stream=None):
    """Allocation-free density/energy step (no context); fills rho, returns
    (E_band, E_ent, N).  For callers that cannot let the library allocate
    device memory."""
    n1, n2, n3 = shape
    eb, es, ne = C.c_double(), C.c_double(), C.c_double()
    _check(load().sq_density_energy_noalloc(int(n1), int(n2), int(n3), float(h), int(npl),
                                            _dptr(moments, "moments"), _dptr(chi, "chi"), _dptr(zeta, "zeta"),
                                            float(mu), float(kT), _dptr(rho, "rho"), C.byref(eb), C.byref(es),
                                            C.byref(ne), stream if stream is not None else _stream()),
           "sq_density_energy_noalloc")
    return eb.value, es.value, ne.value


def sq_sync(ctx):
    _check(load().sq_sync(C.c_void_p(ctx)), "sq_sync")


def sq_launch_count(ctx) -> int:
    return int(load().sq_launch_count(C.c_void_p(ctx)))


NL_GLOBAL, NL_ALL, NL_HOT = 0, 1, 2


def sq_context_info(ctx) -> dict:
    """The launch configuration the context chose: region half-width m, the
    most projector candidates of any node, the projector-table placement
    (NL_GLOBAL / NL_ALL / NL_HOT) and the region kernels' resident CTAs."""
    out = (C.c_int * 4)()
    _check(load().sq_context_info(C.c_void_p(ctx), out, 4), "sq_context_info")
    return dict(m=out[0], ccap=out[1], tables=out[2], blocks=out[3])


def sq_destroy(ctx):
    if ctx:
        load().sq_destroy(C.c_void_p(ctx))


def _ptrs(ts, name):
    arr = (C.c_void_p * len(ts))(*[_dptr(t, f"{name}[{i}]") for i, t in enumerate(ts)])
    return C.cast(arr, C.POINTER(C.c_void_p)), arr


def _dbl(xs):
    return (C.c_double * len(xs))(*[float(x) for x in xs])


def sq_batch_create(ctxs, stream=None):
    """Returns an opaque batch handle over the given context handles."""
    lib = load()
    b = C.c_void_p()
    arr = (C.c_void_p * len(ctxs))(*[C.c_void_p(c) for c in ctxs])
    _check(lib.sq_batch_create(C.byref(b), len(ctxs), C.cast(arr, C.POINTER(C.c_void_p)),
                               stream if stream is not None else _stream()), "sq_batch_create")
    return b.value


def sq_batch_run(batch, V, chi, zeta, moments, rho, n_electrons, kT, n_lanczos, margin):
    """Lists (one entry per system) of device tensors and per-system N_e, kT."""
    keep = [_ptrs(V, "V"), _ptrs(chi, "chi"), _ptrs(zeta, "zeta"), _ptrs(moments, "moments"), _ptrs(rho, "rho")]
    ne, kt = _dbl(n_electrons), _dbl(kT)
    _check(load().sq_batch_run(C.c_void_p(batch), *[k[0] for k in keep], ne, kt, int(n_lanczos), float(margin)),
           "sq_batch_run")


def sq_batch_results(batch, n):
    """Waits for the batch; returns lists (mu, E_band, E_ent, N)."""
    out = [(C.c_double * n)() for _ in range(4)]
    _check(load().sq_batch_results(C.c_void_p(batch), *out), "sq_batch_results")
    return [list(o) for o in out]


def sq_batch_blocks(batch, n):
    out = (C.c_int * n)()
    _check(load().sq_batch_blocks(C.c_void_p(batch), out), "sq_batch_blocks")
    return list(out)


SQ_BATCH_AUTO, SQ_BATCH_STREAMS, SQ_BATCH_STREAMS_SHARE, SQ_BATCH_QUEUE = -1, 0, 1, 2


def sq_batch_set_plan(batch, plan, nodes_per_item=1):
    _check(load().sq_batch_set_plan(C.c_void_p(batch), int(plan), int(nodes_per_item)), "sq_batch_set_plan")


def sq_batch_plan(batch):
    """(plan, nodes_per_item) in use after the first run."""
    p, k = C.c_int(0), C.c_int(0)
    _check(load().sq_batch_plan(C.c_void_p(batch), C.byref(p), C.byref(k)), "sq_batch_plan")
    return p.value, k.value


def sq_batch_set_wait(batch, budget_cycles, wait_on_unset=0):
    _check(load().sq_batch_set_wait(C.c_void_p(batch), int(budget_cycles), int(wait_on_unset)), "sq_batch_set_wait")


def sq_batch_destroy(batch):
    if batch:
        load().sq_batch_destroy(C.c_void_p(batch))


def sq_poisson(ctx, rho, phi, tol=1e-12, max_iter=5000):
    """Fills phi; returns (iterations, relative residual)."""
    it, res = C.c_int(), C.c_double()
    _check(load().sq_poisson(C.c_void_p(ctx), _dptr(rho, "rho"), _dptr(phi, "phi"), float(tol), int(max_iter),
                             C.byref(it), C.byref(res)), "sq_poisson")
    return it.value, res.value


def sq_widen_bounds(ctx, V, V_ref, chi_ref, zeta_ref, chi, zeta) -> float:
    """chi = chi_ref, zeta = zeta_ref + w with w = max|V - V_ref| (Weyl enclosure); returns w."""
    w = C.c_double()
    _check(load().sq_widen_bounds(C.c_void_p(ctx), _dptr(V, "V"), _dptr(V_ref, "V_ref"), _dptr(chi_ref, "chi_ref"),
                                  _dptr(zeta_ref, "zeta_ref"), _dptr(chi, "chi"), _dptr(zeta, "zeta"), C.byref(w)),
           "sq_widen_bounds")
    return w.value


def sq_effective_potential(ctx, V_loc, phi, rho, alpha, V_out):
    _check(load().sq_effective_potential(C.c_void_p(ctx), _dptr(V_loc, "V_loc"), _dptr(phi, "phi"),
                                         _dptr(rho, "rho"), float(alpha), _dptr(V_out, "V_out")),
           "sq_effective_potential")


def sq_kerker(ctx, v_in, v_out, k0, amin, v_pre, tol=1e-10, max_iter=2000):
    """Fills v_pre = v_in + P (v_out - v_in); returns (||v_out - v_in|| / ||v_out||, CG iterations)."""
    res, it = C.c_double(), C.c_int()
    _check(load().sq_kerker(C.c_void_p(ctx), _dptr(v_in, "v_in"), _dptr(v_out, "v_out"), float(k0), float(amin),
                            float(tol), int(max_iter), _dptr(v_pre, "v_pre"), C.byref(res), C.byref(it)), "sq_kerker")
    return res.value, it.value


def sq_mixer_create(n, history, beta, stream=None):
    m = C.c_void_p()
    _check(load().sq_mixer_create(C.byref(m), int(n), int(history), float(beta),
                                  stream if stream is not None else _stream()), "sq_mixer_create")
    return m.value


def sq_mixer_step(mixer, v_in, v_out, v_next) -> float:
    res = C.c_double()
    _check(load().sq_mixer_step(C.c_void_p(mixer), _dptr(v_in, "v_in"), _dptr(v_out, "v_out"),
                                _dptr(v_next, "v_next"), C.byref(res)), "sq_mixer_step")
    return res.value


def sq_mixer_set_period(mixer, period, steps_done=0):
    _check(load().sq_mixer_set_period(C.c_void_p(mixer), int(period), int(steps_done)), "sq_mixer_set_period")


def sq_mixer_export(mixer, n):
    """The stored history as numpy arrays (X, F), each (count, n), oldest first."""
    lib = load()
    cnt = C.c_int()
    _check(lib.sq_mixer_history(C.c_void_p(mixer), C.byref(cnt)), "sq_mixer_history")
    X = np.zeros((cnt.value, n))
    F = np.zeros((cnt.value, n))
    _check(lib.sq_mixer_export(C.c_void_p(mixer), X.ctypes.data_as(C.POINTER(C.c_double)),
                               F.ctypes.data_as(C.POINTER(C.c_double))), "sq_mixer_export")
    return X, F


def sq_mixer_import(mixer, X, F):
    X = np.ascontiguousarray(X, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    _check(load().sq_mixer_import(C.c_void_p(mixer), int(X.shape[0]), X.ctypes.data_as(C.POINTER(C.c_double)),
                                  F.ctypes.data_as(C.POINTER(C.c_double))), "sq_mixer_import")


def sq_mixer_reset(mixer):
    _check(load().sq_mixer_reset(C.c_void_p(mixer)), "sq_mixer_reset")


def sq_mixer_destroy(mixer):
    if mixer:
        load().sq_mixer_destroy(C.c_void_p(mixer))


def sq_cnn_param_count(channels=32) -> int:
    return int(load().sq_cnn_param_count(int(channels)))


def sq_cnn_create(channels=32, bf16=True, stream=None):
    net = C.c_void_p()
    _check(load().sq_cnn_create(C.byref(net), int(channels), int(bool(bf16)),
                                stream if stream is not None else _stream()), "sq_cnn_create")
    return net.value


def sq_cnn_set_params(net, params, v_shift, v_scale, rho_scale):
    """params: flat float64 array in the network's natural order."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    if p.size != sq_cnn_param_count():
        raise ValueError("wrong parameter count")
    _check(load().sq_cnn_set_params(C.c_void_p(net), p.ctypes.data_as(C.POINTER(C.c_double)), float(v_shift),
                                    float(v_scale), float(rho_scale)), "sq_cnn_set_params")


def sq_cnn_get_params(net):
    p = np.zeros(sq_cnn_param_count())
    _check(load().sq_cnn_get_params(C.c_void_p(net), p.ctypes.data_as(C.POINTER(C.c_double))), "sq_cnn_get_params")
    return p


def sq_cnn_forward(net, shape, V, rho):
    n1, n2, n3 = shape
    _check(load().sq_cnn_forward(C.c_void_p(net), int(n1), int(n2), int(n3), _dptr(V, "V"), _dptr(rho, "rho")),
           "sq_cnn_forward")


def sq_cnn_set_shift(net, shift):
    _check(load().sq_cnn_set_shift(C.c_void_p(net), float(shift)), "sq_cnn_set_shift")


def sq_cnn_forward_sum(net, shape, V, rho) -> float:
    n1, n2, n3 = shape
    tot = C.c_double()
    _check(load().sq_cnn_forward_sum(C.c_void_p(net), int(n1), int(n2), int(n3), _dptr(V, "V"), _dptr(rho, "rho"),
                                     C.byref(tot)), "sq_cnn_forward_sum")
    return tot.value


def sq_cnn_backward(net, shape, V, rho_ref, rho, accumulate=False, want_loss=True):
    n1, n2, n3 = shape
    L = C.c_double()
    _check(load().sq_cnn_backward(C.c_void_p(net), int(n1), int(n2), int(n3), _dptr(V, "V"),
                                  _dptr(rho_ref, "rho_ref"), _dptr(rho, "rho"), int(bool(accumulate)),
                                  C.byref(L) if want_loss else None), "sq_cnn_backward")
    return L.value if want_loss else None


def sq_cnn_get_grads(net):
    g = np.zeros(sq_cnn_param_count())
    _check(load().sq_cnn_get_grads(C.c_void_p(net), g.ctypes.data_as(C.POINTER(C.c_double))), "sq_cnn_get_grads")
    return g


def sq_cnn_adam_step(net, lr, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0):
    _check(load().sq_cnn_adam_step(C.c_void_p(net), float(lr), float(beta1), float(beta2), float(eps),
                                   float(grad_scale)), "sq_cnn_adam_step")


def sq_cnn_destroy(net):
    if net:
        load().sq_cnn_destroy(C.c_void_p(net))
