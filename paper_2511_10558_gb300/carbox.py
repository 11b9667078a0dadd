"""ctypes binding of the C ABI in include/carbox.h (argument marshalling only).

Every function of the header is exposed under its own name on ``lib``; the
helpers below only convert between numpy / torch objects and the C structures.
All numerical work happens in libcarbox.so. Importing this module loads the
library and raises if it has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libcarbox.so")

CBX_OK = 0
CBX_E_ARG, CBX_E_CUDA, CBX_E_NOMEM, CBX_E_TOO_LARGE = -1, -2, -3, -4
CBX_CELL_OK, CBX_CELL_MAX_STEPS, CBX_CELL_H_UNDERFLOW, CBX_CELL_BAD_INPUT = 0, 1, 2, 5
CBX_CELL_TAPE_FULL = 6
CBX_TWO_BODY, CBX_COSMIC_RAY, CBX_PHOTO, CBX_CR_PHOTO = 0, 1, 2, 3
CBX_FP64, CBX_MIXED = 0, 1
CBX_METHOD_BDF, CBX_METHOD_ESDIRK = 0, 1


class cbx_species(C.Structure):
    _fields_ = [("composition", C.c_int * 5), ("charge", C.c_int)]


class cbx_reaction(C.Structure):
    _fields_ = [("type", C.c_int), ("reac", C.c_int * 2), ("prod", C.c_int * 4),
                ("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double)]


class cbx_cell_params(C.Structure):
    _fields_ = [("n_H", C.c_double), ("T", C.c_double), ("A_V", C.c_double), ("G0", C.c_double),
                ("zeta", C.c_double)]


class cbx_options(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("max_steps", C.c_int), ("precision", C.c_int),
                ("max_refine", C.c_int), ("method", C.c_int), ("refine_tol", C.c_double)]


class cbx_cell_stats(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("steps", "attempts", "error_fails", "newton_fails", "rhs_evals",
                                        "jac_evals", "lu_factors", "newton_iters", "refine_sweeps", "reserved")] + \
        [("t_begin_ns", C.c_longlong), ("t_end_ns", C.c_longlong)]


STATS_FIELDS = ["steps", "attempts", "error_fails", "newton_fails", "rhs_evals", "jac_evals", "lu_factors",
                "newton_iters", "refine_sweeps"]
STATS_INTS = 14  # int32 words per cbx_cell_stats (10 ints + 2 int64)


def stats_tensor(n_cells, device):
    """A zeroed device buffer for per-cell cbx_cell_stats, as int32 [C, 14]."""
    import torch
    return torch.zeros((n_cells, STATS_INTS), dtype=torch.int32, device=device)


def stats_dict(arr):
    """Decode int32 [C, 14] stats rows into a dict of numpy arrays."""
    arr = np.ascontiguousarray(arr, dtype=np.int32)
    out = {f: arr[:, i] for i, f in enumerate(STATS_FIELDS)}
    t = arr[:, 10:14].copy().view(np.int64)
    out["t_begin_ns"] = t[:, 0]
    out["t_end_ns"] = t[:, 1]
    return out


class cbx_netinfo(C.Structure):
    _fields_ = [("S", C.c_int), ("R", C.c_int), ("nnz_jac", C.c_int), ("nnz_lu", C.c_int),
                ("lu_flops", C.c_double), ("lu_flops_dense", C.c_double), ("smem_bytes_fp64", C.c_int),
                ("smem_bytes_mixed", C.c_int)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is not built: run paper_2511_10558_gb300.build.build() "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(_LIB_PATH)
    P = C.c_void_p
    sig = {
        "cbx_version": (C.c_int, []),
        "cbx_last_error": (C.c_char_p, []),
        "cbx_default_options": (C.c_int, [C.POINTER(cbx_options)]),
        "cbx_network_create": (C.c_int, [C.POINTER(cbx_species), C.c_int, C.POINTER(cbx_reaction), C.c_int,
                                         C.POINTER(P)]),
        "cbx_network_destroy": (C.c_int, [P]),
        "cbx_network_info": (C.c_int, [P, C.POINTER(cbx_netinfo)]),
        "cbx_network_symbolic": (C.c_int, [P, P, P, C.POINTER(C.c_int)]),
        "cbx_solve": (C.c_int, [P, P, P, C.c_int, C.c_double, C.c_double, C.POINTER(cbx_options), P, P, P, P]),
        "cbx_solve_host": (C.c_int, [P, P, P, C.c_int, C.c_double, C.c_double, C.POINTER(cbx_options), P, P,
                                     P, P]),
        "cbx_network_set_alpha": (C.c_int, [P, P]),
        "cbx_network_set_albedo": (C.c_int, [P, C.c_double]),
        "cbx_tape_create": (C.c_int, [P, C.c_int, C.c_int, C.POINTER(P)]),
        "cbx_tape_destroy": (C.c_int, [P]),
        "cbx_solve_record": (C.c_int, [P, P, P, C.c_int, C.c_double, C.c_double, C.POINTER(cbx_options), P, P, P,
                                       P, P]),
        "cbx_solve_with_alpha": (C.c_int, [P, P, P, P, C.c_int, C.c_double, C.c_double, C.POINTER(cbx_options), P,
                                           P, P, P, P]),
        "cbx_grad": (C.c_int, [P, P, P, P, P, P]),
        "cbx_grad_env": (C.c_int, [P, P, P, P, P, P, P, P, P]),
        "cbx_solve_track": (C.c_int, [P, P, C.c_int, P, C.c_int, C.c_double, C.c_double, C.POINTER(cbx_options), P,
                                      P, P, P]),
        "cbx_tape_program": (C.c_int, [P, C.c_int, P, P, P, C.c_int]),
        "cbx_tape_step_times": (C.c_int, [P, C.c_int, P, C.c_int]),
        "cbx_solve_track_record": (C.c_int, [P, P, C.c_int, P, C.c_int, C.c_double, C.c_double,
                                             C.POINTER(cbx_options), P, P, P, P, P]),
        "cbx_server_create": (C.c_int, [C.c_size_t, C.c_int, C.c_int, C.POINTER(P)]),
        "cbx_server_submit": (C.c_int, [P, P, P, P, C.c_int, C.c_double, C.c_double, C.POINTER(cbx_options),
                                        C.POINTER(C.c_uint64)]),
        "cbx_server_poll": (C.c_int, [P, C.c_uint64, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "cbx_server_wait": (C.c_int, [P, C.c_uint64, P, P, P]),
        "cbx_server_stats": (C.c_int, [P, C.POINTER(C.c_size_t), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "cbx_server_destroy": (C.c_int, [P]),
        "cbx_server_info": (C.c_int, [P, C.POINTER(C.c_size_t), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
        "cbx_peak_fma": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, P, P]),
        "cbx_esdirk_tableau": (C.c_int, [P, P, C.POINTER(C.c_double)]),
        "cbx_peak_fma_flops": (C.c_double, [C.c_int, C.c_int, C.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class CarboxError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where} failed ({code}): {lib.cbx_last_error().decode()}")
        self.code = code


def check(code, where):
    if code != CBX_OK:
        raise CarboxError(code, where)


def options(rtol=1e-4, atol=1e-20, max_steps=100000, precision=CBX_FP64, max_refine=5, refine_tol=1e-10,
            method=CBX_METHOD_BDF):
    o = cbx_options()
    check(lib.cbx_default_options(C.byref(o)), "cbx_default_options")
    o.rtol, o.atol, o.max_steps, o.precision = rtol, atol, max_steps, precision
    o.max_refine, o.refine_tol, o.method = max_refine, refine_tol, method
    return o


def esdirk_tableau():
    """(A [5, 5], c [5], gamma) of CBX_METHOD_ESDIRK as the library derived it."""
    a = np.zeros(25)
    c = np.zeros(5)
    g = C.c_double()
    check(lib.cbx_esdirk_tableau(a.ctypes.data_as(C.c_void_p), c.ctypes.data_as(C.c_void_p), C.byref(g)),
          "cbx_esdirk_tableau")
    return a.reshape(5, 5), c, g.value


class Network:
    """Owns a cbx_network handle built from plain arrays (see synth.Network)."""

    def __init__(self, composition, charge, rtype, reac, prod, alpha, beta, gamma):
        S = len(charge)
        R = len(rtype)
        sp = (cbx_species * S)()
        for i in range(S):
            sp[i].composition[:] = [int(v) for v in composition[i]]
            sp[i].charge = int(charge[i])
        rx = (cbx_reaction * max(R, 1))()
        for j in range(R):
            rx[j].type = int(rtype[j])
            rx[j].reac[:] = [int(v) for v in reac[j]]
            rx[j].prod[:] = [int(v) for v in prod[j]]
            rx[j].alpha, rx[j].beta, rx[j].gamma = float(alpha[j]), float(beta[j]), float(gamma[j])
        h = C.c_void_p()
        check(lib.cbx_network_create(sp, S, rx, R, C.byref(h)), "cbx_network_create")
        self.handle = h
        self.S, self.R = S, R

    @classmethod
    def from_synth(cls, net):
        n = cls(net.composition, net.charge, net.rtype, net.reac, net.prod, net.alpha, net.beta, net.gamma)
        n.set_albedo(getattr(net, "albedo", 0.0))
        return n

    def set_albedo(self, omega):
        check(lib.cbx_network_set_albedo(self.handle, float(omega)), "cbx_network_set_albedo")

    def set_alpha(self, alpha):
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        assert a.shape == (self.R,)
        check(lib.cbx_network_set_alpha(self.handle, a.ctypes.data_as(C.c_void_p)), "cbx_network_set_alpha")

    def info(self):
        inf = cbx_netinfo()
        check(lib.cbx_network_info(self.handle, C.byref(inf)), "cbx_network_info")
        return {f: getattr(inf, f) for f, _ in cbx_netinfo._fields_}

    def symbolic(self):
        """(perm [S], fill [S, S] bool, kdense): the host compiler's ordering and L + U pattern."""
        perm = np.zeros(self.S, np.int32)
        fill = np.zeros((self.S, self.S), np.uint8)
        kd = C.c_int()
        check(lib.cbx_network_symbolic(self.handle, perm.ctypes.data_as(C.c_void_p), fill.ctypes.data_as(C.c_void_p),
                                       C.byref(kd)), "cbx_network_symbolic")
        return perm, fill.astype(bool), kd.value

    def close(self):
        if self.handle:
            lib.cbx_network_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def solve(net, phi, x0, t0, t_end, opt=None, stream=None, x_out=None, status=None, stats=None):
    """cbx_solve on torch CUDA tensors: phi [C, 5] f64, x0 [S, C] f64 (contiguous).

    Returns (x_out [S, C], status [C] int32, stats [C, 14] int32 or None; see stats_dict).
    """
    import torch
    Cn = phi.shape[0]
    assert phi.is_cuda and phi.dtype == torch.float64 and phi.is_contiguous() and phi.shape[1] == 5
    assert x0.is_cuda and x0.dtype == torch.float64 and x0.is_contiguous() and tuple(x0.shape) == (net.S, Cn)
    dev = phi.device
    if stats is not None:
        assert (stats.is_cuda and stats.dtype == torch.int32 and stats.is_contiguous()
                and tuple(stats.shape) == (Cn, STATS_INTS)), "stats must be stats_tensor(C, device)"
    if x_out is not None:
        assert x_out.is_cuda and x_out.dtype == torch.float64 and x_out.is_contiguous() and tuple(x_out.shape) == (net.S, Cn)
    if status is not None:
        assert status.is_cuda and status.dtype == torch.int32 and status.is_contiguous() and tuple(status.shape) == (Cn,)
    if x_out is None:
        x_out = torch.empty((net.S, Cn), dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty(Cn, dtype=torch.int32, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    o = opt if opt is not None else options()
    check(lib.cbx_solve(net.handle, _ptr(phi), _ptr(x0), Cn, float(t0), float(t_end), C.byref(o),
                        C.c_void_p(stream.cuda_stream), _ptr(x_out), _ptr(status), _ptr(stats)), "cbx_solve")
    return x_out, status, stats


def solve_track(net, track, x0, t0, t_end, opt=None, stream=None, stats=None):
    """cbx_solve_track on torch CUDA tensors: track [C, K, 6] f64 knots (t, n_H, T, A_V,
    G0, zeta), x0 [S, C] f64. Returns (x_out [S, C], status [C] int32, stats or None)."""
    import torch
    assert track.is_cuda and track.dtype == torch.float64 and track.is_contiguous() and track.dim() == 3
    assert track.shape[2] == 6
    Cn, K = int(track.shape[0]), int(track.shape[1])
    assert x0.is_cuda and x0.dtype == torch.float64 and x0.is_contiguous() and tuple(x0.shape) == (net.S, Cn)
    dev = track.device
    if stats is not None:
        assert (stats.is_cuda and stats.dtype == torch.int32 and stats.is_contiguous()
                and tuple(stats.shape) == (Cn, STATS_INTS)), "stats must be stats_tensor(C, device)"
    x_out = torch.empty((net.S, Cn), dtype=torch.float64, device=dev)
    status = torch.empty(Cn, dtype=torch.int32, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    o = opt if opt is not None else options()
    check(lib.cbx_solve_track(net.handle, _ptr(track), K, _ptr(x0), Cn, float(t0), float(t_end), C.byref(o),
                              C.c_void_p(stream.cuda_stream), _ptr(x_out), _ptr(status), _ptr(stats)),
          "cbx_solve_track")
    return x_out, status, stats


def solve_host(net, phi, x0, t0, t_end, opt=None, stream=None, want_stats=False):
    """cbx_solve_host on numpy arrays: phi [C, 5], x0 [S, C]; returns numpy results."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    Cn = phi.shape[0]
    assert x0.shape == (net.S, Cn)
    x_out = np.empty((net.S, Cn))
    status = np.empty(Cn, dtype=np.int32)
    stats = np.zeros((Cn, STATS_INTS), dtype=np.int32) if want_stats else None
    o = opt if opt is not None else options()
    s = C.c_void_p(stream.cuda_stream) if stream is not None else None
    check(lib.cbx_solve_host(net.handle, phi.ctypes.data_as(C.c_void_p), x0.ctypes.data_as(C.c_void_p), Cn,
                             float(t0), float(t_end), C.byref(o), s, x_out.ctypes.data_as(C.c_void_p),
                             status.ctypes.data_as(C.c_void_p),
                             stats.ctypes.data_as(C.c_void_p) if stats is not None else None), "cbx_solve_host")
    return x_out, status, stats


class Tape:
    """Owns a cbx_tape: the recorded forward trajectory of up to C cells."""

    def __init__(self, net, n_cells, max_steps=2000):
        h = C.c_void_p()
        check(lib.cbx_tape_create(net.handle, int(n_cells), int(max_steps), C.byref(h)), "cbx_tape_create")
        self.handle = h
        self.net = net
        self.C = n_cells

    def program(self, cell, cap=100000):
        """The recorded ops of one cell: list of (kind, q, value); kind 0 init, 1 rescale, 2 step."""
        kinds = np.zeros(cap, np.int32)
        qs = np.zeros(cap, np.int32)
        vals = np.zeros(cap)
        n = lib.cbx_tape_program(self.handle, int(cell), kinds.ctypes.data_as(C.c_void_p),
                                 qs.ctypes.data_as(C.c_void_p), vals.ctypes.data_as(C.c_void_p), cap)
        if n < 0:
            raise CarboxError(n, "cbx_tape_program")
        return [(int(kinds[i]), int(qs[i]), float(vals[i])) for i in range(min(n, cap))]

    def step_times(self, cell, cap=100000):
        """t_new of every recorded accepted step of one cell (numpy)."""
        ts = np.zeros(cap)
        n = lib.cbx_tape_step_times(self.handle, int(cell), ts.ctypes.data_as(C.c_void_p), cap)
        if n < 0:
            raise CarboxError(n, "cbx_tape_step_times")
        return ts[:min(n, cap)].copy()

    def close(self):
        if self.handle:
            lib.cbx_tape_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_record(net, tape, phi, x0, t0, t_end, opt=None, stream=None, stats=None):
    """cbx_solve_record on torch CUDA tensors (as ``solve``), recording into ``tape``."""
    import torch
    Cn = phi.shape[0]
    assert phi.is_cuda and phi.dtype == torch.float64 and phi.is_contiguous() and phi.shape[1] == 5
    assert x0.is_cuda and x0.dtype == torch.float64 and x0.is_contiguous() and tuple(x0.shape) == (net.S, Cn)
    if stats is not None:
        assert stats.dtype == torch.int32 and stats.is_contiguous() and tuple(stats.shape) == (Cn, STATS_INTS)
    x_out = torch.empty((net.S, Cn), dtype=torch.float64, device=phi.device)
    status = torch.empty(Cn, dtype=torch.int32, device=phi.device)
    if stream is None:
        stream = torch.cuda.current_stream(phi.device)
    o = opt if opt is not None else options()
    check(lib.cbx_solve_record(net.handle, _ptr(phi), _ptr(x0), Cn, float(t0), float(t_end), C.byref(o),
                               C.c_void_p(stream.cuda_stream), _ptr(x_out), _ptr(status), _ptr(stats),
                               tape.handle), "cbx_solve_record")
    return x_out, status


def solve_with_alpha(net, alpha, phi, x0, t0, t_end, opt=None, stream=None, tape=None, stats=None):
    """cbx_solve_with_alpha on torch CUDA tensors: the network's alpha replaced by
    alpha [R] (f64, device) for this call only; records into ``tape`` when given.
    Returns (x_out [S, C], status [C] int32)."""
    import torch
    Cn = phi.shape[0]
    assert alpha.is_cuda and alpha.dtype == torch.float64 and alpha.is_contiguous() and tuple(alpha.shape) == (net.R,)
    assert phi.is_cuda and phi.dtype == torch.float64 and phi.is_contiguous() and phi.shape[1] == 5
    assert x0.is_cuda and x0.dtype == torch.float64 and x0.is_contiguous() and tuple(x0.shape) == (net.S, Cn)
    if stats is not None:
        assert stats.dtype == torch.int32 and stats.is_contiguous() and tuple(stats.shape) == (Cn, STATS_INTS)
    x_out = torch.empty((net.S, Cn), dtype=torch.float64, device=phi.device)
    status = torch.empty(Cn, dtype=torch.int32, device=phi.device)
    if stream is None:
        stream = torch.cuda.current_stream(phi.device)
    o = opt if opt is not None else options()
    check(lib.cbx_solve_with_alpha(net.handle, _ptr(alpha), _ptr(phi), _ptr(x0), Cn, float(t0), float(t_end),
                                   C.byref(o), C.c_void_p(stream.cuda_stream), _ptr(x_out), _ptr(status),
                                   _ptr(stats), tape.handle if tape is not None else None), "cbx_solve_with_alpha")
    return x_out, status


def solve_track_record(net, tape, track, x0, t0, t_end, opt=None, stream=None, stats=None):
    """cbx_solve_track_record on torch CUDA tensors: track [C, K, 6] f64, x0 [S, C];
    returns (x_out [S, C], status [C] int32)."""
    import torch
    assert track.is_cuda and track.dtype == torch.float64 and track.is_contiguous() and track.dim() == 3
    Cn, K = int(track.shape[0]), int(track.shape[1])
    assert x0.is_cuda and x0.dtype == torch.float64 and x0.is_contiguous() and tuple(x0.shape) == (net.S, Cn)
    x_out = torch.empty((net.S, Cn), dtype=torch.float64, device=track.device)
    status = torch.empty(Cn, dtype=torch.int32, device=track.device)
    if stream is None:
        stream = torch.cuda.current_stream(track.device)
    o = opt if opt is not None else options()
    check(lib.cbx_solve_track_record(net.handle, _ptr(track), K, _ptr(x0), Cn, float(t0), float(t_end), C.byref(o),
                                     C.c_void_p(stream.cuda_stream), _ptr(x_out), _ptr(status), _ptr(stats),
                                     tape.handle), "cbx_solve_track_record")
    return x_out, status


def grad(tape, cot_x, n_cells, stream=None):
    """cbx_grad: (dL/d ln alpha [R], dL/d ln n_H [C], dL/dT [C]) for dL/dx(t_end) = cot_x [S, C]."""
    import torch
    assert cot_x.is_cuda and cot_x.dtype == torch.float64 and cot_x.is_contiguous()
    dev = cot_x.device
    ga = torch.empty(tape.net.R, dtype=torch.float64, device=dev)
    gn = torch.empty(n_cells, dtype=torch.float64, device=dev)
    gt = torch.empty(n_cells, dtype=torch.float64, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    check(lib.cbx_grad(tape.handle, _ptr(cot_x), C.c_void_p(stream.cuda_stream), _ptr(ga), _ptr(gn), _ptr(gt)),
          "cbx_grad")
    return ga, gn, gt


def grad_env(tape, cot_x, n_cells, stream=None):
    """cbx_grad_env: (dL/d ln alpha [R], dL/d ln n_H [C], dL/dT [C], dL/d ln zeta [C],
    dL/d ln G0 [C], dL/dA_V [C]) for dL/dx(t_end) = cot_x [S, C]."""
    import torch
    assert cot_x.is_cuda and cot_x.dtype == torch.float64 and cot_x.is_contiguous()
    dev = cot_x.device
    ga = torch.empty(tape.net.R, dtype=torch.float64, device=dev)
    out = [torch.empty(n_cells, dtype=torch.float64, device=dev) for _ in range(5)]
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    check(lib.cbx_grad_env(tape.handle, _ptr(cot_x), C.c_void_p(stream.cuda_stream), _ptr(ga),
                           *[_ptr(t) for t in out]), "cbx_grad_env")
    return (ga, *out)


def _make_function():
    import torch

    class CellSolve(torch.autograd.Function):
        """log10 x(t_end) [S, C] as a function of (ln alpha [R], ln n_H [C], T [C]).

        Forward: cbx_solve_with_alpha recording a tape (FP64 or mixed, per
        ``opt``), with alpha = exp(ln alpha) for this call only (the network
        is not modified); backward: cbx_grad, the hand-written discrete
        adjoint. Other inputs (x0, A_V, G0, zeta, times) are constants.
        """

        @staticmethod
        def forward(ctx, log_alpha, log_nH, T, net, x0, av_g0_zeta, t_end, opt, max_steps):
            alpha = torch.exp(log_alpha.detach()).to(device=x0.device, dtype=torch.float64).contiguous()
            phi = torch.stack([torch.exp(log_nH.detach()), T.detach(), av_g0_zeta[:, 0], av_g0_zeta[:, 1],
                               av_g0_zeta[:, 2]], dim=1).contiguous()
            tape = Tape(net, phi.shape[0], max_steps)
            x, status = solve_with_alpha(net, alpha, phi, x0, 0.0, t_end, opt, tape=tape)
            ctx.tape, ctx.x, ctx.status = tape, x, status
            return torch.log10(x)

        @staticmethod
        def backward(ctx, g):
            x = ctx.x
            g = g.contiguous()
            cot = torch.where(g != 0, g / (x * np.log(10.0)), torch.zeros_like(g)).contiguous()
            ga, gn, gt = grad(ctx.tape, cot, x.shape[1])
            return ga, gn, gt, None, None, None, None, None, None

    return CellSolve


_cell_solve = None


def cell_solve(log_alpha, log_nH, T, net, x0, av_g0_zeta, t_end, opt=None, max_steps=2000):
    """Differentiable solve: returns log10 x(t_end) [S, C] (see CellSolve)."""
    global _cell_solve
    if _cell_solve is None:
        _cell_solve = _make_function()
    return _cell_solve.apply(log_alpha, log_nH, T, net, x0, av_g0_zeta, t_end,
                             opt if opt is not None else options(), max_steps)


class Server:
    """cbx_server: continuous-batching solves of host-side requests."""

    def __init__(self, mem_budget=0, n_streams=8, max_ctas=76):
        h = C.c_void_p()
        check(lib.cbx_server_create(int(mem_budget), int(n_streams), int(max_ctas), C.byref(h)), "cbx_server_create")
        self.handle = h
        self._nets = {}

    def submit(self, net, phi, x0, t0, t_end, opt=None):
        """phi [C, 5], x0 [S, C] numpy arrays; returns a request id."""
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        rid = C.c_uint64()
        o = opt if opt is not None else options()
        check(lib.cbx_server_submit(self.handle, net.handle, phi.ctypes.data_as(C.c_void_p),
                                    x0.ctypes.data_as(C.c_void_p), phi.shape[0], float(t0), float(t_end),
                                    C.byref(o), C.byref(rid)), "cbx_server_submit")
        self._nets[rid.value] = (net.S, phi.shape[0])
        return rid.value

    def poll(self, rid):
        st = C.c_int()
        lat = C.c_double()
        check(lib.cbx_server_poll(self.handle, C.c_uint64(rid), C.byref(st), C.byref(lat)), "cbx_server_poll")
        return st.value, lat.value

    def wait(self, rid):
        """Blocks; returns (x_out [S, C], status [C], (t_submit, t_start, t_done))."""
        S, Cn = self._nets.pop(rid)
        x = np.empty((S, Cn))
        st = np.empty(Cn, dtype=np.int32)
        t = np.empty(3)
        check(lib.cbx_server_wait(self.handle, C.c_uint64(rid), x.ctypes.data_as(C.c_void_p),
                                  st.ctypes.data_as(C.c_void_p), t.ctypes.data_as(C.c_void_p)), "cbx_server_wait")
        return x, st, tuple(t)

    def stats(self):
        b = C.c_size_t()
        r = C.c_int()
        q = C.c_int()
        check(lib.cbx_server_stats(self.handle, C.byref(b), C.byref(r), C.byref(q)), "cbx_server_stats")
        return {"peak_bytes": b.value, "peak_running": r.value, "queued": q.value}

    def info(self):
        b = C.c_size_t()
        n = C.c_longlong()
        m = C.c_longlong()
        check(lib.cbx_server_info(self.handle, C.byref(b), C.byref(n), C.byref(m)), "cbx_server_info")
        return {"budget": b.value, "launches": n.value, "merged_requests": m.value}

    def close(self):
        if self.handle:
            lib.cbx_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
