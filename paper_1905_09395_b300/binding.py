"""ctypes binding of libstev.so (include/stev.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; this module
checks shapes and dtypes, hands raw pointers over, and turns error codes into
exceptions.  It never falls back to anything: without the built library every
call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstev.so")

STEV_OK, STEV_EINVAL, STEV_ENOMEM, STEV_ECUDA, STEV_ETIMEOUT, STEV_EUNBALANCED, \
    STEV_EINCOMPLETE = range(7)
CELL_OK, CELL_MAXITER, CELL_NONFINITE, CELL_TRANGE = range(4)
FP64, MIXED = 0, 1
THERMO_POLY, THERMO_MLP, THERMO_MLP_CPH = 0, 1, 2

# every symbol include/stev.h declares
EXPORTS = (
    "stev_default_options", "stev_mechanism_create", "stev_mechanism_set_options",
    "stev_mechanism_get_options", "stev_solve", "stev_solve_soa", "stev_solve_host",
    "stev_resident_slots", "stev_destroy", "stev_last_error", "stev_solve_host_noalloc",
    "stev_mlp_num_params", "stev_mlp_train", "stev_mlp_set_params", "stev_mlp_get_params",
    "stev_mlp_loss_grad", "stev_mlp_eval", "stev_solve_batched",
    "stev_server_create", "stev_server_submit", "stev_server_poll", "stev_server_get_stats",
    "stev_server_clock", "stev_server_stop", "stev_server_destroy", "stev_mlp_stalls",
    "stev_mlp_train_lm", "stev_mlp_jacobian", "stev_mechanism_create_orders",
    "stev_is_specialized", "stev_spec_compile_check", "stev_gram_tf32", "stev_damped_cg",
    "stev_mp_solve",
)


class StevError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("stev error %d: %s" % (code, msg))
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [
        ("y_step_max", ctypes.c_double), ("delta_max", ctypes.c_double),
        ("alpha", ctypes.c_double), ("dft_n", ctypes.c_int), ("dft_hi_first", ctypes.c_int),
        ("tol_ring", ctypes.c_double), ("tol_freq", ctypes.c_double),
        ("r_fac", ctypes.c_double), ("rof_min", ctypes.c_double), ("max_iters", ctypes.c_int),
        ("precision", ctypes.c_int), ("thermo", ctypes.c_int), ("dft_on", ctypes.c_int),
        ("lanes_per_cell", ctypes.c_int), ("specialize", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RequestInfo(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("mechanism", ctypes.c_int), ("status", ctypes.c_int),
                ("n_cells", ctypes.c_long), ("cells_done", ctypes.c_long),
                ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("admitted", ctypes.c_longlong),
                ("completed", ctypes.c_longlong), ("cancelled", ctypes.c_longlong),
                ("cells_completed", ctypes.c_longlong), ("resident_bytes", ctypes.c_size_t),
                ("peak_resident_bytes", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t),
                ("kernel_launches", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libstev.so is not built (run __graft_entry__.build() or "
                               "python paper_1905_09395_b300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D, LNG = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
        L.stev_default_options.argtypes = [P]
        L.stev_default_options.restype = None
        L.stev_mechanism_create.argtypes = [I, I, P, P, P, P, P, P, P, P, P, P, P, P]
        L.stev_mechanism_create.restype = I
        L.stev_mechanism_create_orders.argtypes = [I, I, P, P, P, P, P, P, P, P, P, P, P, P, P]
        L.stev_mechanism_create_orders.restype = I
        L.stev_mechanism_set_options.argtypes = [P, P]
        L.stev_mechanism_set_options.restype = I
        L.stev_mechanism_get_options.argtypes = [P, P]
        L.stev_mechanism_get_options.restype = I
        for name in ("stev_solve", "stev_solve_soa", "stev_solve_host", "stev_solve_host_noalloc"):
            f = getattr(L, name)
            f.argtypes = [P, LNG, P, P, P, D, P, P, P, P, P]
            f.restype = I
        L.stev_mlp_num_params.argtypes = [P]
        L.stev_mlp_num_params.restype = LNG
        L.stev_mlp_train.argtypes = [P, P, LNG, I, I, ctypes.c_float, ctypes.c_ulonglong, P]
        L.stev_mlp_train.restype = I
        L.stev_mlp_train_lm.argtypes = [P, P, LNG, I, I, D, I, ctypes.c_ulonglong, P]
        L.stev_mlp_train_lm.restype = I
        L.stev_mlp_jacobian.argtypes = [P, P, P, LNG, P]
        L.stev_mlp_jacobian.restype = I
        L.stev_mp_solve.argtypes = [LNG, P, D, P, P, P, P, P, P]
        L.stev_mp_solve.restype = I
        L.stev_gram_tf32.argtypes = [LNG, LNG, P, LNG, P, LNG, P]
        L.stev_gram_tf32.restype = I
        L.stev_damped_cg.argtypes = [LNG, P, LNG, P, ctypes.c_double, ctypes.c_double, P,
                                     I, ctypes.c_double, P, P]
        L.stev_damped_cg.restype = I
        L.stev_mlp_set_params.argtypes = [P, P, LNG, P, P]
        L.stev_mlp_set_params.restype = I
        L.stev_mlp_get_params.argtypes = [P, P, LNG, P, P]
        L.stev_mlp_get_params.restype = I
        L.stev_mlp_loss_grad.argtypes = [P, P, P, P, LNG, P, P]
        L.stev_mlp_loss_grad.restype = I
        L.stev_mlp_eval.argtypes = [P, P, LNG, P, P]
        L.stev_mlp_eval.restype = I
        L.stev_solve_batched.argtypes = [P, I, P, P, P, P, P, P, P, P, P, P]
        L.stev_solve_batched.restype = I
        L.stev_server_create.argtypes = [P, I, P, ctypes.c_size_t, I, P]
        L.stev_server_create.restype = I
        L.stev_server_submit.argtypes = [P, I, LNG, D, P, P, P, P, P, P, P, P]
        L.stev_server_submit.restype = I
        L.stev_server_poll.argtypes = [P, P, I, P, D]
        L.stev_server_poll.restype = I
        L.stev_server_get_stats.argtypes = [P, P]
        L.stev_server_get_stats.restype = I
        L.stev_server_clock.argtypes = [P]
        L.stev_server_clock.restype = D
        L.stev_server_stop.argtypes = [P, D]
        L.stev_server_stop.restype = I
        L.stev_server_destroy.argtypes = [P, D]
        L.stev_server_destroy.restype = I
        L.stev_mlp_stalls.argtypes = [P]
        L.stev_mlp_stalls.restype = ctypes.c_longlong
        L.stev_resident_slots.argtypes = [P]
        L.stev_resident_slots.restype = LNG
        L.stev_is_specialized.argtypes = [P]
        L.stev_is_specialized.restype = I
        L.stev_spec_compile_check.argtypes = [I, I, I, I, I, I, I, ctypes.c_char_p, ctypes.c_size_t]
        L.stev_spec_compile_check.restype = I
        L.stev_destroy.argtypes = [P]
        L.stev_destroy.restype = None
        L.stev_last_error.argtypes = []
        L.stev_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(code: int):
    if code != STEV_OK:
        raise StevError(code, lib().stev_last_error().decode())


def default_options(**overrides) -> Options:
    o = Options()
    lib().stev_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Mechanism:
    """A mechanism staged on the current CUDA device (stev_mechanism_create)."""

    def __init__(self, tables, **options):
        self._h = ctypes.c_void_p()
        self.S = int(np.asarray(tables.mol_weight).shape[0])
        self.R = int(np.asarray(tables.A).shape[0])
        keep = dict(
            W=_np(tables.mol_weight, np.float64), nasa7=_np(tables.nasa7, np.float64),
            t_range=_np(tables.t_range, np.float64), ptr=_np(tables.rxn_ptr, np.int32),
            sp=_np(tables.rxn_species, np.int32), nu=_np(tables.rxn_nu, np.float64),
            A=_np(tables.A, np.float64), beta=_np(tables.beta, np.float64),
            Ea=_np(tables.Ea, np.float64), rev=_np(tables.reversible, np.uint8))
        opt = default_options(**options)
        p = lambda a: a.ctypes.data
        order = getattr(tables, "rxn_order", None)
        if order is None:
            _check(lib().stev_mechanism_create(
                self.S, self.R, p(keep["W"]), p(keep["nasa7"]), p(keep["t_range"]),
                p(keep["ptr"]), p(keep["sp"]), p(keep["nu"]), p(keep["A"]), p(keep["beta"]),
                p(keep["Ea"]), p(keep["rev"]), ctypes.byref(opt), ctypes.byref(self._h)))
        else:   # global rate laws: real stoichiometry and orders
            keep["order"] = _np(order, np.float64)
            _check(lib().stev_mechanism_create_orders(
                self.S, self.R, p(keep["W"]), p(keep["nasa7"]), p(keep["t_range"]),
                p(keep["ptr"]), p(keep["sp"]), p(keep["nu"]), p(keep["order"]), p(keep["A"]),
                p(keep["beta"]), p(keep["Ea"]), p(keep["rev"]), ctypes.byref(opt),
                ctypes.byref(self._h)))

    # -- options ----------------------------------------------------------------
    @property
    def options(self) -> Options:
        o = Options()
        _check(lib().stev_mechanism_get_options(self._h, ctypes.byref(o)))
        return o

    def set_options(self, **changes):
        o = self.options
        for k, v in changes.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        _check(lib().stev_mechanism_set_options(self._h, ctypes.byref(o)))

    @property
    def mlp_stalls(self) -> int:
        """Network answers that timed out (the step took the polynomials); expected 0."""
        return int(lib().stev_mlp_stalls(self._h))

    @property
    def resident_slots(self) -> int:
        return int(lib().stev_resident_slots(self._h))

    @property
    def is_specialized(self) -> bool:
        """True when the solves run a kernel compiled for this mechanism."""
        return bool(lib().stev_is_specialized(self._h))

    # -- device entry points ----------------------------------------------------
    def _check_dev(self, T, P, Y, soa):
        import torch
        n = T.shape[0]
        for name, t in (("T", T), ("P", P), ("Y", Y)):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)
        if P.shape != (n,) or T.shape != (n,):
            raise ValueError("T and P must have shape [n_cells]")
        if Y.shape != ((self.S, n) if soa else (n, self.S)):
            raise ValueError("Y has the wrong shape")
        return n

    def solve(self, T, P, Y, dt: float, out=None, stream=None, soa: bool = False):
        """Device solve (stev_solve, or stev_solve_soa when soa=True).

        T, P: [n] float64 CUDA tensors; Y: [n][S] (or [S][n] with soa=True).
        Returns (T_out, Y_out, iters, status) CUDA tensors; asynchronous on
        `stream` (default: torch's current stream)."""
        import torch
        n = self._check_dev(T, P, Y, soa)
        if out is None:
            out = (torch.empty_like(T), torch.empty_like(Y),
                   torch.empty(n, dtype=torch.int32, device=T.device),
                   torch.empty(n, dtype=torch.uint8, device=T.device))
        To, Yo, it, st = out
        fn = lib().stev_solve_soa if soa else lib().stev_solve
        _check(fn(self._h, n, T.data_ptr(), P.data_ptr(), Y.data_ptr(), float(dt), To.data_ptr(),
                  Yo.data_ptr(), it.data_ptr(), st.data_ptr(), _stream_handle(stream)))
        return To, Yo, it, st

    def solve_batched(self, batches, dt, stream=None):
        """Independent batches in one launch (stev_solve_batched).

        batches: list of (T, P, Y) CUDA tensors; dt: one float or one per batch.
        Returns a list of (T_out, Y_out, iters, status) per batch."""
        import torch
        nb = len(batches)
        dts = np.full(nb, float(dt)) if np.isscalar(dt) else _np(dt, np.float64)
        outs, keep = [], []
        arr = lambda vals: (ctypes.c_void_p * max(nb, 1))(*vals)
        ptrs = {k: [] for k in ("T", "P", "Y", "To", "Yo", "it", "st")}
        sizes = np.zeros(nb, dtype=np.int64)
        for b, (T, P, Y) in enumerate(batches):
            n = self._check_dev(T, P, Y, False)
            sizes[b] = n
            o = (torch.empty_like(T), torch.empty_like(Y),
                 torch.empty(n, dtype=torch.int32, device=T.device),
                 torch.empty(n, dtype=torch.uint8, device=T.device))
            outs.append(o)
            for k, t in zip(("T", "P", "Y", "To", "Yo", "it", "st"), (T, P, Y) + o):
                ptrs[k].append(t.data_ptr())
        c = {k: arr(v) for k, v in ptrs.items()}
        _check(lib().stev_solve_batched(self._h, nb, sizes.ctypes.data, c["T"], c["P"], c["Y"],
                                        dts.ctypes.data, c["To"], c["Yo"], c["it"], c["st"],
                                        _stream_handle(stream)))
        return outs

    def solve_host(self, T, P, Y, dt: float, out=None, stream=None):
        """Host-pointer solve (stev_solve_host): numpy in, numpy out, blocking."""
        T, P, Y = _np(T, np.float64), _np(P, np.float64), _np(Y, np.float64)
        n = T.shape[0]
        if P.shape != (n,) or Y.shape != (n, self.S):
            raise ValueError("bad shapes")
        if out is None:
            out = (np.empty(n), np.empty((n, self.S)), np.empty(n, np.int32), np.empty(n, np.uint8))
        To, Yo, it, st = out
        h = 0 if stream is None else _stream_handle(stream)
        _check(lib().stev_solve_host(self._h, n, T.ctypes.data, P.ctypes.data, Y.ctypes.data,
                                     float(dt), To.ctypes.data, Yo.ctypes.data, it.ctypes.data,
                                     st.ctypes.data, h))
        return To, Yo, it, st

    # -- thermo network (Sec. 3) --------------------------------------------
    @property
    def mlp_num_params(self) -> int:
        return int(lib().stev_mlp_num_params(self._h))

    def mlp_train(self, T_samples, epochs: int = 30, batch: int = 4096, lr: float = 1e-3,
                  seed: int = 0):
        """Trains the thermo network on the GPU; returns the loss of every epoch."""
        T = _np(T_samples, np.float64)
        hist = np.zeros(epochs, np.float32)
        _check(lib().stev_mlp_train(self._h, T.ctypes.data, len(T), int(epochs), int(batch),
                                    float(lr), int(seed), hist.ctypes.data))
        return hist

    def mlp_train_lm(self, T_samples, iterations: int = 50, batch: int = 512,
                     lambda0: float = 1e-2, init: int = 0, seed: int = 0):
        """Levenberg-Marquardt training (stev_mlp_train_lm); returns the loss of
        every iteration."""
        T = _np(T_samples, np.float64)
        hist = np.zeros(iterations, np.float32)
        _check(lib().stev_mlp_train_lm(self._h, T.ctypes.data, len(T), int(iterations),
                                       int(batch), float(lambda0), int(init), int(seed),
                                       hist.ctypes.data))
        return hist

    def mlp_jacobian(self, params, T):
        """d(standardised outputs)/d(params) at host temperatures: [n*3S][n_params]."""
        p, Tn = _np(params, np.float32), _np(T, np.float64)
        J = np.zeros((len(Tn) * 3 * self.S, len(p)), np.float32)
        _check(lib().stev_mlp_jacobian(self._h, p.ctypes.data, Tn.ctypes.data, len(Tn),
                                       J.ctypes.data))
        return J

    def mlp_params(self):
        """(flat float32 parameters, mean [3S], std [3S])."""
        n = self.mlp_num_params
        p, mu, sd = np.zeros(n, np.float32), np.zeros(3 * self.S, np.float32), \
            np.zeros(3 * self.S, np.float32)
        _check(lib().stev_mlp_get_params(self._h, p.ctypes.data, n, mu.ctypes.data,
                                         sd.ctypes.data))
        return p, mu, sd

    def mlp_set_params(self, params, mean, std):
        p, mu, sd = _np(params, np.float32), _np(mean, np.float32), _np(std, np.float32)
        _check(lib().stev_mlp_set_params(self._h, p.ctypes.data, len(p), mu.ctypes.data,
                                         sd.ctypes.data))

    def mlp_loss_grad(self, params, T, target):
        """(loss, gradient) of the network on standardised targets, host arrays."""
        p, Tn, tg = _np(params, np.float32), _np(T, np.float64), _np(target, np.float32)
        g = np.zeros(len(p), np.float32)
        loss = ctypes.c_double(0.0)
        _check(lib().stev_mlp_loss_grad(self._h, p.ctypes.data, Tn.ctypes.data, tg.ctypes.data,
                                        len(Tn), g.ctypes.data, ctypes.addressof(loss)))
        return loss.value, g

    def mlp_eval(self, T, stream=None):
        """Network values [n][3S] (cp/R, H/RT, S/R) at CUDA float64 temperatures."""
        import torch
        out = torch.empty((T.shape[0], 3 * self.S), dtype=torch.float32, device=T.device)
        _check(lib().stev_mlp_eval(self._h, T.data_ptr(), T.shape[0], out.data_ptr(),
                                   _stream_handle(stream)))
        return out

    def close(self):
        if self._h:
            lib().stev_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_ptr(a):
    """Address of a contiguous host array (numpy array or CPU torch tensor)."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("host arrays must be contiguous")
        return a.ctypes.data
    if getattr(a, "is_cuda", False) or not a.is_contiguous():
        raise ValueError("host arrays must be contiguous CPU tensors")
    return a.data_ptr()


class Server:
    """Continuous-batching solve server (stev_server_*).

    mechanisms: Mechanism objects (kept alive by the server); sm_share: SMs per
    mechanism (None = even split); mem_budget: bytes of the device arena;
    queue_len: request slots per mechanism (0 = library default)."""

    def __init__(self, mechanisms, sm_share=None, mem_budget: int = 1 << 30,
                 queue_len: int = 0):
        self.mechanisms = list(mechanisms)
        self._h = ctypes.c_void_p()
        hs = (ctypes.c_void_p * len(self.mechanisms))(*[m._h.value for m in self.mechanisms])
        share = None
        if sm_share is not None:
            share = (ctypes.c_int * len(self.mechanisms))(*[int(x) for x in sm_share])
        _check(lib().stev_server_create(hs, len(self.mechanisms), share, int(mem_budget),
                                        int(queue_len), ctypes.byref(self._h)))
        self._live = {}

    def submit(self, mech: int, T, P, Y, dt: float, out=None) -> int:
        """Queues a request (host arrays; pinned memory copies asynchronously).
        out = (T_out, Y_out, iters, status) host arrays, allocated if None.
        The arrays are held until poll() reports the request."""
        S = self.mechanisms[mech].S
        n = int(T.shape[0])
        if tuple(P.shape) != (n,) or tuple(Y.shape) != (n, S):
            raise ValueError("bad shapes")
        if out is None:
            out = (np.empty(n), np.empty((n, S)), np.empty(n, np.int32), np.empty(n, np.uint8))
        rid = ctypes.c_longlong(-1)
        ptrs = [_host_ptr(a) for a in (T, P, Y) + tuple(out)]
        _check(lib().stev_server_submit(self._h, int(mech), n, float(dt), *ptrs,
                                        ctypes.byref(rid)))
        self._live[rid.value] = ((T, P, Y), out)
        return rid.value

    def poll(self, timeout: float = 0.0, max_done: int = 1024):
        """Finished requests: a list of dicts (id, mechanism, status, n_cells,
        t_submit, t_admit, t_done, out=(T_out, Y_out, iters, status))."""
        buf = (RequestInfo * max_done)()
        k = ctypes.c_int(0)
        _check(lib().stev_server_poll(self._h, buf, max_done, ctypes.byref(k), float(timeout)))
        res = []
        for i in range(k.value):
            r = buf[i]
            d = {f: getattr(r, f) for f, _ in RequestInfo._fields_}
            d["out"] = self._live.pop(r.id, (None, None))[1]
            res.append(d)
        return res

    @property
    def stats(self):
        st = ServerStats()
        _check(lib().stev_server_get_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    def clock(self) -> float:
        return float(lib().stev_server_clock(self._h))

    def stop(self, timeout: float = 30.0):
        """Stops serving (stev_server_stop); poll() still returns every report,
        cancelled requests with status STEV_EINCOMPLETE and their cells_done."""
        _check(lib().stev_server_stop(self._h, float(timeout)))

    def close(self, timeout: float = 30.0):
        """Stops the server (stev_server_destroy); poll() first for reports."""
        if not self._h:
            return
        code = lib().stev_server_destroy(self._h, float(timeout))
        msg = lib().stev_last_error().decode()
        self._h = ctypes.c_void_p()
        self._live.clear()
        if code != STEV_OK:
            raise StevError(code, msg)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mp_solve(cells, dt: float, out=None, stream=None, **options):
    """Multiphase coal gasification cells (stev_mp_solve, Sec. 7.2): cells is a
    CUDA float64 tensor [n][24]; returns (cells_out, rho_g, iters, status)."""
    import torch
    n = int(cells.shape[0])
    if tuple(cells.shape) != (n, 24) or cells.dtype != torch.float64 or not cells.is_cuda:
        raise ValueError("cells must be a CUDA float64 tensor of shape [n, 24]")
    cells = cells.contiguous()
    if out is None:
        out = (torch.empty_like(cells), torch.empty(n, dtype=torch.float64, device=cells.device),
               torch.empty(n, dtype=torch.int32, device=cells.device),
               torch.empty(n, dtype=torch.uint8, device=cells.device))
    o = default_options(**options)
    _check(lib().stev_mp_solve(n, cells.data_ptr(), float(dt), ctypes.byref(o), out[0].data_ptr(),
                               out[1].data_ptr(), out[2].data_ptr(), out[3].data_ptr(),
                               _stream_handle(stream)))
    return out


def gram_tf32(X, k: Optional[int] = None, stream=None):
    """G = X X^T (stev_gram_tf32) for a CUDA float32 tensor X [n][ldx] (the
    first k columns; ldx a multiple of 4): TF32 tensor-core products, FP32
    accumulation.  Returns G [n][n] (torch, on X's device)."""
    import torch
    n, ldx = int(X.shape[0]), int(X.shape[1])
    k = ldx if k is None else int(k)
    G = torch.empty((n, n), dtype=torch.float32, device=X.device)
    _check(lib().stev_gram_tf32(n, k, X.data_ptr(), ldx, G.data_ptr(), n, _stream_handle(stream)))
    return G


def damped_cg(A, b, lam: float = 0.0, eps: float = 0.0, max_iters: int = 1000,
              rtol: float = 1e-6, stream=None):
    """Solves (A + lam diag(A) + eps I) x = b (stev_damped_cg) for CUDA float32
    tensors A [n][n] (symmetric) and b [n]; returns (x, iterations)."""
    import torch
    n = int(A.shape[0])
    x = torch.empty(n, dtype=torch.float32, device=A.device)
    it = ctypes.c_int(0)
    _check(lib().stev_damped_cg(n, A.data_ptr(), int(A.stride(0)), b.data_ptr(), float(lam),
                                float(eps), x.data_ptr(), int(max_iters), float(rtol),
                                ctypes.byref(it), _stream_handle(stream)))
    return x, it.value


def spec_compile_check(n_species: int, n_reactions: int, n_reversible: int, general: bool = False,
                       lanes_per_cell: int = 32, dft_n: int = 13, network: bool = False) -> str:
    """Compiles the per-mechanism kernel for these sizes (no GPU needed) and
    returns NVRTC's log; raises StevError if it does not compile."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib().stev_spec_compile_check(int(n_species), int(n_reactions), int(n_reversible),
                                         int(bool(general)), int(lanes_per_cell), int(dft_n),
                                         int(bool(network)), buf, len(buf)))
    return buf.value.decode(errors="replace")
