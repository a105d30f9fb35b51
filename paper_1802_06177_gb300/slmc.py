"""Thin ctypes binding of libslmc (include/slmc.h). Argument marshalling only: every step
of the computation runs in the library's CUDA kernels. Arrays are torch CUDA tensors;
torch provides device memory and the current stream. There is no CPU fallback: if the
library is missing or fails to load, every call raises."""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libslmc.so")

PRECISION = {"fp64": 0, "fp32": 1, "tf32x3": 2, "bf16x9": 3}
STATUS = {0: "ok", 1: "invalid argument", 2: "non-finite input or result", 3: "CUDA runtime error",
          4: "bounded device wait timed out", 5: "unsupported shape or mode", 6: "out of device memory",
          7: "singular matrix"}


class SlmcError(RuntimeError):
    def __init__(self, fn, status):
        super().__init__("%s failed: %s (status %d)" % (fn, STATUS.get(status, "unknown"), status))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("L", ctypes.c_int), ("dtau", ctypes.c_double),
                ("t", ctypes.c_double), ("mu", ctypes.c_double), ("omega0", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("n_s", ctypes.c_int), ("precision", ctypes.c_int),
                ("sweep_delta", ctypes.c_double), ("seed", ctypes.c_uint64), ("qr_mode", ctypes.c_int)]

QR_MODE = {"prepivot": 0, "pivoted": 1}


EXPORTS = ("slmc_status_string", "slmc_init", "slmc_destroy", "slmc_get_error", "slmc_logdet", "slmc_greens",
           "slmc_log_weight", "slmc_eff_features", "slmc_eff_log_weight", "slmc_eff_sweep", "slmc_chain_init",
           "slmc_cumulative_update", "slmc_fit_eff", "slmc_measure_cdw", "slmc_launch_count", "slmc_profile_enable",
           "slmc_profile_read", "slmc_logdet_noalloc", "slmc_logdet_noalloc_scratch_bytes", "slmc_set_update_counter",
           "slmc_get_update_counter", "slmc_set_tuning", "slmc_batch_create", "slmc_batch_destroy",
           "slmc_batch_context", "slmc_batch_bind", "slmc_batch_capture", "slmc_batch_launch", "slmc_autotune",
           "slmc_batch_set_sweep_queue", "slmc_batch_inject_stall", "slmc_set_qr_path",
           "slmc_fit_eff_state", "slmc_fit_eff_merge", "slmc_profile_read_detail",
           "slmc_set_sub_batches", "slmc_set_slice_groups",
           "slmc_set_sub_batch_priorities", "slmc_set_qr_cluster", "slmc_set_wolff", "slmc_get_wolff_sites",
           "slmc_dqmc_sweep", "slmc_set_dense_slices", "slmc_set_tupdate_path")

UPDATE_CONTINUE = (1 << 64) - 1
FIT_STATE_DOUBLES = 64


class TuneResult(ctypes.Structure):
    _fields_ = [("n_s", ctypes.c_int), ("qr_panel", ctypes.c_int), ("slice_cols", ctypes.c_int),
                ("sec_per_eval", ctypes.c_double), ("max_abs_dlndet", ctypes.c_double), ("candidates", ctypes.c_int)]

PROF_CLASSES = ("slice", "qr", "formq", "tupdate", "final", "greens", "sweep", "eff", "bose", "accept", "fit", "cdw",
                "wolff", "dqmc", "qrtc")

_lib = None


def load_library(path=LIB_PATH):
    """Loads libslmc.so and declares the argument types of every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libslmc.so not found at %s: build it with `python -c \"import __graft_entry__ as g; "
                           "g.build()\"` (there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    P, I, D, U64, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p
    sig = {
        "slmc_status_string": ([I], ctypes.c_char_p),
        "slmc_init": ([ctypes.POINTER(Params), I, ctypes.POINTER(P)], I),
        "slmc_destroy": ([P], I),
        "slmc_get_error": ([P, V], I),
        "slmc_logdet": ([P, P, I, P, P, V], I),
        "slmc_greens": ([P, P, I, P, P, P, V], I),
        "slmc_log_weight": ([P, P, I, P, P, P, V], I),
        "slmc_eff_features": ([P, P, I, P, V], I),
        "slmc_eff_log_weight": ([P, P, I, P, P, V], I),
        "slmc_eff_sweep": ([P, P, I, P, I, U64, I, P, V], I),
        "slmc_chain_init": ([P, P, I, P, P, V], I),
        "slmc_cumulative_update": ([P, P, I, P, I, I, U64, P, P, P, P, P, V], I),
        "slmc_fit_eff": ([P, P, P, I, P, P, V], I),
        "slmc_measure_cdw": ([P, P, I, P, V], I),
        "slmc_launch_count": ([P], ctypes.c_longlong),
        "slmc_profile_enable": ([P, I], I),
        "slmc_profile_read": ([P, P, P, V], I),
        "slmc_logdet_noalloc": ([ctypes.POINTER(Params), P, I, P, P, V], I),
        "slmc_logdet_noalloc_scratch_bytes": ([], ctypes.c_size_t),
        "slmc_set_update_counter": ([P, U64, V], I),
        "slmc_get_update_counter": ([P, ctypes.POINTER(ctypes.c_uint64), V], I),
        "slmc_set_tuning": ([P, I, I], I),
        "slmc_batch_create": ([ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_int), I, ctypes.POINTER(P)], I),
        "slmc_batch_destroy": ([P], I),
        "slmc_batch_context": ([P, I], P),
        "slmc_batch_bind": ([P, I, P, P, P, P, P, P], I),
        "slmc_batch_capture": ([P, I, I, V], I),
        "slmc_batch_launch": ([P, I, V], I),
        "slmc_batch_set_sweep_queue": ([P, I], I),
        "slmc_batch_inject_stall": ([P, ctypes.c_longlong], I),
        "slmc_autotune": ([ctypes.POINTER(Params), I, D, ctypes.POINTER(TuneResult)], I),
        "slmc_fit_eff_state": ([P, P, P, I, P, V], I),
        "slmc_fit_eff_merge": ([P, P, I, P, P, V], I),
        "slmc_profile_read_detail": ([P, P, P, P, P, V], I),
        "slmc_set_sub_batches": ([P, I], I),
        "slmc_set_slice_groups": ([P, I], I),
        "slmc_set_sub_batch_priorities": ([P, I], I),
        "slmc_set_qr_cluster": ([P, I], I),
        "slmc_set_dense_slices": ([P, I], I),
        "slmc_set_tupdate_path": ([P, I], I),
        "slmc_set_qr_path": ([P, I], I),
        "slmc_set_wolff": ([P, I], I),
        "slmc_get_wolff_sites": ([P, ctypes.POINTER(ctypes.c_longlong), I, V], I),
        "slmc_dqmc_sweep": ([P, P, I, I, U64, I, P, P, V], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(t, dtype, name, shape=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return t.data_ptr()


def _stream(device):
    return torch.cuda.current_stream(device).cuda_stream


class Context:
    """One libslmc context (model parameters, exp(-dtau K), workspace) on one CUDA device."""

    def __init__(self, Lx, Ly, L, dtau=0.1, t=1.0, mu=0.0, omega0=1.0, lam=1.0, n_s=10, precision="fp64",
                 sweep_delta=0.5, seed=0, max_fields=64, device=None, qr_mode="prepivot"):
        self.lib = load_library()
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.device = torch.device("cuda", torch.cuda.current_device() if dev.index is None else dev.index)
        self.Lx, self.Ly, self.L = Lx, Ly, L
        self.N = Lx * Ly
        self.dtau, self.lam, self.omega0, self.n_s = dtau, lam, omega0, n_s
        self.precision = precision
        self.params = Params(Lx, Ly, L, dtau, t, mu, omega0, lam, n_s, PRECISION[precision], sweep_delta,
                             seed & ((1 << 64) - 1), QR_MODE[qr_mode])
        self._ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            self._check("slmc_init", self.lib.slmc_init(ctypes.byref(self.params), max_fields,
                                                        ctypes.byref(self._ctx)))

    # -- helpers -----------------------------------------------------------------------
    def _check(self, fn, status):
        if status != 0:
            raise SlmcError(fn, status)

    def _fields(self, x, name="x"):
        if x.dim() != 3 or x.shape[1] != self.N or x.shape[2] != self.L:
            raise ValueError("%s must have shape [n, %d, %d]" % (name, self.N, self.L))
        return _ptr(x, torch.float64, name), x.shape[0]

    def _empty(self, shape, dtype=torch.float64):
        return torch.empty(shape, dtype=dtype, device=self.device)

    def close(self):
        if self._ctx:
            self.lib.slmc_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_error(self):
        """Synchronises the current stream and raises if a kernel flagged an error."""
        self._check("slmc_get_error", self.lib.slmc_get_error(self._ctx, _stream(self.device)))

    # -- entry points ------------------------------------------------------------------
    def logdet(self, x, lndet=None, sign=None):
        px, n = self._fields(x)
        lndet = self._empty(n) if lndet is None else lndet
        sign = self._empty(n, torch.int32) if sign is None else sign
        self._check("slmc_logdet", self.lib.slmc_logdet(self._ctx, px, n, _ptr(lndet, torch.float64, "lndet", (n,)),
                                                        _ptr(sign, torch.int32, "sign", (n,)), _stream(self.device)))
        return lndet, sign

    def greens(self, x, G=None, lndet=None, sign=None):
        px, n = self._fields(x)
        G = self._empty((n, self.N, self.N)) if G is None else G
        lndet = self._empty(n) if lndet is None else lndet
        sign = self._empty(n, torch.int32) if sign is None else sign
        self._check("slmc_greens", self.lib.slmc_greens(
            self._ctx, px, n, _ptr(G, torch.float64, "G", (n, self.N, self.N)),
            _ptr(lndet, torch.float64, "lndet", (n,)), _ptr(sign, torch.int32, "sign", (n,)), _stream(self.device)))
        return G, lndet, sign

    def log_weight(self, x):
        px, n = self._fields(x)
        lnw, lndet, sign = self._empty(n), self._empty(n), self._empty(n, torch.int32)
        self._check("slmc_log_weight", self.lib.slmc_log_weight(self._ctx, px, n, _ptr(lnw, torch.float64, "lnw"),
                                                                _ptr(lndet, torch.float64, "lndet"),
                                                                _ptr(sign, torch.int32, "sign"), _stream(self.device)))
        return lnw, lndet, sign

    def eff_features(self, x):
        px, n = self._fields(x)
        F = self._empty((n, 5))
        self._check("slmc_eff_features", self.lib.slmc_eff_features(self._ctx, px, n, _ptr(F, torch.float64, "F"),
                                                                    _stream(self.device)))
        return F

    def eff_log_weight(self, x, J):
        px, n = self._fields(x)
        out = self._empty(n)
        self._check("slmc_eff_log_weight", self.lib.slmc_eff_log_weight(
            self._ctx, px, n, _ptr(J, torch.float64, "J", (6,)), _ptr(out, torch.float64, "out"), _stream(self.device)))
        return out

    def eff_sweep(self, x, J, nsweeps, sweep0=0, first_colour=0, n_acc=None):
        px, n = self._fields(x)
        self._check("slmc_eff_sweep", self.lib.slmc_eff_sweep(
            self._ctx, px, n, _ptr(J, torch.float64, "J", (6,)), nsweeps, sweep0, first_colour,
            _ptr(n_acc, torch.int64, "n_acc", (n,)), _stream(self.device)))
        return x

    def dqmc_sweep(self, x, nsweeps, sweep0=0, nblock=0, n_acc_local=None, n_acc_block=None):
        """Conventional DQMC sweeps (local updates with fast ratios, then nblock block updates)."""
        px, n = self._fields(x)
        self._check("slmc_dqmc_sweep", self.lib.slmc_dqmc_sweep(
            self._ctx, px, n, nsweeps, sweep0, nblock, _ptr(n_acc_local, torch.int64, "n_acc_local", (n,)),
            _ptr(n_acc_block, torch.int64, "n_acc_block", (n,)), _stream(self.device)))
        return x

    def chain_init(self, x, want_cdw=True):
        px, n = self._fields(x)
        lnw = self._empty(n)
        s = self._empty(n) if want_cdw else None
        self._check("slmc_chain_init", self.lib.slmc_chain_init(self._ctx, px, n, _ptr(lnw, torch.float64, "lnw"),
                                                                _ptr(s, torch.float64, "s_cdw"), _stream(self.device)))
        return lnw, s

    def cumulative_update(self, x, J, nsweeps, nupdates, update0, lnw, s_cdw=None, n_acc=None, n_sweep_acc=None,
                          want_obs=False):
        px, n = self._fields(x)
        obs = self._empty((nupdates, n)) if want_obs else None
        self._check("slmc_cumulative_update", self.lib.slmc_cumulative_update(
            self._ctx, px, n, _ptr(J, torch.float64, "J", (6,)), nsweeps, nupdates, update0,
            _ptr(lnw, torch.float64, "lnw", (n,)), _ptr(s_cdw, torch.float64, "s_cdw", (n,)),
            _ptr(n_acc, torch.int64, "n_acc", (n,)), _ptr(n_sweep_acc, torch.int64, "n_sweep_acc", (n,)),
            _ptr(obs, torch.float64, "obs"), _stream(self.device)))
        return obs

    def fit_eff(self, xs, lnw):
        px, n = self._fields(xs, "xs")
        J = self._empty(6)
        resid = self._empty(1)
        self._check("slmc_fit_eff", self.lib.slmc_fit_eff(self._ctx, px, _ptr(lnw, torch.float64, "lnw", (n,)), n,
                                                          _ptr(J, torch.float64, "J"), _ptr(resid, torch.float64, "r"),
                                                          _stream(self.device)))
        return J, resid

    def fit_eff_state(self, xs, lnw):
        """Partial regression state [FIT_STATE_DOUBLES] of this process's configurations (Eq. (5))."""
        px, n = self._fields(xs, "xs")
        state = self._empty(FIT_STATE_DOUBLES)
        self._check("slmc_fit_eff_state", self.lib.slmc_fit_eff_state(
            self._ctx, px if n else None, _ptr(lnw, torch.float64, "lnw", (n,)) if n else None, n,
            _ptr(state, torch.float64, "state"), _stream(self.device)))
        return state

    def fit_eff_merge(self, states):
        """Couplings from partial states [nparts, FIT_STATE_DOUBLES] (all processes' states)."""
        if states.dim() != 2 or states.shape[1] != FIT_STATE_DOUBLES:
            raise ValueError("states must have shape [nparts, %d]" % FIT_STATE_DOUBLES)
        J = self._empty(6)
        resid = self._empty(1)
        self._check("slmc_fit_eff_merge", self.lib.slmc_fit_eff_merge(
            self._ctx, _ptr(states, torch.float64, "states"), states.shape[0], _ptr(J, torch.float64, "J"),
            _ptr(resid, torch.float64, "r"), _stream(self.device)))
        return J, resid

    def launch_count(self):
        """Kernels enqueued by this context so far."""
        return int(self.lib.slmc_launch_count(self._ctx))

    def profile(self, on=True):
        self._check("slmc_profile_enable", self.lib.slmc_profile_enable(self._ctx, 1 if on else 0))

    def profile_read(self):
        """{class: (total ms, timed calls)} of the event-timed launches since profile(True)."""
        return {k: v[:2] for k, v in self.profile_read_detail().items()}

    def profile_read_detail(self):
        """{class: (summed call ms, calls, busy ms = union of call intervals, fields processed)}."""
        n = len(PROF_CLASSES)
        ms = (ctypes.c_double * n)()
        calls = (ctypes.c_longlong * n)()
        busy = (ctypes.c_double * n)()
        units = (ctypes.c_longlong * n)()
        self._check("slmc_profile_read_detail", self.lib.slmc_profile_read_detail(
            self._ctx, ms, calls, busy, units, _stream(self.device)))
        return {k: (ms[q], calls[q], busy[q], units[q]) for q, k in enumerate(PROF_CLASSES)}

    def set_update_counter(self, value):
        self._check("slmc_set_update_counter", self.lib.slmc_set_update_counter(self._ctx, value, _stream(self.device)))

    def get_update_counter(self):
        v = ctypes.c_uint64()
        self._check("slmc_get_update_counter", self.lib.slmc_get_update_counter(self._ctx, ctypes.byref(v),
                                                                                _stream(self.device)))
        return v.value

    def set_tuning(self, qr_panel=0, slice_cols=0):
        self._check("slmc_set_tuning", self.lib.slmc_set_tuning(self._ctx, qr_panel, slice_cols))

    def set_slice_groups(self, groups):
        """Thread layout of the FP32 slice kernel (0 = default, 1, 2 or 4)."""
        self._check("slmc_set_slice_groups", self.lib.slmc_set_slice_groups(self._ctx, groups))

    def set_wolff(self, nwolff):
        """Wolff cluster updates between the two colours of every sweep (0 = local sweeps only)."""
        self._check("slmc_set_wolff", self.lib.slmc_set_wolff(self._ctx, nwolff))

    def wolff_sites(self, reset=False):
        """Columns reflected by Wolff updates so far (synchronises the current stream)."""
        v = ctypes.c_longlong()
        self._check("slmc_get_wolff_sites", self.lib.slmc_get_wolff_sites(self._ctx, ctypes.byref(v), 1 if reset else 0,
                                                                          _stream(self.device)))
        return v.value

    def set_qr_cluster(self, ctas):
        """CTAs per field of the QR and the formation of Q (0 = automatic, 1, 2 or 4)."""
        self._check("slmc_set_qr_cluster", self.lib.slmc_set_qr_cluster(self._ctx, ctas))

    def set_dense_slices(self, dense):
        """FP64 mode: 1 = dense exp(-dtau K) slice products; 0 (default) = through its separable factors."""
        self._check("slmc_set_dense_slices", self.lib.slmc_set_dense_slices(self._ctx, int(dense)))

    def set_tupdate_path(self, path):
        """0: T update on the tensor cores (exact slices, FP64-accurate); 1: FP64 FMAs; 2: the
        tensor kernel with every tile on its FP64 fallback."""
        self._check("slmc_set_tupdate_path", self.lib.slmc_set_tupdate_path(self._ctx, int(path)))


    def set_qr_path(self, path):
        """slmc_set_qr_path: 0 = QR trailing updates on the tensor cores (FP64-accurate sliced
        BF16), 1 = the one-kernel FP64 QR."""
        self._check("slmc_set_qr_path", self.lib.slmc_set_qr_path(self._ctx, path))
    def set_sub_batch_priorities(self, on):
        """Descending stream priorities for the sub-batches (1) or equal priorities (0)."""
        self._check("slmc_set_sub_batch_priorities", self.lib.slmc_set_sub_batch_priorities(self._ctx, 1 if on else 0))

    def set_sub_batches(self, n):
        """Sub-batches (forked streams) a large determinant batch is split into (1..4)."""
        self._check("slmc_set_sub_batches", self.lib.slmc_set_sub_batches(self._ctx, n))

    def measure_cdw(self, G):
        n = G.shape[0]
        S = self._empty(n)
        self._check("slmc_measure_cdw", self.lib.slmc_measure_cdw(
            self._ctx, _ptr(G, torch.float64, "G", (n, self.N, self.N)), n, _ptr(S, torch.float64, "S"),
            _stream(self.device)))
        return S


class _BorrowedContext(Context):
    """A context owned by a Batch (not destroyed by this wrapper)."""

    def __init__(self, handle, Lx, Ly, L, device):
        self.lib = load_library()
        self._ctx = ctypes.c_void_p(handle)
        self.device = device
        self.Lx, self.Ly, self.L, self.N = Lx, Ly, L, Lx * Ly

    def close(self):
        self._ctx = ctypes.c_void_p()


class Batch:
    """Chains of several lattice classes advanced together through one captured CUDA graph
    (slmc_batch_*). classes: list of dicts of Context keyword arguments plus "nchains"."""

    def __init__(self, classes, device=None):
        self.lib = load_library()
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.device = torch.device("cuda", torch.cuda.current_device() if dev.index is None else dev.index)
        n = len(classes)
        arr = (Params * n)()
        nch = (ctypes.c_int * n)()
        self.shapes = []
        for q, cl in enumerate(classes):
            arr[q] = Params(cl["Lx"], cl.get("Ly", cl["Lx"]), cl["L"], cl.get("dtau", 0.1), cl.get("t", 1.0),
                            cl.get("mu", 0.0), cl.get("omega0", 1.0), cl.get("lam", 1.0), cl.get("n_s", 10),
                            PRECISION[cl.get("precision", "fp64")], cl.get("sweep_delta", 0.5),
                            cl.get("seed", 0) & ((1 << 64) - 1), QR_MODE[cl.get("qr_mode", "prepivot")])
            nch[q] = cl["nchains"]
            self.shapes.append((cl["Lx"], cl.get("Ly", cl["Lx"]), cl["L"], cl["nchains"]))
        self._b = ctypes.c_void_p()
        self._keep = []
        self.stream = torch.cuda.Stream(device=self.device)
        with torch.cuda.device(self.device):
            st = self.lib.slmc_batch_create(arr, nch, n, ctypes.byref(self._b))
        if st != 0:
            raise SlmcError("slmc_batch_create", st)

    def context(self, cls):
        Lx, Ly, L, _ = self.shapes[cls]
        return _BorrowedContext(self.lib.slmc_batch_context(self._b, cls), Lx, Ly, L, self.device)

    def bind(self, cls, x, J, lnw, s_cdw=None, n_acc=None, n_sweep_acc=None):
        Lx, Ly, L, nch = self.shapes[cls]
        self._keep.append((x, J, lnw, s_cdw, n_acc, n_sweep_acc))
        st = self.lib.slmc_batch_bind(self._b, cls, _ptr(x, torch.float64, "x", (nch, Lx * Ly, L)),
                                      _ptr(J, torch.float64, "J", (6,)), _ptr(lnw, torch.float64, "lnw", (nch,)),
                                      _ptr(s_cdw, torch.float64, "s_cdw", (nch,)), _ptr(n_acc, torch.int64, "n_acc", (nch,)),
                                      _ptr(n_sweep_acc, torch.int64, "n_sweep_acc", (nch,)))
        if st != 0:
            raise SlmcError("slmc_batch_bind", st)

    def capture(self, nsweeps, nupdates=1):
        st = self.lib.slmc_batch_capture(self._b, nsweeps, nupdates, self.stream.cuda_stream)
        if st != 0:
            raise SlmcError("slmc_batch_capture", st)

    def launch(self, nrounds=1):
        st = self.lib.slmc_batch_launch(self._b, nrounds, self.stream.cuda_stream)
        if st != 0:
            raise SlmcError("slmc_batch_launch", st)

    def set_sweep_queue(self, on):
        """slmc_batch_set_sweep_queue: the E_eff sweeps of every class in one persistent launch
        (on, the default) or as each class's kernel-per-half-sweep sequence; next capture."""
        st = self.lib.slmc_batch_set_sweep_queue(self._b, 1 if on else 0)
        if st != 0:
            raise SlmcError("slmc_batch_set_sweep_queue", st)

    def inject_stall(self, wait_cycles):
        """slmc_batch_inject_stall: test hook; the next capture's first queue item waits for a
        count nothing reaches and gives up after wait_cycles, setting SLMC_ERR_TIMEOUT."""
        st = self.lib.slmc_batch_inject_stall(self._b, int(wait_cycles))
        if st != 0:
            raise SlmcError("slmc_batch_inject_stall", st)

    def close(self):
        if self._b:
            self.lib.slmc_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(Lx, Ly, L, precision="fp32", ntune=32, tol=5e-5, qr_mode="prepivot", dtau=0.1, t=1.0, mu=0.0,
             omega0=1.0, lam=1.0, seed=0):
    """slmc_autotune: fastest (n_s, QR panel, FP32 tile) within tol of the FP64 path."""
    lib = load_library()
    p = Params(Lx, Ly, L, dtau, t, mu, omega0, lam, 8, PRECISION[precision], 0.0, seed, QR_MODE[qr_mode])
    r = TuneResult()
    st = lib.slmc_autotune(ctypes.byref(p), ntune, tol, ctypes.byref(r))
    if st != 0:
        raise SlmcError("slmc_autotune", st)
    return {"n_s": r.n_s, "qr_panel": r.qr_panel, "slice_cols": r.slice_cols, "sec_per_eval": r.sec_per_eval,
            "max_abs_dlndet": r.max_abs_dlndet, "candidates": r.candidates}


def logdet_noalloc(x, Lx, Ly, L, dtau=0.1, t=1.0, mu=0.0, omega0=1.0, lam=1.0, n_s=10, precision="fp64",
                   lndet=None, sign=None, qr_mode="prepivot"):
    """slmc_logdet_noalloc: ln|det| and sign of fields x[n, N, L] without a context and
    without any device allocation inside the library (its workspace is a fixed 16 MiB
    device array). Outputs may be passed in preallocated; errors show as NaN / sign 0."""
    lib = load_library()
    p = Params(Lx, Ly, L, dtau, t, mu, omega0, lam, n_s, PRECISION[precision], 0.0, 0, QR_MODE[qr_mode])
    n = x.shape[0]
    lndet = torch.empty(n, dtype=torch.float64, device=x.device) if lndet is None else lndet
    sign = torch.empty(n, dtype=torch.int32, device=x.device) if sign is None else sign
    st = lib.slmc_logdet_noalloc(ctypes.byref(p), _ptr(x, torch.float64, "x"), n,
                                 _ptr(lndet, torch.float64, "lndet", (n,)), _ptr(sign, torch.int32, "sign", (n,)),
                                 _stream(x.device))
    if st != 0:
        raise SlmcError("slmc_logdet_noalloc", st)
    return lndet, sign
