"""ctypes binding of the C ABI in include/fdph.h (argument marshalling only).

Every step of the method runs inside libfdph.so; this module only converts
Python / numpy / torch arguments to the plain pointers and sizes of the ABI.
Loading fails loudly if the library has not been built: there is no fallback.
Device buffers are anything with ``data_ptr()`` (a torch CUDA tensor) or a raw
integer address; they must hold float64 values, contiguous.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FDPH_LIB=check selects the bounded-index debug build (build.build(check=True))
LIB_PATH = os.path.join(_HERE, "libfdph_check.so" if os.environ.get("FDPH_LIB") == "check" else "libfdph.so")

OK, E_ARG, E_OOM, E_CAUSALITY, E_CUDA, E_TIMEOUT, E_NAN, E_STATE, E_CHECK = 0, -1, -2, -3, -4, -5, -6, -7, -8
FP64, FP32, FP16 = 0, 1, 2


class FdphError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("fdph status %d: %s" % (status, msg))
        self.status = status


class Geometry(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("xy", ctypes.POINTER(ctypes.c_double))]


class Material(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("cs", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("lmin", ctypes.c_double), ("eps_st", ctypes.c_double),
                ("leaf_size", ctypes.c_int32), ("extra_steps", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
                ("soe_terms", ctypes.c_int32), ("art_interp", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p),
                ("host_threads", ctypes.c_int32), ("eta_scheme", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("far_mode", ctypes.c_int32), ("amp_window", ctypes.c_int32), ("eps_q", ctypes.c_double),
                ("aca_min", ctypes.c_int64)]


class Friction(ctypes.Structure):
    _fields_ = [("tau0", ctypes.c_void_p), ("sigma_n", ctypes.c_double), ("mu_s", ctypes.c_double),
                ("mu_d", ctypes.c_double), ("Dc", ctypes.c_double), ("law", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("M", ctypes.c_int32), ("n_admissible", ctypes.c_int32),
                ("n_near", ctypes.c_int32), ("n_subblocks", ctypes.c_int32), ("max_rank", ctypes.c_int32),
                ("extra_steps", ctypes.c_int32), ("max_window", ctypes.c_int32),
                ("mean_rank", ctypes.c_double), ("near_entries", ctypes.c_int64),
                ("far_entries", ctypes.c_int64), ("arena_bytes", ctypes.c_int64),
                ("state_bytes", ctypes.c_int64), ("bytes_per_step", ctypes.c_double),
                ("near_bytes_per_step", ctypes.c_double), ("flops_per_step", ctypes.c_double),
                ("plan_seconds", ctypes.c_double), ("n_exact", ctypes.c_int32), ("n_aca", ctypes.c_int32),
                ("mean_rank_f", ctypes.c_double), ("mean_rank_s", ctypes.c_double), ("mean_rank_tr", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

EXPORTS = ["fdph_default_params", "fdph_plan", "fdph_step", "fdph_run", "fdph_step_host", "fdph_run_host", "fdph_reset",
           "fdph_current_step", "fdph_plan_stream", "fdph_synchronize", "fdph_get_stats", "fdph_save_state", "fdph_load_state",
           "fdph_destroy", "fdph_tree_export", "fdph_strerror", "fdph_last_error", "fdph_set_profiling",
           "fdph_kernel_times", "fdph_plain_step_noalloc", "fdph_rupture_init", "fdph_rupture_step",
           "fdph_rupture_run", "fdph_rupture_slip", "fdph_selftest_wait_timeout", "fdph_autotune",
           "fdph_predict", "fdph_commit", "fdph_self", "fdph_batch_create", "fdph_batch_run", "fdph_quantize",
           "fdph_batch_rupture_run", "fdph_batch_synchronize", "fdph_batch_destroy", "fdph_low_rank",
           "fdph_low_rank_aca", "fdph_kernel_tail"]
KERNEL_NAMES = ["push", "fir", "scatter", "trconv", "near", "gather"]


def lib():
    """The loaded libfdph.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libfdph.so is not built (run __graft_entry__.build() or "
                              "python paper_1903_02118_gb300/build.py); there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        c_p = ctypes.c_void_p
        L.fdph_default_params.argtypes = [ctypes.POINTER(Params)]
        L.fdph_default_params.restype = None
        L.fdph_plan.argtypes = [ctypes.POINTER(Geometry), ctypes.POINTER(Material), ctypes.c_double, ctypes.c_int32,
                                ctypes.c_double, ctypes.POINTER(Params), ctypes.POINTER(c_p)]
        L.fdph_step.argtypes = [c_p, c_p, c_p]
        L.fdph_run.argtypes = [c_p, ctypes.c_int32, c_p, c_p]
        L.fdph_step_host.argtypes = [c_p, c_p, c_p]
        L.fdph_run_host.argtypes = [c_p, ctypes.c_int32, c_p, c_p]
        L.fdph_reset.argtypes = [c_p]
        L.fdph_current_step.argtypes = [c_p, ctypes.POINTER(ctypes.c_int32)]
        L.fdph_plan_stream.argtypes = [c_p, ctypes.POINTER(c_p)]
        L.fdph_plan_stream.restype = ctypes.c_int
        L.fdph_synchronize.argtypes = [c_p]
        L.fdph_get_stats.argtypes = [c_p, ctypes.POINTER(Stats)]
        L.fdph_save_state.argtypes = [c_p, c_p, ctypes.POINTER(ctypes.c_size_t)]
        L.fdph_load_state.argtypes = [c_p, c_p, ctypes.c_size_t]
        L.fdph_destroy.argtypes = [c_p]
        L.fdph_destroy.restype = None
        L.fdph_tree_export.argtypes = [ctypes.POINTER(Geometry), ctypes.POINTER(Material), ctypes.c_double,
                                       ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                                       ctypes.POINTER(ctypes.c_int64)]
        L.fdph_set_profiling.argtypes = [c_p, ctypes.c_int]
        L.fdph_kernel_times.argtypes = [c_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        L.fdph_plain_step_noalloc.argtypes = [c_p, ctypes.c_int32, ctypes.c_int32, c_p, ctypes.c_int32,
                                              ctypes.c_int32, c_p, c_p]
        L.fdph_rupture_init.argtypes = [c_p, ctypes.POINTER(Friction)]
        L.fdph_rupture_step.argtypes = [c_p, c_p, c_p]
        L.fdph_rupture_run.argtypes = [c_p, ctypes.c_int32, c_p, c_p]
        L.fdph_rupture_slip.argtypes = [c_p, c_p]
        L.fdph_predict.argtypes = [c_p, c_p]
        L.fdph_commit.argtypes = [c_p, c_p]
        L.fdph_self.argtypes = [c_p, c_p]
        L.fdph_batch_create.argtypes = [ctypes.POINTER(c_p), ctypes.c_int32, ctypes.POINTER(c_p)]
        L.fdph_batch_run.argtypes = [c_p, ctypes.c_int32, ctypes.POINTER(c_p), ctypes.POINTER(c_p)]
        L.fdph_batch_rupture_run.argtypes = [c_p, ctypes.c_int32, ctypes.POINTER(c_p), ctypes.POINTER(c_p)]
        L.fdph_batch_synchronize.argtypes = [c_p]
        L.fdph_batch_destroy.argtypes = [c_p]
        L.fdph_batch_destroy.restype = None
        L.fdph_low_rank.argtypes = [c_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, c_p, c_p,
                                    ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        L.fdph_low_rank.restype = ctypes.c_int
        L.fdph_low_rank_aca.argtypes = [c_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, c_p, c_p,
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int64)]
        L.fdph_low_rank_aca.restype = ctypes.c_int
        L.fdph_kernel_tail.argtypes = [c_p, c_p, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       c_p]
        L.fdph_kernel_tail.restype = ctypes.c_int
        L.fdph_quantize.argtypes = [c_p, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(ctypes.c_int32), c_p,
                                    ctypes.POINTER(ctypes.c_int32)]
        L.fdph_quantize.restype = ctypes.c_int
        L.fdph_autotune.argtypes = [c_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        L.fdph_autotune.restype = ctypes.c_int
        L.fdph_selftest_wait_timeout.argtypes = [ctypes.c_int32, ctypes.c_int64]
        L.fdph_selftest_wait_timeout.restype = ctypes.c_int
        L.fdph_strerror.argtypes = [ctypes.c_int]
        L.fdph_strerror.restype = ctypes.c_char_p
        L.fdph_last_error.argtypes = []
        L.fdph_last_error.restype = ctypes.c_char_p
        for name in ("fdph_plan", "fdph_step", "fdph_run", "fdph_step_host", "fdph_run_host", "fdph_reset",
                     "fdph_current_step",
                     "fdph_synchronize", "fdph_get_stats", "fdph_save_state", "fdph_load_state",
                     "fdph_tree_export", "fdph_set_profiling", "fdph_kernel_times", "fdph_plain_step_noalloc",
                     "fdph_rupture_init", "fdph_rupture_step", "fdph_rupture_run", "fdph_rupture_slip",
                     "fdph_predict", "fdph_commit", "fdph_self", "fdph_batch_create", "fdph_batch_run", "fdph_quantize",
                     "fdph_batch_rupture_run", "fdph_batch_synchronize"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        L = lib()
        raise FdphError(rc, "%s (%s)" % (L.fdph_strerror(rc).decode(), L.fdph_last_error().decode()))


def _ptr(x):
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(int(x))


def selftest_wait_timeout(device=0, polls=1000):
    """Status of fdph_selftest_wait_timeout (E_TIMEOUT when the bounded-wait path works)."""
    return lib().fdph_selftest_wait_timeout(int(device), int(polls))


def default_params():
    p = Params()
    lib().fdph_default_params(ctypes.byref(p))
    return p


def make_params(eta=None, lmin=None, eps_st=None, leaf_size=None, extra_steps=None, precision=None,
                device=None, stream=None, soe_terms=None, art_interp=None, host_threads=None, eta_scheme=None,
                nrhs=None, far_mode=None, amp_window=None, eps_q=None, aca_min=None):
    p = default_params()
    for k, v in (("eta", eta), ("lmin", lmin), ("eps_st", eps_st), ("leaf_size", leaf_size),
                 ("extra_steps", extra_steps), ("precision", precision), ("device", device),
                 ("host_threads", host_threads), ("eta_scheme", eta_scheme), ("nrhs", nrhs), ("far_mode", far_mode),
                 ("amp_window", amp_window), ("eps_q", eps_q), ("aca_min", aca_min),
                 ("soe_terms", soe_terms), ("art_interp", None if art_interp is None else int(bool(art_interp)))):
        if v is not None:
            setattr(p, k, v)
    if stream is not None:
        p.cuda_stream = ctypes.c_void_p(stream)
    return p


def _geometry(xy):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    g = Geometry(xy.shape[0], xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return g, xy


class Plan:
    """Owner of an fdph_plan_t (see fdph_plan in include/fdph.h)."""

    def __init__(self, xy, dt, M, eps, mu=1.0, cs=1.0, **params):
        L = lib()
        g, self._xy = _geometry(xy)
        mat = Material(mu, cs)
        p = make_params(**params)
        h = ctypes.c_void_p()
        _check(L.fdph_plan(ctypes.byref(g), ctypes.byref(mat), dt, M, eps, ctypes.byref(p), ctypes.byref(h)))
        self.handle = h
        self.n = int(xy.shape[0])
        self.M = int(M)
        self.precision = int(p.precision)
        self.nrhs = max(int(p.nrhs), 1)

    def step(self, D_n, T_n):
        _check(lib().fdph_step(self.handle, _ptr(D_n), _ptr(T_n)))

    def run(self, steps, D, T):
        _check(lib().fdph_run(self.handle, int(steps), _ptr(D), _ptr(T)))

    def step_host(self, D_n, T_n=None):
        D_n = np.ascontiguousarray(D_n, dtype=np.float64)
        if T_n is None:
            T_n = np.empty(self.n * self.nrhs)
        _check(lib().fdph_step_host(self.handle, ctypes.c_void_p(D_n.ctypes.data), ctypes.c_void_p(T_n.ctypes.data)))
        return T_n

    def run_host(self, D, T=None):
        """Steps D.shape[0] steps from host arrays (numpy, or page-locked torch CPU tensors for
        asynchronous copies); returns T of the same shape."""
        if hasattr(D, "data_ptr"):
            steps = int(D.shape[0])
            _check(lib().fdph_run_host(self.handle, steps, _ptr(D), _ptr(T)))
            return T
        D = np.ascontiguousarray(D, dtype=np.float64)
        if T is None:
            T = np.empty_like(D)
        _check(lib().fdph_run_host(self.handle, int(D.shape[0]), ctypes.c_void_p(D.ctypes.data),
                                   ctypes.c_void_p(T.ctypes.data)))
        return T

    def autotune(self, steps=16):
        """fdph_autotune: picks the near-field work-item length; returns it."""
        c = ctypes.c_int32()
        _check(lib().fdph_autotune(self.handle, int(steps), ctypes.byref(c)))
        return c.value

    def reset(self):
        _check(lib().fdph_reset(self.handle))

    def current_step(self):
        n = ctypes.c_int32()
        _check(lib().fdph_current_step(self.handle, ctypes.byref(n)))
        return n.value

    @property
    def stream(self):
        """The cudaStream_t handle (int) the plan runs on (fdph_plan_stream)."""
        h = ctypes.c_void_p()
        _check(lib().fdph_plan_stream(self.handle, ctypes.byref(h)))
        return h.value or 0

    def synchronize(self):
        _check(lib().fdph_synchronize(self.handle))

    def stats(self):
        s = Stats()
        _check(lib().fdph_get_stats(self.handle, ctypes.byref(s)))
        return s.as_dict()

    def rupture_init(self, tau0, sigma_n, mu_s, mu_d, Dc, law=0):
        """Attach slip-weakening friction (fdph_rupture_init), law 0 linear, 1 exponential;
        tau0 is a device buffer."""
        self._tau0 = tau0
        fr = Friction(_ptr(tau0).value, sigma_n, mu_s, mu_d, Dc, int(law))
        _check(lib().fdph_rupture_init(self.handle, ctypes.byref(fr)))

    def predict(self, T_pred):
        """Traction of the current step with D_n = 0 into the device buffer T_pred (fdph_predict)."""
        _check(lib().fdph_predict(self.handle, _ptr(T_pred)))

    def commit(self, D_n):
        """Append D_n (device buffer) and advance one step (fdph_commit)."""
        _check(lib().fdph_commit(self.handle, _ptr(D_n)))

    def self_coefficients(self):
        """K_{ii,0} in geometry order (fdph_self), a numpy array."""
        out = np.empty(self.n, dtype=np.float64)
        _check(lib().fdph_self(self.handle, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def rupture_step(self, D_n, T_n):
        _check(lib().fdph_rupture_step(self.handle, _ptr(D_n), _ptr(T_n)))

    def rupture_run(self, steps, D, T):
        _check(lib().fdph_rupture_run(self.handle, int(steps), _ptr(D), _ptr(T)))

    def rupture_slip(self, out):
        _check(lib().fdph_rupture_slip(self.handle, _ptr(out)))

    def set_profiling(self, on=True):
        _check(lib().fdph_set_profiling(self.handle, 1 if on else 0))

    def kernel_times(self):
        """{kernel name: (total ms, launches)} since profiling was enabled."""
        ms = (ctypes.c_double * len(KERNEL_NAMES))()
        cnt = (ctypes.c_int64 * len(KERNEL_NAMES))()
        _check(lib().fdph_kernel_times(self.handle, ms, cnt))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_NAMES)}

    def save_state(self):
        n = ctypes.c_size_t()
        _check(lib().fdph_save_state(self.handle, None, ctypes.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        _check(lib().fdph_save_state(self.handle, ctypes.c_void_p(buf.ctypes.data), ctypes.byref(n)))
        return buf

    def load_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib().fdph_load_state(self.handle, ctypes.c_void_p(buf.ctypes.data), buf.size))

    def close(self):
        if getattr(self, "handle", None):
            lib().fdph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plain_step_noalloc(K, n, W, D_hist, hist_len, step, T, stream=None):
    """fdph_plain_step_noalloc: one plain step from caller-held device buffers, no allocation.

    K (W n n), D_hist (hist_len n) and T (n) must be contiguous float64 CUDA tensors on one
    device and hold at least those many elements: the library reads and writes them through raw
    pointers, so a short buffer would be read out of bounds on the GPU.  stream: a cudaStream_t
    handle (int); None means torch's current stream on T's device."""
    import torch
    n, W, hist_len, step = int(n), int(W), int(hist_len), int(step)
    need = {"K": (K, W * n * n), "D_hist": (D_hist, hist_len * n), "T": (T, n)}
    for name, (t, count) in need.items():
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise FdphError(E_ARG, "plain_step_noalloc: %s must be a contiguous float64 CUDA tensor" % name)
        if t.device != T.device:
            raise FdphError(E_ARG, "plain_step_noalloc: %s is not on T's device" % name)
        if n > 0 and W > 0 and hist_len > 0 and t.numel() < count:
            raise FdphError(E_ARG, "plain_step_noalloc: %s holds %d elements, %d needed" % (name, t.numel(), count))
    if stream is None:
        stream = torch.cuda.current_stream(T.device).cuda_stream
    s = ctypes.c_void_p(stream) if stream else None
    with torch.cuda.device(T.device):
        _check(lib().fdph_plain_step_noalloc(_ptr(K), n, W, _ptr(D_hist), hist_len, step, _ptr(T), s))


class Batch:
    """Plans stepped together with one near-field launch per step (fdph_batch_create); the
    plans must outlive the batch."""

    def __init__(self, plans):
        L = lib()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(L.fdph_batch_create(arr, len(self.plans), ctypes.byref(h)))
        self.handle = h

    def _ptrs(self, bufs):
        if len(bufs) != len(self.plans):
            raise ValueError("one buffer per plan")
        return (ctypes.c_void_p * len(bufs))(*[_ptr(b).value for b in bufs])

    def run(self, steps, D, T):
        """`steps` steps of every plan: D[p], T[p] device buffers of plan p (fdph_batch_run)."""
        _check(lib().fdph_batch_run(self.handle, int(steps), self._ptrs(D), self._ptrs(T)))

    def rupture_run(self, steps, D, T):
        _check(lib().fdph_batch_rupture_run(self.handle, int(steps), self._ptrs(D), self._ptrs(T)))

    def synchronize(self):
        _check(lib().fdph_batch_synchronize(self.handle))

    def close(self):
        if self.handle:
            lib().fdph_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def quantize(K, eps_q):
    """The plan's quantization rule (fdph_quantize): returns (b, khat) for the values K."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    n = K.shape[0]
    b = np.zeros(n + 1, dtype=np.int32)
    kh = np.zeros(n)
    q = ctypes.c_int32()
    _check(lib().fdph_quantize(ctypes.c_void_p(K.ctypes.data), n, float(eps_q), b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               ctypes.c_void_p(kh.ctypes.data), ctypes.byref(q)))
    return b[:q.value + 1].copy(), kh[:q.value].copy()


def low_rank(A, eps):
    """The plan's low-rank approximation of one block (fdph_low_rank): returns (F, G, exact)
    with A ~ F G^T."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    k = min(m, n)
    F = np.zeros(m * k)
    G = np.zeros(n * k)
    r, ex = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().fdph_low_rank(ctypes.c_void_p(A.ctypes.data), m, n, float(eps), ctypes.c_void_p(F.ctypes.data),
                               ctypes.c_void_p(G.ctypes.data), ctypes.byref(r), ctypes.byref(ex)))
    r = r.value
    return F[:m * r].reshape(m, r), G[:n * r].reshape(n, r), bool(ex.value)


def kernel_tail(p, seg, t1, dt, mu=1.0, cs=1.0):
    """Domain-S remainder of the discrete kernel and its scan bound (fdph_kernel_tail):
    returns (tail_x, tail_y, bound)."""
    pp = np.ascontiguousarray(p, dtype=np.float64)
    sg = np.ascontiguousarray(seg, dtype=np.float64)
    out = np.zeros(3)
    _check(lib().fdph_kernel_tail(ctypes.c_void_p(pp.ctypes.data), ctypes.c_void_p(sg.ctypes.data), float(t1),
                                  float(dt), float(mu), float(cs), ctypes.c_void_p(out.ctypes.data)))
    return out[0], out[1], out[2]


def low_rank_aca(A, eps):
    """The plan's cross approximation of one large block (fdph_low_rank_aca): returns
    (F, G, evaluated) with A ~ F G^T and the number of entries read, or (None, None, evaluated)
    when the cross did not converge."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    k = min(m, n, 96)
    F = np.zeros(m * k)
    G = np.zeros(n * k)
    r, ok, ev = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().fdph_low_rank_aca(ctypes.c_void_p(A.ctypes.data), m, n, float(eps), ctypes.c_void_p(F.ctypes.data),
                                   ctypes.c_void_p(G.ctypes.data), ctypes.byref(r), ctypes.byref(ok), ctypes.byref(ev)))
    if not ok.value:
        return None, None, ev.value
    r = r.value
    return F[:m * r].reshape(m, r), G[:n * r].reshape(n, r), ev.value


def tree_export(xy, dt, mu=1.0, cs=1.0, **params):
    """Host-only block tree + ART integers (fdph_tree_export), parsed."""
    L = lib()
    g, keep = _geometry(xy)
    mat = Material(mu, cs)
    p = make_params(**params)
    n = ctypes.c_int64()
    _check(L.fdph_tree_export(ctypes.byref(g), ctypes.byref(mat), dt, ctypes.byref(p), None, 0, ctypes.byref(n)))
    buf = np.empty(n.value, dtype=np.int32)
    _check(L.fdph_tree_export(ctypes.byref(g), ctypes.byref(mat), dt, ctypes.byref(p),
                              buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n.value, ctypes.byref(n)))
    N = int(buf[0])
    perm = buf[1:1 + N].copy()
    q = 1 + N
    nl = int(buf[q])
    q += 1
    leaves = []
    for _ in range(nl):
        kind, r0, nr, s0, ns = (int(v) for v in buf[q:q + 5])
        q += 5
        lf = dict(kind=kind, r0=r0, nr=nr, s0=s0, ns=ns)
        if kind == 1:
            lf["dm"] = buf[q:q + nr].copy()
            q += nr
            lf["mbar"] = buf[q:q + ns].copy()
            q += ns
            lf["Dm"] = buf[q:q + ns].copy()
            q += ns
        leaves.append(lf)
    return dict(perm=perm, leaves=leaves)
