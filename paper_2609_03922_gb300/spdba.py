"""Thin Python binding of libspdba.so (include/spdba.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels.  PyTorch supplies
device memory and the stream.  If the shared library has not been built this
module raises at load time; there is no fallback path.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libspdba.so")

SPDBA_OK, SPDBA_ERR_ARG, SPDBA_ERR_UNSUPPORTED, SPDBA_ERR_CUDA, SPDBA_ERR_OOM, SPDBA_ERR_TIMEOUT, SPDBA_ERR_STATE = range(7)
SPDBA_MODEL_CH, SPDBA_MODEL_NLS, SPDBA_MODEL_RCD = 0, 1, 2
SPDBA_C64, SPDBA_C128 = 0, 1
SPDBA_MODE_REGULAR, SPDBA_MODE_ADAPTIVE = 0, 1
SPDBA_MEASURE_MAXAMP, SPDBA_MEASURE_ENERGY = 0, 1
SPDBA_TAU_REL_MAX, SPDBA_TAU_ABS = 0, 1
SPDBA_FROZEN, SPDBA_TRANSITION, SPDBA_ACTIVE = 0, 1, 2
SPDBA_FORWARD, SPDBA_INVERSE = -1, 1


class spdba_options(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("precision", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("measure", ctypes.c_int32), ("tau_rule", ctypes.c_int32), ("transitions", ctypes.c_int32),
                ("force_dc", ctypes.c_int32), ("refresh_every", ctypes.c_int32),
                ("warmup_steps", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("fuse_update", ctypes.c_int32),
                ("half_spectrum", ctypes.c_int32),
                ("dt", ctypes.c_double), ("kappa", ctypes.c_double), ("dx", ctypes.c_double),
                ("beta2", ctypes.c_double), ("gamma", ctypes.c_double), ("h", ctypes.c_double),
                ("dt_sample", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("target_ratio", ctypes.c_double), ("control_eta", ctypes.c_double),
                ("control_every", ctypes.c_int32), ("components", ctypes.c_int32),
                ("rcd_d_diag", ctypes.c_double), ("rcd_d_cross", ctypes.c_double), ("rcd_alpha", ctypes.c_double),
                ("rcd_beta", ctypes.c_double), ("rcd_r", ctypes.c_double), ("rcd_a", ctypes.c_double),
                ("tma_update", ctypes.c_int32), ("multi_pass", ctypes.c_int32),
                ("tma_passes", ctypes.c_int32),
                ("half_storage", ctypes.c_int32)]


class spdba_stats(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("assessments", ctypes.c_int64), ("nblocks", ctypes.c_int64),
                ("n_active", ctypes.c_int64), ("n_transition", ctypes.c_int64), ("tau", ctypes.c_double),
                ("max_amp", ctypes.c_double), ("mass", ctypes.c_double), ("active_ratio_sum", ctypes.c_double),
                ("predictions", ctypes.c_int64), ("missed_blocks", ctypes.c_int64),
                ("threshold", ctypes.c_double), ("controls", ctypes.c_int64)]


TUNE_MAX = 16


class spdba_tune_report(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int32), ("fuse_update", ctypes.c_int32 * TUNE_MAX),
                ("use_graph", ctypes.c_int32 * TUNE_MAX), ("half_spectrum", ctypes.c_int32 * TUNE_MAX),
                ("tma_update", ctypes.c_int32 * TUNE_MAX),
                ("ms_per_step", ctypes.c_double * TUNE_MAX), ("chosen", ctypes.c_int32),
                ("multi_pass", ctypes.c_int32 * TUNE_MAX), ("cached", ctypes.c_int32)]


class spdba_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


# Every symbol include/spdba.h declares, with its ctypes signature.
_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_I64P = ctypes.POINTER(ctypes.c_int64)
_I32P = ctypes.POINTER(ctypes.c_int32)
_S = ctypes.c_int
SIGNATURES = {
    "spdba_options_default": (None, [ctypes.POINTER(spdba_options)]),
    "spdba_plan_create": (_S, [_PP, ctypes.c_int32, _I64P, _I32P, ctypes.c_double, ctypes.c_int32,
                               ctypes.POINTER(spdba_options)]),
    "spdba_batch_create": (_S, [_PP, ctypes.c_int32, ctypes.c_int32, _I64P, _I32P, ctypes.c_double,
                                ctypes.c_int32, ctypes.POINTER(spdba_options)]),
    "spdba_set_field": (_S, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    "spdba_step": (_S, [_P, ctypes.c_int64]),
    "spdba_get_field": (_S, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    "spdba_get_spectrum": (_S, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    "spdba_set_spectrum": (_S, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    "spdba_get_mask": (_S, [_P, ctypes.c_int32, _P, ctypes.c_int64]),
    "spdba_get_stats": (_S, [_P, ctypes.c_int32, ctypes.POINTER(spdba_stats)]),
    "spdba_sync": (_S, [_P]),
    "spdba_get_activity": (_S, [_P, ctypes.c_int32, _P, _P, ctypes.c_int32]),
    "spdba_plan_attach_predictor": (_S, [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_float]),
    "spdba_plan_autotune": (_S, [_P, ctypes.c_int32, ctypes.POINTER(spdba_tune_report)]),
    "spdba_plan_autotune_cached": (_S, [_P, ctypes.c_int32, ctypes.POINTER(spdba_tune_report)]),
    "spdba_tune_cache_clear": (None, []),
    "spdba_plan_get_config": (_S, [_P, ctypes.POINTER(spdba_options)]),
    "spdba_profile_begin": (_S, [_P]),
    "spdba_profile_begin_sampled": (_S, [_P, ctypes.c_int32]),
    "spdba_profile_end": (_S, [_P, ctypes.POINTER(spdba_kernel_time), ctypes.c_int32, _I32P,
                              ctypes.POINTER(ctypes.c_int64)]),
    "spdba_plan_destroy": (None, [_P]),
    "spdba_last_error": (ctypes.c_char_p, []),
    "spdba_debug_fail_alloc": (None, [ctypes.c_int64]),
    "spdba_debug_live_allocs": (ctypes.c_int64, []),
    "spdba_debug_set_wait_limit": (None, [ctypes.c_int64]),
    "spdba_debug_stall_waits": (None, [ctypes.c_int32]),
    "spdba_status_string": (ctypes.c_char_p, [_S]),
    "spdba_fft_plan_create": (_S, [_PP, ctypes.c_int32, ctypes.c_int32, _I64P, ctypes.c_int64]),
    "spdba_fft_exec": (_S, [_P, _P, _P, ctypes.c_int32, _P]),
    "spdba_fft_plan_destroy": (None, [_P]),
    "spdba_block_activity": (_S, [ctypes.c_int32, ctypes.c_int32, _I64P, _I32P, _P, _P, _P, _P, _P]),
    "spdba_classify_scratch_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "spdba_classify": (_S, [ctypes.c_int32, _I64P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P,
                            _P, _P]),
    "spdba_classify_static": (_S, [ctypes.c_int32, _I64P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P,
                                   _P, _P]),
    "spdba_predictor_num_params": (ctypes.c_int64, []),
    "spdba_predictor_create": (_S, [_PP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P]),
    "spdba_predictor_destroy": (None, [_P]),
    "spdba_predictor_get_params": (_S, [_P, _P]),
    "spdba_predictor_set_params": (_S, [_P, _P]),
    "spdba_predictor_features": (_S, [_P, _P, _P, _P, ctypes.c_int32, _P, _P]),
    "spdba_predictor_forward": (_S, [_P, _P, ctypes.c_int32, _P, _P]),
    "spdba_predictor_gradients": (_S, [_P, _P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), _P]),
    "spdba_predictor_train_step": (_S, [_P, _P, _P, ctypes.c_int32, ctypes.c_float, ctypes.POINTER(ctypes.c_double),
                                        _P]),
}

_lib = None


class SpdbaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("spdba error %d: %s" % (status, msg))
        self.status = status


def lib():
    """Load libspdba.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libspdba.so is not built (%s); run __graft_entry__.build() first" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != SPDBA_OK:
        raise SpdbaError(status, lib().spdba_last_error().decode())


def _i64(vals):
    return (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])


def _i32(vals):
    return (ctypes.c_int32 * len(vals))(*[int(v) for v in vals])


def _ptr(x):
    """(pointer, on_device) of a torch tensor or numpy array (contiguous)."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, 0
    import torch
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), 1 if x.is_cuda else 0
    raise TypeError("expected a numpy array or torch tensor")


def current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def options_default(**kw):
    o = spdba_options()
    lib().spdba_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError("unknown option %s" % k)
        setattr(o, k, v)
    return o


class Plan:
    """One sp-DBA plan (spdba_plan_create / spdba_batch_create)."""

    def __init__(self, dims, block, threshold=1e-6, reassess=10, batch_dims=None, stream=None, **opts):
        o = options_default(**opts)
        o.stream = current_stream() if stream is None else stream
        self.opts = o
        self._p = ctypes.c_void_p()
        if batch_dims is None:
            self.ndim = len(dims)
            self.run_dims = [tuple(int(d) for d in dims)]
            check(lib().spdba_plan_create(ctypes.byref(self._p), self.ndim, _i64(dims), _i32(block),
                                          float(threshold), int(reassess), ctypes.byref(o)))
        else:
            self.ndim = len(batch_dims[0])
            self.run_dims = [tuple(int(d) for d in r) for r in batch_dims]
            flat = [d for r in self.run_dims for d in r]
            check(lib().spdba_batch_create(ctypes.byref(self._p), len(self.run_dims), self.ndim, _i64(flat),
                                           _i32(block), float(threshold), int(reassess), ctypes.byref(o)))
        self.block = tuple(block)
        self.complex_dtype = np.complex64 if o.precision == SPDBA_C64 else np.complex128
        self.real_dtype = np.float32 if o.precision == SPDBA_C64 else np.float64

    def close(self):
        if self._p:
            lib().spdba_plan_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_field(self, x, run=0):
        p, dev = _ptr(x)
        check(lib().spdba_set_field(self._p, run, p, dev))

    def step(self, n=1):
        check(lib().spdba_step(self._p, int(n)))

    def sync(self):
        check(lib().spdba_sync(self._p))

    def field_dtype(self):
        return self.complex_dtype if self.opts.model == SPDBA_MODEL_NLS else self.real_dtype

    def field_shape(self, run=0):
        """Shape of a run's field: (components, *dims) for RCD plans, dims otherwise."""
        if self.opts.model == SPDBA_MODEL_RCD:
            return (int(self.opts.components),) + tuple(self.run_dims[run])
        return tuple(self.run_dims[run])

    def get_field(self, out=None, run=0):
        if out is None:
            out = np.empty(self.field_shape(run), dtype=self.field_dtype())
        p, dev = _ptr(out)
        check(lib().spdba_get_field(self._p, run, p, dev))
        return out

    def spectrum_shape(self, run=0):
        """Shape of a run's stored spectrum: with half-spectrum storage the last axis
        keeps x frequencies 0 .. N2/2."""
        shape = self.field_shape(run)
        if self.opts.half_storage:
            shape = shape[:-1] + (shape[-1] // 2 + 1,)
        return shape

    def get_spectrum(self, out=None, run=0):
        if out is None:
            out = np.empty(self.spectrum_shape(run), dtype=self.complex_dtype)
        p, dev = _ptr(out)
        check(lib().spdba_get_spectrum(self._p, run, p, dev))
        return out

    def set_spectrum(self, x, run=0):
        p, dev = _ptr(x)
        check(lib().spdba_set_spectrum(self._p, run, p, dev))

    def nblocks_shape(self, run=0):
        if self.opts.model == SPDBA_MODEL_NLS and self.block[0] <= 0:
            return (-self.block[0],)
        shape = tuple(d // b for d, b in zip(self.run_dims[run], self.block))
        if self.opts.half_storage:
            shape = shape[:-1] + (self.run_dims[run][-1] // (2 * self.block[-1]) + 1,)
        return shape

    def get_mask(self, run=0):
        shape = self.nblocks_shape(run)
        out = np.empty(shape, dtype=np.uint8)
        check(lib().spdba_get_mask(self._p, run, out.ctypes.data, out.size))
        return out

    def autotune(self, steps=20, cached=False):
        """Pick the fastest launch configuration (spdba_plan_autotune, or with
        cached=True spdba_plan_autotune_cached); returns the candidates with their
        ms per step, the chosen index and whether a stored choice was applied."""
        rep = spdba_tune_report()
        fn = lib().spdba_plan_autotune_cached if cached else lib().spdba_plan_autotune
        check(fn(self._p, int(steps), ctypes.byref(rep)))
        cands = [{"fuse_update": int(rep.fuse_update[i]), "use_graph": int(rep.use_graph[i]),
                  "half_spectrum": int(rep.half_spectrum[i]), "tma_update": int(rep.tma_update[i]),
                  "multi_pass": int(rep.multi_pass[i]), "ms_per_step": float(rep.ms_per_step[i])}
                 for i in range(rep.n_candidates)]
        return {"candidates": cands, "chosen": int(rep.chosen), "cached": int(rep.cached)}

    def get_config(self):
        """The options in force (spdba_plan_get_config) as a dict."""
        o = spdba_options()
        check(lib().spdba_plan_get_config(self._p, ctypes.byref(o)))
        return {f: getattr(o, f) for f, _ in spdba_options._fields_ if f != "stream"}

    def profile_begin(self, every=1):
        """Record kernel events of every step, or of one step in `every`."""
        check(lib().spdba_profile_begin_sampled(self._p, int(every)))

    def profile_end(self):
        """Returns ({kind: {launches, total_ms, bytes}}, kernel launches since begin)."""
        buf = (spdba_kernel_time * 16)()
        n = ctypes.c_int32()
        launches = ctypes.c_int64()
        check(lib().spdba_profile_end(self._p, buf, 16, ctypes.byref(n), ctypes.byref(launches)))
        out = {}
        for i in range(n.value):
            k = buf[i]
            out[k.name.decode()] = {"launches": int(k.launches), "total_ms": float(k.total_ms), "bytes": float(k.bytes)}
        return out, int(launches.value)

    def get_activity(self, maxsq=None, tau=None, run=0):
        """Per-block max |q|^2 and tau of the last exact reassessment (numpy, or into
        the given device tensors)."""
        if maxsq is None:
            maxsq = np.empty(self.nblocks_shape(run), dtype=np.float64)
            tau_h = np.empty(1, dtype=np.float64)
            check(lib().spdba_get_activity(self._p, run, maxsq.ctypes.data, tau_h.ctypes.data, 0))
            return maxsq, float(tau_h[0])
        check(lib().spdba_get_activity(self._p, run, maxsq.data_ptr(), tau.data_ptr(), 1))
        return maxsq, tau

    def attach_predictor(self, predictor, horizon=20, judge_every=100, prob_threshold=0.5):
        self._pred = predictor
        check(lib().spdba_plan_attach_predictor(self._p, predictor._p if predictor is not None else None,
                                                int(horizon), int(judge_every), float(prob_threshold)))

    def get_stats(self, run=0):
        s = spdba_stats()
        check(lib().spdba_get_stats(self._p, run, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in spdba_stats._fields_}


class FFTPlan:
    """Batched multi-dimensional FFT (spdba_fft_plan_create / spdba_fft_exec)."""

    def __init__(self, dims, batch=1, precision=SPDBA_C64):
        self._p = ctypes.c_void_p()
        check(lib().spdba_fft_plan_create(ctypes.byref(self._p), precision, len(dims), _i64(dims), int(batch)))

    def exec(self, x, out, direction, stream=None):
        pin, _ = _ptr(x)
        pout, _ = _ptr(out)
        check(lib().spdba_fft_exec(self._p, pin, pout, direction, current_stream() if stream is None else stream))

    def close(self):
        if self._p:
            lib().spdba_fft_plan_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_cache_clear():
    """Forget every stored autotuner choice (spdba_tune_cache_clear)."""
    lib().spdba_tune_cache_clear()


def block_activity(q, block, maxsq, sumsq, gmax, precision=SPDBA_C64, stream=None):
    check(lib().spdba_block_activity(precision, q.dim(), _i64(q.shape), _i32(block), q.data_ptr(),
                                     maxsq.data_ptr(), sumsq.data_ptr() if sumsq is not None else None,
                                     gmax.data_ptr(), current_stream() if stream is None else stream))


def classify_scratch_bytes(nb):
    return int(lib().spdba_classify_scratch_bytes(int(nb)))


def classify(nblocks, measure, tau, force_dc, transitions, states, chi, lst, count, scratch, stream=None):
    check(lib().spdba_classify(len(nblocks), _i64(nblocks), measure.data_ptr(), tau.data_ptr(), int(force_dc),
                               int(transitions), states.data_ptr(), chi.data_ptr(), lst.data_ptr(),
                               count.data_ptr(), scratch.data_ptr(),
                               current_stream() if stream is None else stream))


CLASSIFY_STATIC_MAX_BLOCKS = 1 << 20


def classify_static(nblocks, measure, tau, force_dc, transitions, states, chi, lst, count, stream=None):
    """spdba_classify with the library's fixed scratch array (no allocation)."""
    check(lib().spdba_classify_static(len(nblocks), _i64(nblocks), measure.data_ptr(), tau.data_ptr(),
                                      int(force_dc), int(transitions), states.data_ptr(), chi.data_ptr(),
                                      lst.data_ptr(), count.data_ptr(),
                                      current_stream() if stream is None else stream))


def predictor_init_params(seed=0):
    """He-style random initial parameters (FP32), in the library's flat order."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in ((2, 8), (8, 16), (16, 8)):
        parts.append(rng.standard_normal(co * 27 * ci) * np.sqrt(2.0 / (27 * ci)))
        parts.append(np.zeros(co))
    parts.append(rng.standard_normal(8) * np.sqrt(1.0 / 8))
    parts.append(np.zeros(1))
    return np.concatenate(parts).astype(np.float32)


class Predictor:
    """The learned block-activity predictor (spdba_predictor_*)."""

    def __init__(self, map_dims, max_batch=1, params=None, seed=0):
        self.map_dims = tuple(int(d) for d in map_dims)
        self.nparams = int(lib().spdba_predictor_num_params())
        p = predictor_init_params(seed) if params is None else np.ascontiguousarray(params, dtype=np.float32)
        self._p = ctypes.c_void_p()
        check(lib().spdba_predictor_create(ctypes.byref(self._p), *self.map_dims, int(max_batch), p.ctypes.data))

    def close(self):
        if self._p:
            lib().spdba_predictor_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.empty(self.nparams, dtype=np.float32)
        check(lib().spdba_predictor_get_params(self._p, out.ctypes.data))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        check(lib().spdba_predictor_set_params(self._p, p.ctypes.data))

    def features(self, maxsq, tau, states, x_out, nmaps=1, stream=None):
        check(lib().spdba_predictor_features(self._p, maxsq.data_ptr(), tau.data_ptr(), states.data_ptr(), nmaps,
                                             x_out.data_ptr(), current_stream() if stream is None else stream))

    def forward(self, x, prob, nmaps=1, stream=None):
        check(lib().spdba_predictor_forward(self._p, x.data_ptr(), nmaps, prob.data_ptr(),
                                            current_stream() if stream is None else stream))

    def gradients(self, x, labels, nmaps=1):
        loss = ctypes.c_double()
        g = np.empty(self.nparams, dtype=np.float32)
        check(lib().spdba_predictor_gradients(self._p, x.data_ptr(), labels.data_ptr(), nmaps, ctypes.byref(loss),
                                              g.ctypes.data))
        return loss.value, g

    def train_step(self, x, labels, lr, nmaps=1, want_loss=True, stream=None):
        loss = ctypes.c_double()
        check(lib().spdba_predictor_train_step(self._p, x.data_ptr(), labels.data_ptr(), nmaps, float(lr),
                                               ctypes.byref(loss) if want_loss else None,
                                               current_stream() if stream is None else stream))
        return loss.value if want_loss else None
