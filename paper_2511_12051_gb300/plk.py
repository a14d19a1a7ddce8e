"""Python binding of libplk (include/plk.h): argument marshalling only.

Every function takes CUDA torch tensors, checks dtype/device/contiguity, and
calls the C entry point of the same name on the context's stream; all
arithmetic runs in the library's CUDA kernels.  There is no CPU fallback: if
libplk.so is missing or no GPU is present, calls raise.

Layouts follow include/plk.h: stacks complex64 [N, H, W]; per-output-pixel
arrays [Ho, Wo] with Ho = H // sy, Wo = W // sx; masks uint64 [Ho, Wo, words]
(stored in an int64 tensor); packed coherences complex64 [Ho, Wo, N(N+1)/2].
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# PLK_LIB_PATH selects another build of the same library (e.g. a variant built
# with extra compile-time flags); by default the in-tree build is loaded.
LIB_PATH = os.environ.get("PLK_LIB_PATH") or os.path.join(_HERE, "_build", "libplk.so")

PLK_MAX_N = 32
PX_EMI, PX_EMI_FP64, PX_EVD, PX_NODATA, PX_NOCONV, PX_PS = 0, 1, 2, 3, 4, 5
_STATUS = {0: "PLK_OK", 1: "PLK_EINVAL", 2: "PLK_ENOMEM", 3: "PLK_ECUDA", 4: "PLK_ETIMEOUT", 5: "PLK_EUNSUPPORTED"}


class PlkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class Window(ctypes.Structure):
    _fields_ = [("wy", ctypes.c_int32), ("wx", ctypes.c_int32), ("sy", ctypes.c_int32), ("sx", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_float), ("mu", ctypes.c_float),
                ("tol", ctypes.c_float), ("max_iter", ctypes.c_int32), ("cond_max", ctypes.c_float),
                ("fp64_resolve", ctypes.c_int32), ("err_max", ctypes.c_float), ("cov_precision", ctypes.c_int32),
                ("ref_scheme", ctypes.c_int32), ("ps_da_max", ctypes.c_float), ("decay", ctypes.c_float)]


class StackDesc(ctypes.Structure):
    _fields_ = [("slc", ctypes.c_void_p), ("N", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("ref_idx", ctypes.c_int32), ("phase", ctypes.c_void_p), ("tcoh", ctypes.c_void_p),
                ("status", ctypes.c_void_p)]


class Tile(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("y0", "x0", "h", "w", "oy0", "ox0", "oh", "ow", "cy0", "cx0",
                                                "py0", "px0", "ph", "pw")]


COV_FP32 = 0  # PLK_COV_FP32
COV_BF16 = 1  # PLK_COV_BF16
COV_FP16 = 2  # PLK_COV_FP16
REF_FIRST = 0  # PLK_REF_FIRST
REF_LAST_REAL = 1  # PLK_REF_LAST_REAL


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "plk_create": [ctypes.POINTER(_P), _I, _P],
    "plk_destroy": [_P],
    "plk_set_stream": [_P, _P],
    "plk_sync": [_P],
    "plk_selftest_bounded_wait": [_P],
    "plk_default_params": [ctypes.POINTER(Params)],
    "plk_output_shape": [_I, _I, Window, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "plk_glrt_threshold": [ctypes.c_double, _I, ctypes.POINTER(ctypes.c_double)],
    "plk_glrt_threshold_looks": [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)],
    "plk_amp_stats": [_P, _P, _I, _I, _I, _P, _P, _I],
    "plk_shp_select": [_P, _P, _I, _I, _I, Window, ctypes.c_double, _P, _P],
    "plk_estimate_covariance": [_P, _P, _I, _I, _I, Window, _P, _I, _P],
    "plk_phase_link": [_P, _P, _I, ctypes.c_int64, _I, ctypes.POINTER(Params), _P, _P, _P, _P],
    "plk_compress": [_P, _P, _I, _I, _I, _I, Window, _P, _P],
    "plk_ps_regrid": [_P, _P, _I, _I, _I, _I, Window, _P, _P, _I, _I, ctypes.c_float, _P, _P],
    "plk_phase_similarity": [_P, _P, _I, _I, _I, _I, _P],
    "plk_invert_l1": [_P, _P, _I, _P, _I, ctypes.c_int64, ctypes.c_float, _I, _P, _P],
    "plk_state_create": [_P, _I, _I, Window, _I, _I, ctypes.POINTER(_P)],
    "plk_state_destroy": [_P],
    "plk_state_info": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "plk_state_weights": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "plk_state_kappa": [_P, _I, ctypes.POINTER(_P)],
    "plk_state_sums": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)],
    "plk_state_save": [_P, _P, ctypes.c_char_p],
    "plk_state_load": [_P, ctypes.c_char_p, _I, ctypes.POINTER(_P)],
    "plk_ministack_step": [_P, _P, _P, _I, ctypes.POINTER(Params), _P, _P, _P, _P],
    "plk_ministack_step_host": [_P, _P, _P, _I, ctypes.POINTER(Params), _P, _P, _P, _P],
    "plk_state_enable_host_io": [_P, _P],
    "plk_state_enable_host_io_ci16": [_P, _P],
    "plk_ministack_step_host_ci16": [_P, _P, _P, _I, ctypes.POINTER(Params), _P, _P, _P, _P],
    "plk_state_reset": [_P],
    "plk_profile_enable": [_P, _I],
    "plk_profile_collect": [_P, ctypes.POINTER(_I)],
    "plk_profile_get": [_P, _I, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I)],
    "plk_phase_link_stack_noalloc": [_P, _I, _I, _I, Window, _I, ctypes.POINTER(Params), _P, _P, _P, _P, _P],
    "plk_backward_workspace_size": [_I, _I, _I, Window, ctypes.POINTER(ctypes.c_size_t)],
    "plk_phase_link_backward": [_P, _P, _I, _I, _I, Window, _P, _I, ctypes.POINTER(Params), _P, _P,
                                ctypes.c_size_t, _P],
    "plk_shp_weight_gradient": [_P, _P, _I, _I, _I, Window, _P, _I, ctypes.POINTER(Params), _P, _P,
                                ctypes.c_size_t, _P],
    "plk_phase_uncertainty": [_P, _P, _I, _I, _I, Window, _P, _I, ctypes.POINTER(Params), ctypes.c_float, _P,
                              ctypes.c_size_t, _P],
    "plk_batch_create": [_P, _P, _I, Window, ctypes.POINTER(Params), ctypes.POINTER(_P)],
    "plk_batch_run": [_P, _P],
    "plk_batch_info": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "plk_batch_destroy": [_P],
    "plk_tuned_schedule": [_P, _I, Window, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "plk_tile_plan": [_I, _I, Window, _I, _I, _I, ctypes.POINTER(Tile)],
}
EXPORTS = sorted(list(_SIGS) + ["plk_last_error", "plk_mask_words", "plk_device_allocations"])


def lib():
    """Load libplk.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise PlkError(5, f"{LIB_PATH} is not built; run `python -m paper_2511_12051_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.plk_last_error.argtypes = [_P]
            L.plk_last_error.restype = ctypes.c_char_p
            L.plk_mask_words.argtypes = [Window]
            L.plk_mask_words.restype = ctypes.c_int
            L.plk_device_allocations.argtypes = []
            L.plk_device_allocations.restype = ctypes.c_int64
            _lib = L
    return _lib


def _check(code: int, ctx=None):
    if code != 0:
        msg = lib().plk_last_error(ctx).decode(errors="replace")
        raise PlkError(code, msg)


def window(w) -> Window:
    if isinstance(w, Window):
        return w
    wy, wx, sy, sx = (int(v) for v in w)
    return Window(wy, wx, sy, sx)


def default_params(**over) -> Params:
    p = Params()
    _check(lib().plk_default_params(ctypes.byref(p)))
    for k, v in over.items():
        setattr(p, k, v)
    return p


def glrt_threshold(alpha: float, n_eff: int) -> float:
    c = ctypes.c_double()
    _check(lib().plk_glrt_threshold(float(alpha), int(n_eff), ctypes.byref(c)))
    return c.value


def glrt_threshold_looks(alpha: float, nu: float) -> float:
    c = ctypes.c_double()
    _check(lib().plk_glrt_threshold_looks(float(alpha), float(nu), ctypes.byref(c)))
    return c.value


def tile_plan(H: int, W: int, win, tiles_y: int, tiles_x: int, steps: int = 1) -> list[dict]:
    """plk_tile_plan: tiles_y x tiles_x spatial tiles of an H x W burst (row-major),
    each with the input crop that makes its owned outputs exact for `steps`
    mini-stack steps."""
    arr = (Tile * (int(tiles_y) * int(tiles_x)))()
    _check(lib().plk_tile_plan(int(H), int(W), window(win), int(tiles_y), int(tiles_x), int(steps), arr))
    return [{k: int(getattr(t, k)) for k, _ in Tile._fields_} for t in arr]


def device_allocations() -> int:
    """Device allocations the library has made in this process."""
    return int(lib().plk_device_allocations())


def output_shape(H: int, W: int, win) -> tuple[int, int]:
    w = window(win)
    return H // w.sy, W // w.sx


def mask_words(win) -> int:
    return int(lib().plk_mask_words(window(win)))


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t: torch.Tensor, dtype, name: str, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if t.device.type != "cuda":
        raise ValueError(f"{name}: must be a CUDA tensor (no CPU path)")
    if device is not None and t.device != device:
        raise ValueError(f"{name}: on {t.device}, context on {device}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")


class Context:
    """plk_ctx bound to a CUDA device and stream (default: the current stream)."""

    def __init__(self, device=None, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise PlkError(3, "no CUDA device available (libplk has no CPU path)")
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        h = ctypes.c_void_p()
        _check(lib().plk_create(ctypes.byref(h), dev.index, ctypes.c_void_p(self.stream.cuda_stream)))
        self.h = h

    def sync(self):
        """Wait for this context's work; raises on a timed-out device wait."""
        _check(lib().plk_sync(self.h), self.h)

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        _check(lib().plk_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)), self.h)

    def close(self):
        if getattr(self, "h", None):
            lib().plk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------- kernel timing
    def profile(self, enable: bool = True):
        _check(lib().plk_profile_enable(self.h, int(enable)), self.h)

    def profile_collect(self) -> dict:
        """{stage: (total_ms, launches)} for the launches since the last collect."""
        n = ctypes.c_int()
        _check(lib().plk_profile_collect(self.h, ctypes.byref(n)), self.h)
        out = {}
        for i in range(n.value):
            nm, ms, cnt = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_int()
            _check(lib().plk_profile_get(self.h, i, ctypes.byref(nm), ctypes.byref(ms), ctypes.byref(cnt)))
            out[nm.value.decode()] = (ms.value, cnt.value)
        return out

    # ---------------------------------------------------------------- calls
    def amp_stats(self, slc: torch.Tensor, sum_pow: torch.Tensor | None = None,
                  sum_amp: torch.Tensor | None = None, accumulate: bool = False):
        _need(slc, torch.complex64, "slc", self.device)
        n, H, W = slc.shape
        if sum_pow is None:
            sum_pow = torch.empty((H, W), dtype=torch.float32, device=self.device)
        _need(sum_pow, torch.float32, "sum_pow", self.device)
        if sum_amp is not None:
            _need(sum_amp, torch.float32, "sum_amp", self.device)
        _check(lib().plk_amp_stats(self.h, _ptr(slc), n, H, W, _ptr(sum_pow), _ptr(sum_amp), int(accumulate)), self.h)
        return sum_pow, sum_amp

    def shp_select(self, sum_pow: torch.Tensor, n_eff: int, win, alpha: float = 1e-3,
                   mask: torch.Tensor | None = None, count: torch.Tensor | None = None):
        _need(sum_pow, torch.float32, "sum_pow", self.device)
        H, W = sum_pow.shape
        w = window(win)
        Ho, Wo = output_shape(H, W, w)
        nw = mask_words(w)
        if mask is None:
            mask = torch.empty((Ho, Wo, nw), dtype=torch.int64, device=self.device)
        if count is None:
            count = torch.empty((Ho, Wo), dtype=torch.int16, device=self.device)
        _need(mask, torch.int64, "mask", self.device)
        _need(count, torch.int16, "count", self.device)
        _check(lib().plk_shp_select(self.h, _ptr(sum_pow), int(n_eff), H, W, w, float(alpha), _ptr(mask),
                                    _ptr(count)), self.h)
        return mask, count

    def estimate_covariance(self, slc: torch.Tensor, win, mask: torch.Tensor, C: torch.Tensor | None = None,
                            precision: int = COV_FP32):
        _need(slc, torch.complex64, "slc", self.device)
        _need(mask, torch.int64, "mask", self.device)
        N, H, W = slc.shape
        w = window(win)
        Ho, Wo = output_shape(H, W, w)
        if C is None:
            C = torch.empty((Ho, Wo, N * (N + 1) // 2), dtype=torch.complex64, device=self.device)
        _need(C, torch.complex64, "C", self.device)
        _check(lib().plk_estimate_covariance(self.h, _ptr(slc), N, H, W, w, _ptr(mask), int(precision), _ptr(C)),
               self.h)
        return C

    def phase_link(self, C: torch.Tensor, N: int, ref: int, params: Params | None = None,
                   want_lambda: bool = True):
        _need(C, torch.complex64, "C", self.device)
        if C.shape[-1] != N * (N + 1) // 2:
            raise ValueError("C: last dimension must be N(N+1)/2")
        lead = tuple(C.shape[:-1])
        npx = 1
        for s in lead:
            npx *= s
        phase = torch.empty((N,) + lead, dtype=torch.float32, device=self.device)
        tcoh = torch.empty(lead, dtype=torch.float32, device=self.device)
        lam = torch.empty(lead, dtype=torch.float32, device=self.device) if want_lambda else None
        status = torch.empty(lead, dtype=torch.uint8, device=self.device)
        p = params if params is not None else default_params()
        _check(lib().plk_phase_link(self.h, _ptr(C), N, npx, int(ref), ctypes.byref(p), _ptr(phase), _ptr(tcoh),
                                    _ptr(lam), _ptr(status)), self.h)
        return {"phase": phase, "tcoh": tcoh, "lam": lam, "status": status}

    def phase_link_backward(self, slc: torch.Tensor, win, mask: torch.Tensor, ref: int, dphase: torch.Tensor,
                            params: Params | None = None, dslc: torch.Tensor | None = None) -> torch.Tensor:
        """Adjoint of coherence -> EMI -> referenced phase (mask frozen): the
        gradient dL/dRe z + j dL/dIm z of L = sum(dphase * phase)."""
        _need(slc, torch.complex64, "slc", self.device)
        _need(mask, torch.int64, "mask", self.device)
        _need(dphase, torch.float32, "dphase", self.device)
        N, H, W = slc.shape
        w = window(win)
        nbytes = ctypes.c_size_t()
        _check(lib().plk_backward_workspace_size(N, H, W, w, ctypes.byref(nbytes)))
        ws = torch.empty(max(1, nbytes.value), dtype=torch.uint8, device=self.device)
        if dslc is None:
            dslc = torch.empty_like(slc)
        p = params if params is not None else default_params()
        _check(lib().plk_phase_link_backward(self.h, _ptr(slc), N, H, W, w, _ptr(mask), int(ref), ctypes.byref(p),
                                             _ptr(dphase), _ptr(ws), nbytes.value, _ptr(dslc)), self.h)
        return dslc

    def shp_weight_gradient(self, slc: torch.Tensor, win, mask: torch.Tensor, ref: int, dphase: torch.Tensor,
                            params: Params | None = None, out: torch.Tensor | None = None) -> torch.Tensor:
        """Gradient [Ho, Wo, wy*wx] of L = sum(dphase * phase) with respect to
        real per-sample window weights, evaluated at the SHP mask."""
        _need(slc, torch.complex64, "slc", self.device)
        _need(mask, torch.int64, "mask", self.device)
        _need(dphase, torch.float32, "dphase", self.device)
        N, H, W = slc.shape
        w = window(win)
        Ho, Wo = output_shape(H, W, win)
        nbytes = ctypes.c_size_t()
        _check(lib().plk_backward_workspace_size(N, H, W, w, ctypes.byref(nbytes)))
        ws = torch.empty(max(1, nbytes.value), dtype=torch.uint8, device=self.device)
        if out is None:
            out = torch.empty((Ho, Wo, w.wy * w.wx), dtype=torch.float32, device=self.device)
        _need(out, torch.float32, "out", self.device)
        p = params if params is not None else default_params()
        _check(lib().plk_shp_weight_gradient(self.h, _ptr(slc), N, H, W, w, _ptr(mask), int(ref), ctypes.byref(p),
                                             _ptr(dphase), _ptr(ws), nbytes.value, _ptr(out)), self.h)
        return out

    def phase_uncertainty(self, slc: torch.Tensor, win, mask: torch.Tensor, ref: int, sigma2: float,
                          params: Params | None = None, out: torch.Tensor | None = None) -> torch.Tensor:
        """First-order standard deviation [N, Ho, Wo] of the linked phases under
        white circular noise of variance sigma2 on every sample (the adjoint)."""
        _need(slc, torch.complex64, "slc", self.device)
        _need(mask, torch.int64, "mask", self.device)
        N, H, W = slc.shape
        w = window(win)
        Ho, Wo = output_shape(H, W, win)
        nbytes = ctypes.c_size_t()
        _check(lib().plk_backward_workspace_size(N, H, W, w, ctypes.byref(nbytes)))
        ws = torch.empty(max(1, nbytes.value), dtype=torch.uint8, device=self.device)
        if out is None:
            out = torch.empty((N, Ho, Wo), dtype=torch.float32, device=self.device)
        _need(out, torch.float32, "out", self.device)
        p = params if params is not None else default_params()
        _check(lib().plk_phase_uncertainty(self.h, _ptr(slc), N, H, W, w, _ptr(mask), int(ref), ctypes.byref(p),
                                           float(sigma2), _ptr(ws), nbytes.value, _ptr(out)), self.h)
        return out

    def compress(self, slc: torch.Tensor, first_real: int, win, phase: torch.Tensor,
                 kappa: torch.Tensor | None = None):
        _need(slc, torch.complex64, "slc", self.device)
        _need(phase, torch.float32, "phase", self.device)
        N, H, W = slc.shape
        if kappa is None:
            kappa = torch.empty((H, W), dtype=torch.complex64, device=self.device)
        _need(kappa, torch.complex64, "kappa", self.device)
        _check(lib().plk_compress(self.h, _ptr(slc), N, int(first_real), H, W, window(win), _ptr(phase),
                                  _ptr(kappa)), self.h)
        return kappa

    def phase_similarity(self, phase: torch.Tensor, radius: int, out: torch.Tensor | None = None):
        """gamma_s [Ho, Wo] of linked phases [M, Ho, Wo] over a disk of `radius` output pixels."""
        _need(phase, torch.float32, "phase", self.device)
        M, Ho, Wo = phase.shape
        if out is None:
            out = torch.empty((Ho, Wo), dtype=torch.float32, device=self.device)
        _need(out, torch.float32, "gamma_s", self.device)
        if tuple(out.shape) != (Ho, Wo):
            raise ValueError("phase_similarity: output shape mismatch")
        _check(lib().plk_phase_similarity(self.h, _ptr(phase), M, Ho, Wo, int(radius), _ptr(out)), self.h)
        return out

    def invert_l1(self, unw: torch.Tensor, n_dates: int, pairs, rho: float = 1.0, iters: int = 50,
                  residual: bool = False):
        """x [n_dates-1, ...] (and b - A x) of unwrapped phases unw [n_ifg, ...] by L1 ADMM."""
        _need(unw, torch.float32, "unw", self.device)
        n_ifg = unw.shape[0]
        npx = unw[0].numel() if n_ifg else 0
        pr = (ctypes.c_int32 * (2 * len(pairs)))(*[int(v) for ab in pairs for v in ab])
        if len(pairs) != n_ifg:
            raise ValueError("invert_l1: one pair per interferogram plane")
        x = torch.empty((n_dates - 1,) + tuple(unw.shape[1:]), dtype=torch.float32, device=self.device)
        r = torch.empty_like(unw) if residual else None
        _check(lib().plk_invert_l1(self.h, _ptr(unw), int(n_dates), ctypes.cast(pr, ctypes.c_void_p), n_ifg, npx,
                                   float(rho), int(iters), _ptr(x), _ptr(r)), self.h)
        return (x, r) if residual else x

    def ps_regrid(self, slc: torch.Tensor, first_real: int, win, sum_pow: torch.Tensor, sum_amp: torch.Tensor,
                  n_eff: int, ref: int, da_max: float, phase: torch.Tensor, status: torch.Tensor):
        """PS cells of phase [N - first_real, Ho, Wo] and status [Ho, Wo] take
        the phases of their lowest-D_A persistent scatterer (in place)."""
        _need(slc, torch.complex64, "slc", self.device)
        _need(sum_pow, torch.float32, "sum_pow", self.device)
        _need(sum_amp, torch.float32, "sum_amp", self.device)
        _need(phase, torch.float32, "phase", self.device)
        _need(status, torch.uint8, "status", self.device)
        N, H, W = slc.shape
        Ho, Wo = output_shape(H, W, win)
        if tuple(phase.shape) != (N - first_real, Ho, Wo) or tuple(status.shape) != (Ho, Wo) or \
                tuple(sum_pow.shape) != (H, W) or tuple(sum_amp.shape) != (H, W):
            raise ValueError("ps_regrid: shape mismatch")
        _check(lib().plk_ps_regrid(self.h, _ptr(slc), N, int(first_real), H, W, window(win), _ptr(sum_pow),
                                   _ptr(sum_amp), int(n_eff), int(ref), float(da_max), _ptr(phase), _ptr(status)),
               self.h)
        return phase, status


class PhaseLinkFn(torch.autograd.Function):
    """phase = coherence -> EMI -> referenced phase of a stack, with the SHP
    mask given (frozen); differentiable in the stack.  The gradient follows
    torch's convention for complex inputs (dL/dRe z + j dL/dIm z for real L)."""

    @staticmethod
    def forward(fctx, slc, mask, win, ref, plk_ctx, params=None):
        C = plk_ctx.estimate_covariance(slc, win, mask)
        N = slc.shape[0]
        p = params if params is not None else default_params()
        p = Params.from_buffer_copy(p)
        p.fp64_resolve = 0  # the adjoint differentiates the single-precision solve
        out = plk_ctx.phase_link(C, N, ref, p)
        fctx.save_for_backward(slc, mask)
        fctx.win, fctx.ref, fctx.plk_ctx, fctx.params = win, ref, plk_ctx, p
        return out["phase"]

    @staticmethod
    def backward(fctx, dphase):
        slc, mask = fctx.saved_tensors
        g = fctx.plk_ctx.phase_link_backward(slc, fctx.win, mask, fctx.ref, dphase.contiguous().float(), fctx.params)
        return g, None, None, None, None, None


class Batch:
    """plk_batch: S1-S6 for many independent stacks (uneven N, one window), run
    as one recorded CUDA graph after a first, tuning, call.  Outputs per stack:
    phase [N][Ho][Wo], tcoh and status [Ho][Wo] (allocated here)."""

    def __init__(self, ctx: Context, stacks, win, params: Params | None = None, refs=None):
        self.ctx = ctx
        self.win = window(win)
        self.stacks = list(stacks)  # keep the inputs alive
        refs = refs or [0] * len(self.stacks)
        self.out = []
        descs = (StackDesc * len(self.stacks))()
        for i, (z, ref) in enumerate(zip(self.stacks, refs)):
            _need(z, torch.complex64, f"stacks[{i}]", ctx.device)
            N, H, W = z.shape
            Ho, Wo = output_shape(H, W, self.win)
            o = {"phase": torch.empty((N, Ho, Wo), device=ctx.device),
                 "tcoh": torch.empty((Ho, Wo), device=ctx.device),
                 "status": torch.empty((Ho, Wo), dtype=torch.uint8, device=ctx.device)}
            self.out.append(o)
            descs[i] = StackDesc(z.data_ptr(), N, H, W, int(ref), o["phase"].data_ptr(), o["tcoh"].data_ptr(),
                                 o["status"].data_ptr())
        p = params if params is not None else default_params()
        h = ctypes.c_void_p()
        _check(lib().plk_batch_create(ctx.h, ctypes.cast(descs, ctypes.c_void_p), len(self.stacks), self.win,
                                      ctypes.byref(p), ctypes.byref(h)), ctx.h)
        self.h = h

    def run(self):
        _check(lib().plk_batch_run(self.ctx.h, self.h), self.ctx.h)
        return self.out

    def info(self) -> dict:
        g, s, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().plk_batch_info(self.h, ctypes.byref(g), ctypes.byref(s), ctypes.byref(n)))
        return {"graph_built": g.value, "streams": s.value, "nodes": n.value}

    def close(self):
        if getattr(self, "h", None):
            lib().plk_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tuned_schedule(ctx: Context, N: int, win) -> dict:
    ty, tx, np_ = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().plk_tuned_schedule(ctx.h, int(N), window(win), ctypes.byref(ty), ctypes.byref(tx),
                                    ctypes.byref(np_)), ctx.h)
    return {"cov_tile": (ty.value, tx.value), "emi_lanes": np_.value}


class State:
    """plk_state: the sequential chain (kappa ring, merged sums, counters)."""

    def __init__(self, ctx: Context, H: int, W: int, win, K_max: int, M_max: int, _handle=None):
        self.ctx = ctx
        self.H, self.W = H, W
        self.win = window(win)
        self.K_max, self.M_max = K_max, M_max
        if _handle is None:
            h = ctypes.c_void_p()
            _check(lib().plk_state_create(ctx.h, H, W, self.win, K_max, M_max, ctypes.byref(h)), ctx.h)
            self.h = h
        else:
            self.h = _handle
        self.Ho, self.Wo = output_shape(H, W, self.win)

    @classmethod
    def load(cls, ctx: Context, path: str, M_max: int):
        h = ctypes.c_void_p()
        _check(lib().plk_state_load(ctx.h, os.fsencode(path), int(M_max), ctypes.byref(h)), ctx.h)
        # read the geometry back from the file header
        import struct
        with open(path, "rb") as f:
            f.read(8)
            hdr = struct.unpack("<10i", f.read(40))
        return cls(ctx, hdr[0], hdr[1], hdr[2:6], hdr[6], M_max, _handle=h)

    def save(self, path: str):
        _check(lib().plk_state_save(self.ctx.h, self.h, os.fsencode(path)), self.ctx.h)

    def reset(self):
        _check(lib().plk_state_reset(self.h))

    def info(self) -> dict:
        k, n, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().plk_state_info(self.h, ctypes.byref(k), ctypes.byref(n), ctypes.byref(s)))
        return {"K_used": k.value, "n_eff": n.value, "steps": s.value}

    def weights(self) -> tuple[float, float]:
        """(W1, W2): sums of the merged image weights and of their squares."""
        w1, w2 = ctypes.c_double(), ctypes.c_double()
        _check(lib().plk_state_weights(self.h, ctypes.byref(w1), ctypes.byref(w2)))
        return w1.value, w2.value

    def kappa_ptr(self, i: int) -> int:
        p = ctypes.c_void_p()
        _check(lib().plk_state_kappa(self.h, int(i), ctypes.byref(p)))
        return p.value

    def kappa(self, i: int) -> torch.Tensor:
        """Copy of compressed SLC i of the ring (0 = oldest)."""
        return _copy_from_ptr(self.kappa_ptr(i), (self.H, self.W), torch.complex64, self.ctx)

    def sum_pow(self) -> torch.Tensor:
        p, a = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().plk_state_sums(self.h, ctypes.byref(p), ctypes.byref(a)))
        return _copy_from_ptr(p.value, (self.H, self.W), torch.float32, self.ctx)

    def step(self, new_slc: torch.Tensor, params: Params | None = None, out: dict | None = None,
             want_count: bool = True) -> dict:
        _need(new_slc, torch.complex64, "new_slc", self.ctx.device)
        M = new_slc.shape[0]
        if tuple(new_slc.shape[1:]) != (self.H, self.W):
            raise ValueError("new_slc: wrong image size")
        dev = self.ctx.device
        if out is None:
            out = {
                "phase": torch.empty((M, self.Ho, self.Wo), dtype=torch.float32, device=dev),
                "tcoh": torch.empty((self.Ho, self.Wo), dtype=torch.float32, device=dev),
                "status": torch.empty((self.Ho, self.Wo), dtype=torch.uint8, device=dev),
                "count": torch.empty((self.Ho, self.Wo), dtype=torch.int16, device=dev) if want_count else None,
            }
        p = params if params is not None else default_params()
        _check(lib().plk_ministack_step(self.ctx.h, self.h, _ptr(new_slc), M, ctypes.byref(p), _ptr(out["phase"]),
                                        _ptr(out["tcoh"]), _ptr(out["status"]), _ptr(out.get("count"))),
               self.ctx.h)
        return out

    def _host_outputs(self, M: int, out: dict | None, want_count: bool) -> dict:
        if out is None:
            pin = torch.cuda.is_available()
            out = {
                "phase": torch.empty((M, self.Ho, self.Wo), dtype=torch.float32, pin_memory=pin),
                "tcoh": torch.empty((self.Ho, self.Wo), dtype=torch.float32, pin_memory=pin),
                "status": torch.empty((self.Ho, self.Wo), dtype=torch.uint8, pin_memory=pin),
                "count": torch.empty((self.Ho, self.Wo), dtype=torch.int16, pin_memory=pin) if want_count else None,
            }
        for key in ("phase", "tcoh", "status", "count"):
            t = out.get(key)
            if t is not None and (t.device.type != "cpu" or not t.is_contiguous()):
                raise TypeError(f"{key}: expected a contiguous CPU tensor")
        return out

    def enable_host_io(self):
        """Allocate the device staging of step_host (plk_state_enable_host_io)."""
        _check(lib().plk_state_enable_host_io(self.ctx.h, self.h), self.ctx.h)

    def step_host(self, new_slc: torch.Tensor, params: Params | None = None, out: dict | None = None,
                  want_count: bool = False) -> dict:
        """One step from host memory (plk_ministack_step_host): new_slc a CPU
        complex64 tensor [M, H, W] (pinned, so that its copy overlaps the
        previous step's compute), outputs written to CPU tensors.  Needs
        enable_host_io() first.  Asynchronous: call ctx.sync() before reading
        the outputs or reusing new_slc."""
        if new_slc.device.type != "cpu" or new_slc.dtype != torch.complex64 or not new_slc.is_contiguous():
            raise TypeError("new_slc: expected a contiguous CPU complex64 tensor")
        M = new_slc.shape[0]
        if tuple(new_slc.shape[1:]) != (self.H, self.W):
            raise ValueError("new_slc: wrong image size")
        out = self._host_outputs(M, out, want_count)
        p = params if params is not None else default_params()
        _check(lib().plk_ministack_step_host(self.ctx.h, self.h, ctypes.c_void_p(new_slc.data_ptr()), M,
                                             ctypes.byref(p), _ptr(out["phase"]), _ptr(out["tcoh"]),
                                             _ptr(out["status"]), _ptr(out.get("count"))), self.ctx.h)
        return out

    def enable_host_io_ci16(self):
        """Allocate the staging of step_host_ci16 (plk_state_enable_host_io_ci16)."""
        _check(lib().plk_state_enable_host_io_ci16(self.ctx.h, self.h), self.ctx.h)

    def step_host_ci16(self, new_slc: torch.Tensor, params: Params | None = None, out: dict | None = None,
                       want_count: bool = False) -> dict:
        """step_host with complex 16-bit samples (plk_ministack_step_host_ci16):
        new_slc a CPU int16 tensor [M, H, W, 2] (re, im; pinned for overlap).
        Needs enable_host_io_ci16() first; asynchronous like step_host."""
        if new_slc.device.type != "cpu" or new_slc.dtype != torch.int16 or not new_slc.is_contiguous():
            raise TypeError("new_slc: expected a contiguous CPU int16 tensor")
        M = new_slc.shape[0]
        if tuple(new_slc.shape[1:]) != (self.H, self.W, 2):
            raise ValueError("new_slc: expected shape [M, H, W, 2]")
        out = self._host_outputs(M, out, want_count)
        p = params if params is not None else default_params()
        _check(lib().plk_ministack_step_host_ci16(self.ctx.h, self.h, ctypes.c_void_p(new_slc.data_ptr()), M,
                                                  ctypes.byref(p), _ptr(out["phase"]), _ptr(out["tcoh"]),
                                                  _ptr(out["status"]), _ptr(out.get("count"))), self.ctx.h)
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().plk_state_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DevArray:
    """Minimal __cuda_array_interface__ view of a library-owned device buffer."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


_TYPESTR = {torch.complex64: "<c8", torch.float32: "<f4"}


def _copy_from_ptr(ptr: int, shape, dtype, ctx: Context) -> torch.Tensor:
    """Copy of a library-owned device buffer into a new tensor (stream-ordered)."""
    view = torch.as_tensor(_DevArray(ptr, shape, _TYPESTR[dtype]), device=ctx.device)
    with torch.cuda.stream(ctx.stream):
        return view.clone()


_default_ctx: dict = {}


def context(device=None) -> Context:
    """Process-wide default context for `device` on its current stream."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    key = (dev.index, torch.cuda.current_stream(dev).cuda_stream)
    if key not in _default_ctx:
        _default_ctx[key] = Context(dev)
    return _default_ctx[key]


# Module-level functions with the ABI's names, on the default context.
def amp_stats(slc, sum_pow=None, sum_amp=None, accumulate=False):
    return context(slc.device).amp_stats(slc, sum_pow, sum_amp, accumulate)


def shp_select(sum_pow, n_eff, win, alpha=1e-3):
    return context(sum_pow.device).shp_select(sum_pow, n_eff, win, alpha)


def estimate_covariance(slc, win, mask):
    return context(slc.device).estimate_covariance(slc, win, mask)


def phase_link(C, N, ref, params=None):
    return context(C.device).phase_link(C, N, ref, params)


def compress(slc, first_real, win, phase):
    return context(slc.device).compress(slc, first_real, win, phase)


def invert_l1(unw, n_dates, pairs, rho=1.0, iters=50, residual=False):
    return context(unw.device).invert_l1(unw, n_dates, pairs, rho, iters, residual)


def phase_similarity(phase, radius, out=None):
    return context(phase.device).phase_similarity(phase, radius, out)


def ps_regrid(slc, first_real, win, sum_pow, sum_amp, n_eff, ref, da_max, phase, status):
    return context(slc.device).ps_regrid(slc, first_real, win, sum_pow, sum_amp, n_eff, ref, da_max, phase, status)


def ministack_step(state: State, new_slc, params=None):
    return state.step(new_slc, params)
