"""FP64 CPU oracle for the sequential phase-linking hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2511_12051_gb300``) and never imports it.

The arithmetic lives in ``plk_oracle.c`` (plain C, double precision, one
pixel at a time, each function citing the section of the paper it follows);
this module only builds it with gcc, marshals numpy arrays and runs the
mini-stack bookkeeping of Sec. II-B in ``chain.py``.  The phase cosine
similarity of Sec. III-C is plain numpy in ``similarity.py``, the L1 network
inversion by ADMM (Sec. III-E, Appendix) numpy and scipy in ``inversion.py``.

Function pins (tests/test_oracle_*.py) tie every routine to something other
than itself: closed forms, invariants, brute force on tiny inputs, a library
F-quantile and a library eigensolver.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "plk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libplk_oracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: no fused multiply-add, so the single-precision power sums
# and threshold products round exactly as written (they decide mask bits).
CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile plk_oracle.c into oracle/_build/libplk_oracle.so (gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64, f64, f32 = ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_float
            lib.orc_amp_stats.argtypes = [P, i32, i32, i32, P, P, i32]
            lib.orc_glrt_threshold.argtypes = [f64, i32]
            lib.orc_glrt_threshold.restype = f64
            lib.orc_shp_select.argtypes = [P, i32, i32, i32, i32, i32, i32, f32, P, P]
            lib.orc_covariance.argtypes = [P, i32, i32, i32, i32, i32, i32, i32, P, P]
            lib.orc_phase_link.argtypes = [P, i32, i64, i32, f64, P, P, P, P, P, P]
            lib.orc_amp_dispersion.argtypes = [P, P, i64, i32, P]
            lib.orc_ps_regrid.argtypes = [P, i32, i32, i32, i32, i32, i32, P, P, i32, i32, f32, P, P, i32]
            lib.orc_ps_compress.argtypes = [P, i32, i32, i32, i32, P, P, i32, i32, f32, i32, P]
            lib.orc_temporal_coherence.argtypes = [i32, P, P]
            lib.orc_temporal_coherence.restype = f64
            lib.orc_compress.argtypes = [P, i32, i32, i32, i32, i32, i32, P, P]
            lib.orc_num_threads.restype = i32
            lib.orc_set_num_threads.argtypes = [i32]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def ntri(N: int) -> int:
    return N * (N + 1) // 2


def out_shape(H: int, W: int, window) -> tuple[int, int]:
    wy, wx, sy, sx = window
    return H // sy, W // sx


def amp_stats(slc: np.ndarray, sum_pow: np.ndarray | None = None,
              sum_amp: np.ndarray | None = None, accumulate: bool = False):
    """Per-pixel power and amplitude sums over the real SLCs (single precision)."""
    slc = np.ascontiguousarray(slc, dtype=np.complex64)
    n, H, W = slc.shape
    if sum_pow is None:
        sum_pow = np.zeros((H, W), np.float32)
    if sum_amp is None:
        sum_amp = np.zeros((H, W), np.float32)
    assert sum_pow.dtype == np.float32 and sum_pow.flags.c_contiguous
    _load().orc_amp_stats(_ptr(slc), n, H, W, _ptr(sum_pow), _ptr(sum_amp), int(accumulate))
    return sum_pow, sum_amp


def glrt_threshold(alpha: float, n: int) -> float:
    """c = F^{-1}_{2n,2n}(1 - alpha/2) by bisection on the incomplete beta."""
    return float(_load().orc_glrt_threshold(float(alpha), int(n)))


def shp_select(sum_pow: np.ndarray, window, c: float):
    """SHP masks [Ho, Wo, nwords] uint64 and counts [Ho, Wo] uint16."""
    wy, wx, sy, sx = window
    P = np.ascontiguousarray(sum_pow, dtype=np.float32)
    H, W = P.shape
    Ho, Wo = H // sy, W // sx
    nw = (wy * wx + 63) // 64
    mask = np.zeros((Ho, Wo, nw), np.uint64)
    count = np.zeros((Ho, Wo), np.uint16)
    _load().orc_shp_select(_ptr(P), H, W, wy, wx, sy, sx, np.float32(c), _ptr(mask), _ptr(count))
    return mask, count


def covariance(z: np.ndarray, window, mask: np.ndarray) -> np.ndarray:
    """Coherence, packed upper triangle, complex128 [Ho, Wo, N(N+1)/2]."""
    wy, wx, sy, sx = window
    z = np.ascontiguousarray(z, dtype=np.complex128)
    N, H, W = z.shape
    Ho, Wo = H // sy, W // sx
    mask = np.ascontiguousarray(mask, dtype=np.uint64)
    assert mask.shape[:2] == (Ho, Wo)
    C = np.zeros((Ho, Wo, ntri(N)), np.complex128)
    _load().orc_covariance(_ptr(z), N, H, W, wy, wx, sy, sx, _ptr(mask), _ptr(C))
    return C


def phase_link(C: np.ndarray, N: int, ref: int, beta: float = 0.0, cond: bool = False) -> dict:
    """EMI phase linking of packed coherences C [..., N(N+1)/2].

    Returns a dict with phase [N, ...], tcoh, lam, gap, condG (or None), status.
    """
    lead = C.shape[:-1]
    assert C.shape[-1] == ntri(N)
    Cf = np.ascontiguousarray(C.reshape(-1, ntri(N)), dtype=np.complex128)
    npx = Cf.shape[0]
    phase = np.zeros((N, npx), np.float64)
    tcoh = np.zeros(npx, np.float64)
    lam = np.zeros(npx, np.float64)
    gap = np.zeros(npx, np.float64)
    condG = np.zeros(npx, np.float64) if cond else None
    status = np.zeros(npx, np.uint8)
    _load().orc_phase_link(_ptr(Cf), N, npx, int(ref), float(beta), _ptr(phase), _ptr(tcoh),
                           _ptr(lam), _ptr(gap), _ptr(condG), _ptr(status))
    return {
        "phase": phase.reshape((N,) + lead),
        "tcoh": tcoh.reshape(lead),
        "lam": lam.reshape(lead),
        "gap": gap.reshape(lead),
        "condG": None if condG is None else condG.reshape(lead),
        "status": status.reshape(lead),
    }


def temporal_coherence(Cpacked: np.ndarray, phihat: np.ndarray) -> float:
    """Eq. (temporal-coherence) for one pixel: packed C and linked phases."""
    N = len(phihat)
    Cp = np.ascontiguousarray(Cpacked, dtype=np.complex128)
    ph = np.ascontiguousarray(phihat, dtype=np.float64)
    return float(_load().orc_temporal_coherence(N, _ptr(Cp), _ptr(ph)))


def compress(z: np.ndarray, first_real: int, window, phase: np.ndarray) -> np.ndarray:
    """Compressed SLC kappa [H, W] complex128 from the real SLCs of z."""
    wy, wx, sy, sx = window
    z = np.ascontiguousarray(z, dtype=np.complex128)
    N, H, W = z.shape
    ph = np.ascontiguousarray(phase, dtype=np.float64)
    assert ph.shape == (N, H // sy, W // sx)
    kappa = np.zeros((H, W), np.complex128)
    _load().orc_compress(_ptr(z), N, int(first_real), H, W, sy, sx, _ptr(ph), _ptr(kappa))
    return kappa


# Status code of an output cell that takes a PS phase (the phase-linking codes
# are 0-4: EMI, EMI re-solved in double precision, EVD, no data, not converged).
PS_STATUS = 5


def amp_dispersion(sum_pow: np.ndarray, sum_amp: np.ndarray, n: int) -> np.ndarray:
    """D_A = sigma_A / mu_A = sqrt(n SP - SA^2) / SA per pixel from the merged sums (single precision;
    NaN where SA <= 0)."""
    sp = np.ascontiguousarray(sum_pow, dtype=np.float32)
    sa = np.ascontiguousarray(sum_amp, dtype=np.float32)
    assert sp.shape == sa.shape
    da = np.empty(sp.shape, np.float32)
    _load().orc_amp_dispersion(_ptr(sp), _ptr(sa), sp.size, int(n), _ptr(da))
    return da


def ps_regrid(z: np.ndarray, first_real: int, window, sum_pow: np.ndarray, sum_amp: np.ndarray, n: int,
              ref: int, da_max: float, phase: np.ndarray, status: np.ndarray):
    """PS cells of the output grid take the phase of their lowest-D_A PS.

    phase [N - first_real, Ho, Wo] and status [Ho, Wo] are copied and returned
    updated (float64, uint8)."""
    wy, wx, sy, sx = window
    z = np.ascontiguousarray(z, dtype=np.complex128)
    N, H, W = z.shape
    Ho, Wo = H // sy, W // sx
    ph = np.array(phase, dtype=np.float64, order="C", copy=True)
    st = np.array(status, dtype=np.uint8, order="C", copy=True)
    assert ph.shape == (N - first_real, Ho, Wo) and st.shape == (Ho, Wo)
    sp = np.ascontiguousarray(sum_pow, dtype=np.float32)
    sa = np.ascontiguousarray(sum_amp, dtype=np.float32)
    assert sp.shape == (H, W) and sa.shape == (H, W)
    _load().orc_ps_regrid(_ptr(z), N, int(first_real), H, W, sy, sx, _ptr(sp), _ptr(sa), int(n), int(ref),
                          np.float32(da_max), _ptr(ph), _ptr(st), PS_STATUS)
    return ph, st


def ps_compress(z: np.ndarray, first_real: int, sum_pow: np.ndarray, sum_amp: np.ndarray, n: int, ref: int,
                da_max: float, kappa: np.ndarray, shift: int = -1) -> np.ndarray:
    """Compressed SLC with every PS pixel compressed on its own phases (a copy of kappa)."""
    z = np.ascontiguousarray(z, dtype=np.complex128)
    N, H, W = z.shape
    k = np.array(kappa, dtype=np.complex128, order="C", copy=True)
    assert k.shape == (H, W)
    sp = np.ascontiguousarray(sum_pow, dtype=np.float32)
    sa = np.ascontiguousarray(sum_amp, dtype=np.float32)
    _load().orc_ps_compress(_ptr(z), N, int(first_real), H, W, _ptr(sp), _ptr(sa), int(n), int(ref),
                            np.float32(da_max), int(shift), _ptr(k))
    return k


from .chain import OracleChain, ministack  # noqa: E402,F401
from .similarity import disk_offsets, nearest3_pairs, phase_similarity  # noqa: E402,F401
from .inversion import incidence, l1_invert, soft_threshold  # noqa: E402,F401
from .weights import mask_weights, weighted_coherence, window_samples  # noqa: E402,F401
from .decay import (decay_weights, effective_looks, glrt_threshold_real, merge_group, merge_group_f32,  # noqa: E402,F401
                    merged_mean_variance, step_weights, weight_sums)
