"""Helpers shared by the GPU parity tests (comparison only, no method arithmetic)."""
import numpy as np
import torch

PHASE_TOL = 1e-4   # rad, single precision vs the FP64 oracle
TCOH_TOL = 1e-5
# Relative eigengap (lambda_2 - lambda_1) / |lambda_1| below which the
# eigenvector is not unique (several answers are correct): such pixels are left
# out of phase parity and counted; gamma_t is still compared.
GAP_MIN = 1e-9


def wrapped_diff(a, b):
    return np.abs(np.angle(np.exp(1j * (np.asarray(a, np.float64) - np.asarray(b, np.float64)))))


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy()


def mask_np(t: torch.Tensor) -> np.ndarray:
    return to_np(t).view(np.uint64)


def count_np(t: torch.Tensor) -> np.ndarray:
    return to_np(t).view(np.uint16)


def phase_report(gpu_phase, orc_phase, valid=None):
    d = wrapped_diff(gpu_phase, orc_phase)
    if valid is not None:
        d = d[..., valid] if d.ndim > valid.ndim else d[valid]
    d = d[np.isfinite(d)]
    if d.size == 0:
        return {"max": 0.0, "p99": 0.0, "n": 0}
    return {"max": float(d.max()), "p99": float(np.percentile(d, 99)), "n": int(d.size)}


def write_state_file(path, chain, M_max=None):
    """Write an oracle chain's state in the library's checkpoint format
    (magic, int32 header, for format 2 the weight sums W1, W2 as float64, ring
    oldest..newest as complex64, power and amplitude sums as float32).  Format
    1 (equal weights) unless the chain decays its image weights."""
    H, W = chain.H, chain.W
    wy, wx, sy, sx = chain.window
    hdr = np.array([H, W, wy, wx, sy, sx, chain.K_max, len(chain.ring), chain.n, 0], np.int32)
    decaying = getattr(chain, "decay", 1.0) != 1.0
    with open(path, "wb") as f:
        f.write(b"PLKSTAT2" if decaying else b"PLKSTAT1")
        f.write(hdr.tobytes())
        if decaying:
            f.write(np.array(chain.wsum if chain.wsum is not None else (0.0, 0.0), np.float64).tobytes())
        for k in chain.ring:
            f.write(np.ascontiguousarray(k, np.complex64).tobytes())
        f.write(np.ascontiguousarray(chain.sum_pow, np.float32).tobytes())
        f.write(np.ascontiguousarray(chain.sum_amp, np.float32).tobytes())


def clear_of_degenerate(o, live):
    """Live pixels whose smallest eigenvalue is separated (GAP_MIN), and how
    many live pixels were left out."""
    lam = np.abs(np.nan_to_num(np.asarray(o["lam"], np.float64), nan=1.0))
    clear = live & (np.asarray(o["gap"]) > GAP_MIN * lam)
    return clear, int(np.sum(live) - np.sum(clear))
