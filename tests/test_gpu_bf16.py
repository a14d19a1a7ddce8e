"""Reduced-precision coherence (PLK_COV_BF16): the samples are rounded to
bfloat16 and the products summed in single precision on the tensor cores.

Two bars:
- Exactness of the contraction: the oracle fed the same bfloat16-rounded
  samples (rounded here, on the CPU, round-to-nearest-even) gives the same
  coherence within single-precision accumulation error.
- Accuracy of the mode against the full-precision oracle: coherence and linked
  phases within the stated, measured bounds (p50 / p99 / max printed)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_12051_gb300 import synth
from parity_util import to_np, wrapped_diff

pytestmark = pytest.mark.gpu

# Bounds of the bfloat16 mode against the FP64 oracle on the unrounded samples
# (burst-shaped 90x300 stack, N = 15, 11x5 window, strides 6x3), each at most
# twice the measured value: coherence max error 3.9e-3; linked phase p50
# 1.10e-3, p99 3.00e-3, max 7.63e-3 rad.
BF16_COH_MAX = 7.8e-3     # max |C_bf16 - C| over all entries
BF16_PHASE_P99 = 6e-3     # rad, 99th percentile of the linked-phase error
BF16_PHASE_P50 = 2.2e-3   # rad, median
BF16_PHASE_MAX = 1.5e-2   # rad, largest


@pytest.fixture(scope="module")
def plk():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2511_12051_gb300 import build, plk as _plk
    build.build()
    return _plk


@pytest.fixture(scope="module")
def ctx(plk):
    return plk.Context("cuda:0")


def round_bf16(x: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def round_stack(z: np.ndarray) -> np.ndarray:
    out = np.empty_like(z)
    out.real = round_bf16(z.real.astype(np.float32))
    out.imag = round_bf16(z.imag.astype(np.float32))
    return out


def test_round_bf16_helper():
    # bfloat16 keeps 8 significand bits: the spacing just above 1 is 2^-7.
    v = np.array([1.0, -2.5, 0.0,
                  1.0 + 2 ** -8,        # tie between 1 and 1 + 2^-7: to even -> 1
                  1.0 + 3 * 2 ** -8,    # tie between 1 + 2^-7 and 1 + 2^-6: to even -> 1 + 2^-6
                  1.0 + 2 ** -9,        # below the half spacing -> 1
                  1.0 + 3 * 2 ** -9],   # above the half spacing -> 1 + 2^-7
                 dtype=np.float32)
    want = np.array([1.0, -2.5, 0.0, 1.0, 1.0 + 2 ** -6, 1.0, 1.0 + 2 ** -7], dtype=np.float32)
    assert np.array_equal(round_bf16(v), want)


def _case(cfg, N, H, W, win, seed):
    spec = synth.config_spec(cfg, N=N, H=H, W=W, seed=seed)
    z = synth.generate(spec).numpy()
    P, _ = oracle.amp_stats(z)
    m, cnt = oracle.shp_select(P, win, np.float32(oracle.glrt_threshold(1e-3, N)))
    return z, m, cnt


@pytest.mark.parametrize("cfg,N,win", [(1, 15, (5, 11, 3, 6)), (0, 10, (5, 11, 1, 1)), (0, 2, (3, 5, 1, 1)),
                                       (0, 16, (5, 11, 3, 6)), (0, 21, (5, 11, 3, 6)), (1, 32, (5, 11, 3, 6)),
                                       (0, 9, (19, 37, 3, 6))])
def test_bf16_contraction_matches_rounded_oracle(ctx, plk, cfg, N, win):
    z, m, cnt = _case(cfg, N, 50, 97, win, seed=21)
    C_o = oracle.covariance(round_stack(z), win, m)
    C_g = to_np(ctx.estimate_covariance(torch.from_numpy(z).cuda(), win, torch.from_numpy(m.view(np.int64)).cuda(),
                                        precision=plk.COV_BF16))
    ok = cnt > 0
    assert np.all(np.isnan(C_g[~ok].real))
    err = np.abs(C_g[ok] - C_o[ok])
    assert err.max() < 2e-5, err.max()


def test_bf16_mode_bounds(ctx, plk):
    """Coherence and linked-phase error of the bfloat16 mode against the
    full-precision oracle on a burst-shaped stack; the bounds are stated
    above and in the design notes."""
    N, win = 15, (5, 11, 3, 6)
    z, m, cnt = _case(1, N, 90, 300, win, seed=5)
    C_o = oracle.covariance(z, win, m)
    zg = torch.from_numpy(z).cuda()
    mg = torch.from_numpy(m.view(np.int64)).cuda()
    C_b = ctx.estimate_covariance(zg, win, mg, precision=plk.COV_BF16)
    ok = cnt > 0
    coh_err = np.abs(to_np(C_b)[ok] - C_o[ok])
    # phases: oracle on the FP64 coherence vs the GPU solve of the bf16 coherence
    o = oracle.phase_link(C_o[ok], N, 0)
    Cb = C_b.reshape(-1, C_b.shape[-1])[torch.from_numpy(ok.ravel()).cuda()].contiguous()
    g = ctx.phase_link(Cb, N, 0)
    st_g = to_np(g["status"])
    evd_o, evd_g = o["status"] == plk.PX_EVD, st_g == plk.PX_EVD
    keep = (o["gap"] > 1e-6 * np.abs(np.nan_to_num(o["lam"], nan=1.0))) & (evd_o == evd_g)
    e = wrapped_diff(to_np(g["phase"]), o["phase"])[:, keep].max(axis=0)
    p50, p99, mx = np.percentile(e, 50), np.percentile(e, 99), e.max()
    print(f"bf16 coherence max err {coh_err.max():.3e}; phase err p50 {p50:.2e} p99 {p99:.2e} max {mx:.2e} rad "
          f"over {keep.sum()} of {ok.sum()} px; EMI/EVD branch disagreements {np.sum(evd_o != evd_g)}")
    assert coh_err.max() < BF16_COH_MAX
    assert p50 < BF16_PHASE_P50
    assert p99 < BF16_PHASE_P99
    assert mx < BF16_PHASE_MAX


def test_bf16_ministack_step_runs_and_tracks_fp32(ctx, plk):
    """The whole step in bfloat16 mode, against the same step in FP32."""
    from paper_2511_12051_gb300 import synth as s
    spec = s.config_spec(1, H=96, W=300, seed=9)
    z = s.generate(spec).cuda()
    N = z.shape[0]
    outs = {}
    for prec in (plk.COV_FP32, plk.COV_BF16):
        st = plk.State(ctx, spec.H, spec.W, (5, 11, 3, 6), K_max=6, M_max=N)
        outs[prec] = st.step(z, plk.default_params(cov_precision=prec))
        st.close()
    a, b = outs[plk.COV_FP32], outs[plk.COV_BF16]
    live = to_np(a["status"]) != plk.PX_NODATA
    d = wrapped_diff(to_np(a["phase"]), to_np(b["phase"]))[:, live]
    assert np.percentile(d.max(axis=0), 50) < BF16_PHASE_P50


def test_bf16_rejects_large_n(ctx, plk):
    z = torch.zeros((33, 8, 8), dtype=torch.complex64, device="cuda")
    mask = torch.zeros((8, 8, 1), dtype=torch.int64, device="cuda")
    with pytest.raises(RuntimeError):
        ctx.estimate_covariance(z, (3, 3, 1, 1), mask, precision=plk.COV_BF16)
