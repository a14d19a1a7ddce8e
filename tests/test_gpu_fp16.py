"""Half-precision coherence (PLK_COV_FP16): per output tile the samples are
scaled by one power of two (largest component into [2^14, 2^15)), rounded to
half precision and the products summed in single precision on the tensor
cores; the scale cancels in C_ik = S_ik / sqrt(S_ii S_kk).

Bars:
- Exactness of the contraction: the oracle fed the samples rounded to 11
  significant bits (round to nearest even; what half precision keeps inside its
  range, which the scaling guarantees here) gives the same coherence within
  single-precision accumulation error.
- The scaling: inputs multiplied by 2^12 or 2^-20 give bit-identical
  coherence; inputs multiplied by 1e6 (far beyond half precision's range)
  stay finite and accurate.
- Accuracy of the mode against the FP64 oracle on the unrounded samples:
  measured, with stated bounds (p50 / p99 / max printed)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_12051_gb300 import synth
from parity_util import to_np, wrapped_diff

pytestmark = pytest.mark.gpu

# Bounds at most twice the measured values (burst-shaped 90x300 stack, N = 15,
# 11x5, strides 6x3): coherence max error 4.0e-4; phase p50 1.36e-4, p99
# 3.72e-4, max 5.91e-4 rad.
FP16_COH_MAX = 8e-4      # max |C_fp16 - C| over all entries
FP16_PHASE_P99 = 7.4e-4  # rad, 99th percentile of the linked-phase error
FP16_PHASE_P50 = 2.7e-4  # rad, median
FP16_PHASE_MAX = 1.18e-3 # rad, largest


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


def round11(x: np.ndarray) -> np.ndarray:
    """float32 -> nearest value with an 11-bit significand (ties to even), as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 13) & 1
    r = ((u + 0xFFF + lsb) >> 13) << 13
    return r.astype(np.uint32).view(np.float32)


def round_stack(z: np.ndarray) -> np.ndarray:
    out = np.empty_like(z)
    out.real = round11(z.real.astype(np.float32))
    out.imag = round11(z.imag.astype(np.float32))
    return out


def test_round11_helper():
    # 11 significant bits: the spacing just above 1 is 2^-10.
    v = np.array([1.0, 1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11, 1.0 + 2 ** -12, -3.5], dtype=np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2 ** -9, 1.0, -3.5], dtype=np.float32)
    assert np.array_equal(round11(v), want)
    h = np.random.default_rng(0).normal(0, 1, 1000).astype(np.float32)
    assert np.array_equal(round11(h), h.astype(np.float16).astype(np.float32))


def _case(cfg, N, H, W, win, seed):
    spec = synth.config_spec(cfg, N=N, H=H, W=W, seed=seed)
    z = synth.generate(spec).numpy()
    P, _ = oracle.amp_stats(z)
    m, cnt = oracle.shp_select(P, win, np.float32(oracle.glrt_threshold(1e-3, N)))
    return z, m, cnt


def cov(ctx, plk, z, win, m):
    return to_np(ctx.estimate_covariance(torch.from_numpy(np.ascontiguousarray(z)).cuda(), win,
                                         torch.from_numpy(m.view(np.int64)).cuda(), precision=plk.COV_FP16))


@pytest.mark.parametrize("cfg,N,win", [(1, 15, (5, 11, 3, 6)), (0, 10, (5, 11, 1, 1)), (0, 2, (3, 5, 1, 1)),
                                       (0, 16, (5, 11, 3, 6)), (0, 21, (5, 11, 3, 6)), (1, 32, (5, 11, 3, 6))])
def test_fp16_contraction_matches_rounded_oracle(ctx, plk, cfg, N, win):
    z, m, cnt = _case(cfg, N, 50, 97, win, seed=31)
    C_o = oracle.covariance(round_stack(z), win, m)
    C_g = cov(ctx, plk, z, win, m)
    ok = cnt > 0
    assert np.all(np.isnan(C_g[~ok].real))
    err = np.abs(C_g[ok] - C_o[ok])
    assert err.max() < 2e-5, err.max()


def test_fp16_scaling(ctx, plk):
    N, win = 15, (5, 11, 3, 6)
    z, m, cnt = _case(1, N, 40, 120, win, seed=8)
    ok = cnt > 0
    base = cov(ctx, plk, z, win, m)
    for f in (2.0 ** 12, 2.0 ** -20):
        assert np.array_equal(np.nan_to_num(cov(ctx, plk, (z * np.float32(f)).astype(np.complex64), win, m)),
                              np.nan_to_num(base))
    big = cov(ctx, plk, (z * np.float32(1e6)).astype(np.complex64), win, m)
    assert np.all(np.isfinite(big[ok]))
    C_o = oracle.covariance(z, win, m)
    assert np.abs(big[ok] - C_o[ok]).max() < FP16_COH_MAX


def test_fp16_mode_bounds(ctx, plk):
    N, win = 15, (5, 11, 3, 6)
    z, m, cnt = _case(1, N, 90, 300, win, seed=5)
    C_o = oracle.covariance(z, win, m)
    C_h = torch.from_numpy(cov(ctx, plk, z, win, m)).cuda()
    ok = cnt > 0
    coh_err = np.abs(to_np(C_h)[ok] - C_o[ok])
    o = oracle.phase_link(C_o[ok], N, 0)
    Ch = C_h.reshape(-1, C_h.shape[-1])[torch.from_numpy(ok.ravel()).cuda()].contiguous()
    g = ctx.phase_link(Ch, N, 0)
    st_g = to_np(g["status"])
    evd_o, evd_g = o["status"] == plk.PX_EVD, st_g == plk.PX_EVD
    keep = (o["gap"] > 1e-6 * np.abs(np.nan_to_num(o["lam"], nan=1.0))) & (evd_o == evd_g)
    e = wrapped_diff(to_np(g["phase"]), o["phase"])[:, keep].max(axis=0)
    p50, p99, mx = np.percentile(e, 50), np.percentile(e, 99), e.max()
    print(f"fp16 coherence max err {coh_err.max():.3e}; phase err p50 {p50:.2e} p99 {p99:.2e} max {mx:.2e} rad "
          f"over {keep.sum()} of {ok.sum()} px; EMI/EVD branch disagreements {np.sum(evd_o != evd_g)}")
    assert coh_err.max() < FP16_COH_MAX
    assert p50 < FP16_PHASE_P50
    assert p99 < FP16_PHASE_P99
    assert mx < FP16_PHASE_MAX


def test_fp16_ministack_step_tracks_fp32(ctx, plk):
    spec = synth.config_spec(1, H=96, W=300, seed=9)
    z = synth.generate(spec).cuda()
    N = z.shape[0]
    outs = {}
    for prec in (plk.COV_FP32, plk.COV_FP16):
        st = plk.State(ctx, spec.H, spec.W, (5, 11, 3, 6), K_max=6, M_max=N)
        outs[prec] = st.step(z, plk.default_params(cov_precision=prec))
        st.close()
    a, b = outs[plk.COV_FP32], outs[plk.COV_FP16]
    live = to_np(a["status"]) != plk.PX_NODATA
    d = wrapped_diff(to_np(a["phase"]), to_np(b["phase"]))[:, live]
    assert np.percentile(d.max(axis=0), 50) < FP16_PHASE_P50


def test_fp16_rejects_large_n(ctx, plk):
    z = torch.zeros((33, 8, 8), dtype=torch.complex64, device="cuda")
    mask = torch.zeros((8, 8, 1), dtype=torch.int64, device="cuda")
    with pytest.raises(RuntimeError):
        ctx.estimate_covariance(z, (3, 3, 1, 1), mask, precision=plk.COV_FP16)
