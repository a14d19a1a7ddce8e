"""Phase cosine similarity on the GPU (plk_phase_similarity) against the
oracle on the same seeded phases.

Bar: gamma_s within 1e-5 (single-precision phasors and sums; the median is
1-Lipschitz in the similarities, so their rounding error bounds its error);
NaN exactly where the oracle has NaN.  Sizes span several CTA tiles with
ragged tails; M from 2 to 32; radii 1 to 9; no-data cells; the closed forms
of the oracle pins; the step's own output at the burst's posting."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2511_12051_gb300 import synth
from parity_util import to_np

pytestmark = pytest.mark.gpu

GS_TOL = 1e-5


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


def field(M, Ho, Wo, seed, noise=0.6, nan_frac=0.01):
    # a smooth deformation-like history plus per-pixel noise and offsets, with no-data cells
    rng = np.random.default_rng(seed)
    t = np.arange(M)[:, None, None]
    yy, xx = np.mgrid[0:Ho, 0:Wo]
    defo = 0.15 * np.sin(xx / 9.0 + yy / 13.0)[None] * t
    ph = defo + rng.normal(0, noise, (M, Ho, Wo)) + rng.uniform(-np.pi, np.pi, (Ho, Wo))[None]
    ph = np.angle(np.exp(1j * ph))
    bad = rng.random((Ho, Wo)) < nan_frac
    ph[rng.integers(0, M), bad] = np.nan
    return ph.astype(np.float32)


def compare(ctx, ph, r):
    g = to_np(ctx.phase_similarity(torch.from_numpy(ph).cuda(), r))
    o = oracle.phase_similarity(ph.astype(np.float64), r)
    assert np.array_equal(np.isnan(g), np.isnan(o))
    d = np.abs(g - o)[~np.isnan(o)]
    return d.max() if d.size else 0.0


@pytest.mark.parametrize("M,Ho,Wo,r", [(15, 37, 53, 7), (15, 70, 131, 3), (2, 20, 33, 1), (3, 25, 17, 2),
                                       (8, 41, 40, 5), (16, 23, 70, 4), (17, 30, 45, 6), (32, 19, 36, 3),
                                       (10, 9, 9, 9)])
def test_phase_similarity_parity(ctx, plk, M, Ho, Wo, r):
    err = compare(ctx, field(M, Ho, Wo, seed=M * 100 + r), r)
    print(f"M={M} {Ho}x{Wo} r={r}: max |gamma_s - oracle| = {err:.2e}")
    assert err <= GS_TOL


def test_phase_similarity_closed_forms(ctx, plk):
    M, delta = 15, 0.4
    rng = np.random.default_rng(3)
    hist = np.cumsum(rng.normal(0, 0.5, M))
    ph = (hist[:, None, None] + rng.uniform(-np.pi, np.pi, (40, 50))[None]).astype(np.float32)
    ph[:, 20, 25] += (delta * np.arange(M)).astype(np.float32)
    g = to_np(ctx.phase_similarity(torch.from_numpy(ph).cuda(), 7))
    K = 3 * M - 6
    c = sum((M - d) * math.cos(d * delta) for d in (1, 2, 3)) / K
    assert abs(g[20, 25] - c) < 1e-5
    mask = np.ones_like(g, bool)
    mask[20, 25] = False
    assert np.abs(g[mask] - 1.0).max() < 1e-5


def test_phase_similarity_all_nan_and_rejections(ctx, plk):
    ph = torch.full((5, 6, 7), float("nan"), device="cuda")
    assert torch.all(torch.isnan(ctx.phase_similarity(ph, 2)))
    with pytest.raises(plk.PlkError):
        ctx.phase_similarity(torch.zeros((33, 4, 4), device="cuda"), 2)     # M > 32
    with pytest.raises(plk.PlkError):
        ctx.phase_similarity(torch.zeros((1, 4, 4), device="cuda"), 2)      # M < 2
    with pytest.raises(plk.PlkError):
        ctx.phase_similarity(torch.zeros((4, 4, 4), device="cuda"), 0)      # radius 0
    with pytest.raises(plk.PlkError):
        ctx.phase_similarity(torch.zeros((32, 40, 40), device="cuda"), 32)  # window beyond shared memory


def test_phase_similarity_of_a_step_output(ctx, plk):
    # The burst's posting (11x5 window, strides 6x3) on a 240x900 crop of the
    # burst-shaped workload; gamma_s of the step's phases over the ~200 m
    # window (radius 7), against the oracle on the same phases.
    spec = synth.config_spec(1, H=240, W=900, seed=4)
    z = synth.generate(spec).cuda()
    st = plk.State(ctx, spec.H, spec.W, (5, 11, 3, 6), K_max=2, M_max=spec.N)
    out = st.step(z)
    ph = out["phase"].contiguous()
    g = to_np(ctx.phase_similarity(ph, 7))
    o = oracle.phase_similarity(to_np(ph).astype(np.float64), 7)
    assert np.array_equal(np.isnan(g), np.isnan(o))
    assert np.nanmax(np.abs(g - o)) <= GS_TOL
    # coherent burst pixels agree with their neighbourhood
    assert np.nanmedian(g) > 0.3
    st.close()
