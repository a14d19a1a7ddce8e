"""S1-S2 with exponentially decaying image weights (Sec. III-A, the option
beside equal weights per image; plk_params.decay) against the oracle
(oracle/decay.py through OracleChain(decay=...)).

Bars, per step from identical inputs (the oracle's state loaded through the
checkpoint format): power and amplitude sums bit-exact (single precision in
the fixed decision order on both sides), the effective looks W1, W2 equal,
SHP masks and counts bit-exact, linked phase within 1e-4 rad, gamma_t within
1e-5.  decay = 1 is bit-identical to the default equal-weight step.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_12051_gb300 import synth
from parity_util import clear_of_degenerate, PHASE_TOL, TCOH_TOL, count_np, phase_report, to_np, write_state_file

pytestmark = pytest.mark.gpu


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


def test_real_looks_threshold_matches_the_oracle(plk):
    for nu in (1.0, 2.5, 7.3, 15.0, 28.9):
        c_lib = plk.glrt_threshold_looks(1e-3, nu)
        c_orc = oracle.glrt_threshold_real(1e-3, nu)
        assert c_lib == pytest.approx(c_orc, rel=1e-9), nu
        assert np.float32(c_lib) == np.float32(c_orc), nu
    assert plk.glrt_threshold_looks(1e-3, 15.0) == pytest.approx(plk.glrt_threshold(1e-3, 15), rel=1e-12)


@pytest.mark.parametrize("lam", [0.9, 0.75])
def test_decaying_chain_per_step(plk, ctx, lam, tmp_path):
    spec = synth.config_spec(1, N=30, H=60, W=240, seed=21)   # 5% persistent scatterers
    z = synth.generate(spec)
    window, M, K_max = (5, 11, 3, 6), 10, 6
    H, W = z.shape[1:]
    # the library takes the decay as a float: the oracle gets the same value
    orc = oracle.OracleChain(H, W, window, K_max=K_max, alpha=1e-3, kappa_dtype=np.complex64,
                             decay=float(np.float32(lam)))
    params = plk.default_params(decay=lam)
    zg = z.cuda()
    for k, sl in enumerate(synth.ministack_slices(30, M)):
        path = str(tmp_path / f"d{k}.plk")
        write_state_file(path, orc)
        st = plk.State.load(ctx, path, M_max=M)
        g = st.step(zg[sl].contiguous(), params)
        o = orc.step(z[sl].numpy())
        assert np.array_equal(to_np(st.sum_pow()), orc.sum_pow), k
        st_w = st.weights()
        assert st_w == pytest.approx(orc.wsum, rel=1e-12), k
        assert np.array_equal(count_np(g["count"]), o["count"]), k
        live = o["status"] != 3
        assert np.array_equal(to_np(g["status"]) == 3, ~live)
        clear = clear_of_degenerate(o, live)[0]
        rep = phase_report(to_np(g["phase"]), o["phase"][o["K_used"]:], clear)
        assert rep["max"] <= PHASE_TOL, (k, rep)
        assert np.abs(to_np(g["tcoh"]) - o["tcoh"])[live].max() <= TCOH_TOL
        st.close()
    # T images of weights lam^(T-1-t): W1 = (1 - lam^T) / (1 - lam), W2 = (1 - lam^2T) / (1 - lam^2),
    # so nu = W1^2 / W2 lies below T and tends to (1 + lam) / (1 - lam)
    lam32, T = float(np.float32(lam)), 30
    W1 = (1 - lam32 ** T) / (1 - lam32)
    W2 = (1 - lam32 ** (2 * T)) / (1 - lam32 ** 2)
    assert st_w[0] == pytest.approx(W1, rel=1e-6) and st_w[1] == pytest.approx(W2, rel=1e-6)
    assert 1 < W1 * W1 / W2 < T


def test_decay_one_is_the_equal_weight_step(plk, ctx):
    spec = synth.config_spec(1, N=20, H=48, W=120, seed=22)
    z = synth.generate(spec).cuda()
    outs = []
    for p in (plk.default_params(), plk.default_params(decay=1.0)):
        st = plk.State(ctx, 48, 120, (5, 11, 3, 6), K_max=3, M_max=10)
        res = [st.step(z[sl].contiguous(), p) for sl in synth.ministack_slices(20, 10)]
        outs.append((res, to_np(st.sum_pow()), st.weights()))
        st.close()
    (ra, pa, wa), (rb, pb, wb) = outs
    assert np.array_equal(pa, pb) and wa == wb == (20.0, 20.0)
    for a, b in zip(ra, rb):
        for key in ("phase", "tcoh", "status", "count"):
            assert torch.equal(torch.nan_to_num(a[key].float(), nan=-9), torch.nan_to_num(b[key].float(), nan=-9))


def test_decay_rejects_bad_values_and_ps(plk, ctx):
    st = plk.State(ctx, 30, 60, (5, 11, 3, 6), K_max=2, M_max=5)
    z = torch.zeros((5, 30, 60), dtype=torch.complex64, device="cuda")
    for bad in (0.0, -0.5, 1.5, float("nan")):
        with pytest.raises(plk.PlkError, match="PLK_EINVAL"):
            st.step(z, plk.default_params(decay=bad))
    with pytest.raises(plk.PlkError, match="PLK_EUNSUPPORTED"):
        st.step(z, plk.default_params(decay=0.9, ps_da_max=0.2))
    st.close()
