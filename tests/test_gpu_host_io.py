"""plk_ministack_step_host: the step with host-memory inputs and outputs and
double-buffered staging.  A chain of calls issued back to back (each call's
copy overlapping the previous call's compute) must give exactly the outputs
and compressed SLCs of the same chain through plk_ministack_step on device
buffers; pageable host memory works too."""
import numpy as np
import pytest
import torch

from paper_2511_12051_gb300 import synth
from parity_util import to_np

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


def same(a, b):
    return torch.equal(torch.nan_to_num(a.float(), nan=-9.0), torch.nan_to_num(b.float(), nan=-9.0))


@pytest.mark.parametrize("pinned", [True, False])
def test_host_chain_equals_device_chain(plk, ctx, pinned):
    spec = synth.config_spec(3, scale=0.05, seed=5)        # 60 dates of 102 x 205, four mini-stacks of 15
    z = synth.generate(spec)
    win, M = (5, 11, 1, 1), 15
    H, W = z.shape[1:]
    slices = synth.ministack_slices(60, M)
    dev = plk.State(ctx, H, W, win, K_max=3, M_max=M)
    ref = []
    for sl in slices:
        o = dev.step(z[sl].contiguous().cuda())
        ref.append({k: v.clone() for k, v in o.items() if v is not None})
    ref_kappa = to_np(dev.kappa(dev.info()["K_used"] - 1)).copy()
    hst = plk.State(ctx, H, W, win, K_max=3, M_max=M)
    hst.enable_host_io()
    ins = [z[sl].contiguous().pin_memory() if pinned else z[sl].contiguous() for sl in slices]
    outs = [hst.step_host(x, want_count=True) for x in ins]   # no sync in between
    ctx.sync()
    for r, o in zip(ref, outs):
        for key in ("phase", "tcoh", "status"):
            assert same(o[key], r[key].cpu()), key
        assert torch.equal(o["count"], r["count"].cpu())
    assert np.array_equal(to_np(hst.kappa(hst.info()["K_used"] - 1)), ref_kappa)
    assert hst.info() == dev.info()
    dev.close()
    hst.close()


def test_host_step_rejects_bad_inputs(plk, ctx):
    st = plk.State(ctx, 16, 24, (3, 5, 1, 1), K_max=1, M_max=4)
    with pytest.raises(plk.PlkError, match="enable_host_io"):
        st.step_host(torch.zeros((4, 16, 24), dtype=torch.complex64))    # no staging yet
    st.enable_host_io()
    with pytest.raises(TypeError):
        st.step_host(torch.zeros((4, 16, 24), dtype=torch.complex64, device="cuda"))
    with pytest.raises(ValueError):
        st.step_host(torch.zeros((4, 16, 25), dtype=torch.complex64))
    with pytest.raises(plk.PlkError):
        st.step_host(torch.zeros((5, 16, 24), dtype=torch.complex64))      # M > M_max
    st.close()


def test_steps_allocate_nothing_after_setup(plk, ctx):
    """Every device allocation happens when the context, the state and the
    host-I/O staging are made; the steps (device or host buffers, every
    coherence mode, PS selection, decaying weights, complex 16-bit host
    input) add none."""
    spec = synth.config_spec(1, N=30, H=60, W=120, seed=31)
    z = synth.generate(spec)
    win, M = (5, 11, 3, 6), 10
    st = plk.State(ctx, 60, 120, win, K_max=2, M_max=M)
    st.enable_host_io()
    st.enable_host_io_ci16()
    zg = z.cuda()
    q = _to_ci16(z, 3000.0)
    ctx.sync()
    before = plk.device_allocations()
    params = [plk.default_params(), plk.default_params(cov_precision=plk.COV_BF16),
              plk.default_params(cov_precision=plk.COV_FP16), plk.default_params(ps_da_max=0.2),
              plk.default_params(decay=0.9)]
    for p in params:
        st.reset()
        for sl in synth.ministack_slices(30, M):
            st.step(zg[sl].contiguous(), p)
            st.step_host(z[sl].contiguous(), p)
            st.step_host_ci16(q[sl].contiguous(), p)
        ctx.sync()
    assert plk.device_allocations() == before
    st.close()


def _to_ci16(z: torch.Tensor, scale: float) -> torch.Tensor:
    """Complex samples quantised to complex 16-bit integers [.., 2] (test input)."""
    q = torch.stack([torch.round(z.real * scale), torch.round(z.imag * scale)], dim=-1)
    return q.clamp(-32768, 32767).to(torch.int16).contiguous()


def test_ci16_host_chain_equals_device_chain_on_widened_samples(plk, ctx):
    # complex 16-bit samples through plk_ministack_step_host_ci16, calls back
    # to back, against plk_ministack_step on the same samples widened on the
    # host: identical outputs and compressed SLCs; the int16 extremes and an
    # odd pixel count (a tail of the widening's four-sample vectors) included
    spec = synth.config_spec(3, scale=0.05, seed=6)
    z = synth.generate(spec)[:30, :101, :203].contiguous()
    q = _to_ci16(z, 3000.0)
    q[0, 0, 0] = torch.tensor([-32768, 32767], dtype=torch.int16)
    q[1, 5, 7] = torch.tensor([32767, -32768], dtype=torch.int16)
    zw = torch.complex(q[..., 0].float(), q[..., 1].float())
    win, M = (5, 11, 1, 1), 15
    H, W = zw.shape[1:]
    slices = synth.ministack_slices(30, M)
    dev = plk.State(ctx, H, W, win, K_max=3, M_max=M)
    ref = []
    for sl in slices:
        o = dev.step(zw[sl].contiguous().cuda())
        ref.append({k: v.clone() for k, v in o.items() if v is not None})
    ref_kappa = to_np(dev.kappa(dev.info()["K_used"] - 1)).copy()
    hst = plk.State(ctx, H, W, win, K_max=3, M_max=M)
    hst.enable_host_io_ci16()
    outs = [hst.step_host_ci16(q[sl].contiguous().pin_memory(), want_count=True) for sl in slices]
    ctx.sync()
    for r, o in zip(ref, outs):
        for key in ("phase", "tcoh", "status"):
            assert same(o[key], r[key].cpu()), key
        assert torch.equal(o["count"], r["count"].cpu())
    assert np.array_equal(to_np(hst.kappa(hst.info()["K_used"] - 1)), ref_kappa)
    # the complex64 host path on the same state after the int16 calls
    st2 = plk.State(ctx, H, W, win, K_max=3, M_max=M)
    st2.enable_host_io_ci16()
    a = st2.step_host_ci16(q[slices[0]].contiguous().pin_memory())
    b = st2.step_host(zw[slices[1]].contiguous().pin_memory())
    ctx.sync()
    assert same(a["phase"], ref[0]["phase"].cpu()) and same(b["phase"], ref[1]["phase"].cpu())
    for s_ in (dev, hst, st2):
        s_.close()


def test_ci16_host_step_rejects_bad_inputs(plk, ctx):
    st = plk.State(ctx, 16, 24, (3, 5, 1, 1), K_max=1, M_max=4)
    st.enable_host_io()
    with pytest.raises(plk.PlkError, match="enable_host_io_ci16"):
        st.step_host_ci16(torch.zeros((4, 16, 24, 2), dtype=torch.int16))   # no int16 staging yet
    st.enable_host_io_ci16()
    with pytest.raises(TypeError):
        st.step_host_ci16(torch.zeros((4, 16, 24, 2), dtype=torch.int32))
    with pytest.raises(ValueError):
        st.step_host_ci16(torch.zeros((4, 16, 24), dtype=torch.int16))
    with pytest.raises(plk.PlkError):
        st.step_host_ci16(torch.zeros((5, 16, 24, 2), dtype=torch.int16))     # M > M_max
    st.close()
