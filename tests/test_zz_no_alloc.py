"""plk_phase_link_stack_noalloc, the entry point for callers that cannot
allocate device memory (for example a plug-in inside a host application that
owns every allocation), against the allocating path: plk_ministack_step on a
fresh state computes the same mini-stack.  Two calls in a row, because every
call reuses the same device scratch array.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from parity_util import PHASE_TOL, TCOH_TOL, count_np, to_np, wrapped_diff

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.fixture(scope="module")
def plk():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2511_12051_gb300 import build, plk as _plk
    build.build()
    return _plk


@pytest.mark.parametrize("cov_precision", ["fp32", "fp16"])
def test_noalloc_matches_allocating_path_twice(plk, cov_precision):
    from paper_2511_12051_gb300 import synth
    L = plk.lib()
    ctx = plk.Context("cuda:0")
    win = (5, 11, 3, 6)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    params = plk.default_params(cov_precision={"fp32": plk.COV_FP32, "fp16": plk.COV_FP16}[cov_precision])
    for seed in (41, 42):
        spec = synth.config_spec(1, H=96, W=300, seed=seed)
        z = synth.generate(spec).cuda()
        N, H, W = z.shape
        st = plk.State(ctx, H, W, win, K_max=6, M_max=N)
        ref = st.step(z, params)
        Ho, Wo = st.Ho, st.Wo
        phase = torch.full((N, Ho, Wo), 7.0, device="cuda")
        tcoh = torch.full((Ho, Wo), 7.0, device="cuda")
        status = torch.full((Ho, Wo), 99, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros((Ho, Wo), dtype=torch.int16, device="cuda")
        rc = L.plk_phase_link_stack_noalloc(_p(z), N, H, W, plk.window(win), 0, ctypes.byref(params), _p(phase),
                                            _p(tcoh), _p(status), _p(cnt), stream)
        assert rc == 0, L.plk_last_error(None)
        torch.cuda.synchronize()
        assert np.array_equal(count_np(cnt), count_np(ref["count"]))
        assert np.array_equal(to_np(status), to_np(ref["status"]))
        live = to_np(status) != plk.PX_NODATA
        assert wrapped_diff(to_np(phase), to_np(ref["phase"]))[:, live].max() <= PHASE_TOL
        assert np.abs(to_np(tcoh) - to_np(ref["tcoh"]))[live].max() <= TCOH_TOL
        st.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(plk):
    L = plk.lib()
    z = torch.zeros((15, 2048, 2048), dtype=torch.complex64, device="cuda")
    out = torch.zeros((15, 2048, 2048), device="cuda")
    rc = L.plk_phase_link_stack_noalloc(_p(z), 15, 2048, 2048, plk.window((5, 11, 1, 1)), 0, None, _p(out),
                                        _p(out), _p(out), None, None)
    assert rc == 1
    assert b"PLK_NOALLOC_SCRATCH_BYTES" in L.plk_last_error(None)


def test_noalloc_rejects_what_it_does_not_compute(plk):
    """PS regridding is a plk_ministack_step option this entry point does not
    run: asked for, it refuses instead of returning plain EMI phases.  Bad
    parameters are rejected by the same checks as the other entry points."""
    L = plk.lib()
    z = torch.zeros((15, 30, 60), dtype=torch.complex64, device="cuda")
    out = torch.zeros((15, 10, 10), device="cuda")
    st = torch.zeros((10, 10), dtype=torch.uint8, device="cuda")
    win = plk.window((5, 11, 3, 6))
    p = plk.default_params(ps_da_max=0.2)
    rc = L.plk_phase_link_stack_noalloc(_p(z), 15, 30, 60, win, 0, ctypes.byref(p), _p(out), _p(out), _p(st), None,
                                        None)
    assert rc == 5, L.plk_last_error(None)      # PLK_EUNSUPPORTED
    for bad in ({"mu": -1.0}, {"mu": float("nan")}, {"tol": 0.0}, {"cov_precision": 7}, {"ref_scheme": 9}):
        p = plk.default_params(**bad)
        rc = L.plk_phase_link_stack_noalloc(_p(z), 15, 30, 60, win, 0, ctypes.byref(p), _p(out), _p(out), _p(st),
                                            None, None)
        assert rc == 1, (bad, L.plk_last_error(None))  # PLK_EINVAL
