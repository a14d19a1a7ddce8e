"""Failure detection without a GPU fault: a device-side wait that nothing
completes gives up within its bound and is reported on the host as
PLK_ETIMEOUT; the context keeps working afterwards.  Bad arguments are
rejected on the host before any launch."""
import time

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plk():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2511_12051_gb300 import build, plk as _plk
    build.build()
    return _plk


def test_bounded_wait_reports_timeout_and_context_survives(plk):
    ctx = plk.Context("cuda:0")
    ctx.sync()
    t0 = time.time()
    plk.lib().plk_selftest_bounded_wait(ctx.h)
    with pytest.raises(plk.PlkError) as ei:
        ctx.sync()
    assert ei.value.code == 4  # PLK_ETIMEOUT
    assert time.time() - t0 < 30.0
    # the flag was consumed and the context still computes
    ctx.sync()
    z = torch.randn((3, 20, 30), dtype=torch.complex64, device="cuda")
    P, _ = ctx.amp_stats(z)
    ctx.sync()
    assert torch.allclose(P, (z.abs() ** 2).sum(0), rtol=1e-5)


def test_invalid_arguments_launch_nothing(plk):
    ctx = plk.Context("cuda:0")
    z = torch.zeros((2, 8, 8), dtype=torch.complex64, device="cuda")
    with pytest.raises(plk.PlkError) as ei:
        ctx.estimate_covariance(z, (4, 5, 1, 1), torch.zeros((8, 8, 1), dtype=torch.int64, device="cuda"))
    assert ei.value.code == 1
    with pytest.raises(plk.PlkError):
        ctx.phase_link(torch.zeros((4, 3), dtype=torch.complex64, device="cuda"), 2, 2)
    with pytest.raises(ValueError):
        ctx.amp_stats(z.cpu())
    ctx.sync()
