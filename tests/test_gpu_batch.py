"""Batches of independent stacks of uneven length (plk_batch_*), shaped like the
multi-burst workload (N from 5 to 30, near-singular coherence patches that
exercise the double-precision re-solve): every stack against the FP64 oracle
and against the single-stack path; the recorded graph replays with identical
results; the tuned schedules are valid; descriptors are checked."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_12051_gb300 import synth
from parity_util import clear_of_degenerate, PHASE_TOL, TCOH_TOL, phase_report, to_np, wrapped_diff

pytestmark = pytest.mark.gpu

WIN = (5, 11, 3, 6)


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


def uneven_stack(N, seed, H=48, W=120, rho0=0.6):
    # one stack of the uneven-batch workload, scaled down; 5% of the pixels in
    # 8 x 8 patches of coherence 0.98 (near-singular |Gamma|)
    spec = synth.config_spec(2, N=N, H=H, W=W, seed=seed, rho0=rho0, patches=(0.05, 8, 0.98))
    return synth.generate(spec)


def oracle_stack(z, win, ref):
    zn = z.numpy()
    N = zn.shape[0]
    P, _ = oracle.amp_stats(zn)
    m, _ = oracle.shp_select(P, win, np.float32(oracle.glrt_threshold(1e-3, N)))
    C = oracle.covariance(zn, win, m)
    return oracle.phase_link(C, N, ref)


def test_batch_uneven_stacks_match_oracle(ctx, plk):
    Ns = [5, 9, 15, 17, 24, 30]
    refs = [0, 3, 0, 16, 5, 29]
    rhos = [0.3, 0.9, 0.6, 0.45, 0.75, 0.5]
    zs = [uneven_stack(N, 100 + i, rho0=r) for i, (N, r) in enumerate(zip(Ns, rhos))]
    b = plk.Batch(ctx, [z.cuda() for z in zs], WIN, refs=refs)
    out = b.run()
    torch.cuda.synchronize()
    n_fp64 = 0
    for z, ref, o_g in zip(zs, refs, out):
        o = oracle_stack(z, WIN, ref)
        st_g = to_np(o_g["status"])
        n_fp64 += int(np.sum(st_g == plk.PX_EMI_FP64))
        live = o["status"] != 3
        assert np.array_equal(st_g == plk.PX_NODATA, ~live)
        clear = clear_of_degenerate(o, live)[0]
        rep = phase_report(to_np(o_g["phase"]), o["phase"], clear)
        assert rep["max"] <= PHASE_TOL, (z.shape[0], rep)
        assert np.all(to_np(o_g["phase"])[ref][live] == 0.0)
        assert np.nanmax(np.abs(to_np(o_g["tcoh"])[live] - o["tcoh"][live])) <= TCOH_TOL
        assert clear.sum() >= 0.98 * live.sum()
    assert n_fp64 > 0  # the near-singular patches reach the double-precision re-solve
    info = b.info()
    assert info["graph_built"] == 1 and info["nodes"] > 6 * 4
    b.close()


def test_batch_equals_single_stack_path_and_replays(ctx, plk):
    Ns = [6, 15, 21]
    zs = [uneven_stack(N, 200 + N, H=60, W=150).cuda() for N in Ns]
    b = plk.Batch(ctx, zs, WIN)
    first = [{k: v.clone() for k, v in o.items()} for o in b.run()]
    torch.cuda.synchronize()
    again = b.run()  # graph replay
    torch.cuda.synchronize()
    for f, a in zip(first, again):
        for key in ("phase", "tcoh", "status"):
            assert torch.equal(torch.nan_to_num(f[key].float(), nan=-9.0), torch.nan_to_num(a[key].float(), nan=-9.0))
    for z, f in zip(zs, first):
        N, H, W = z.shape
        st = plk.State(ctx, H, W, WIN, K_max=4, M_max=N)
        ref = st.step(z)
        torch.cuda.synchronize()
        assert torch.equal(ref["status"], f["status"])
        live = to_np(ref["status"]) != plk.PX_NODATA
        assert wrapped_diff(to_np(ref["phase"]), to_np(f["phase"]))[:, live].max() <= PHASE_TOL
        st.close()
    b.close()


def test_batch_tuned_schedules(ctx, plk):
    for N in (6, 15, 21):
        s = plk.tuned_schedule(ctx, N, WIN)  # tuned by the previous tests' first runs
        rows = [8, 16, 20, 24, 28, 32]  # EMI row lengths: the smallest holding N, or the next
        i0 = next(i for i, r in enumerate(rows) if r >= N)
        assert s["emi_lanes"] in (rows[i0], rows[min(i0 + 1, len(rows) - 1)])
        ty, tx = s["cov_tile"]
        ppw = 5 if N <= 18 else 2
        assert ty > 0 and tx > 0 and ty % ppw == 0
    with pytest.raises(RuntimeError):
        plk.tuned_schedule(ctx, 7, (3, 3, 1, 1))


def test_batch_rejects_bad_descriptors(ctx, plk):
    good = torch.zeros((4, 16, 16), dtype=torch.complex64, device="cuda")
    with pytest.raises(RuntimeError):
        plk.Batch(ctx, [good], WIN, refs=[4])          # ref_idx out of range
    with pytest.raises(RuntimeError):
        plk.Batch(ctx, [good[:1]], WIN)                # N = 1
    with pytest.raises(RuntimeError):
        plk.Batch(ctx, [good], (4, 11, 3, 6))          # even window
