"""Continuous-batching serving (ds_submit / ds_poll / ds_wait): results are identical alone
and in the mix, admission by HBM footprint, bounded waits, malformed requests."""
import numpy as np
import pytest

import synthetic as syn
from _helpers import qgrid_tuple, to_library

pytestmark = pytest.mark.gpu


def _requests():
    out = []
    for i, (kind, cells, nsite) in enumerate([(0, (8, 8, 8), 4), (1, (6, 8, 10), 3), (2, (8, 6, 8), 2),
                                              (0, (12, 10, 8), 8), (1, (8, 8, 8), 5), (2, (10, 8, 6), 3),
                                              (0, (16, 16, 16), 16), (1, (12, 12, 12), 8)]):
        m = syn.small_case(kind, cells=cells, nsite=nsite, nmodels=1 + i % 2, seed=300 + i)
        opts = dict(disorder=kind, mode=i % 2, precision=i % 2)
        if kind == 2:
            opts.update(taylor_order=-1, taylor_eps=1e-6)
        if i == 3:
            opts.update(smoothing=1, lanczos_m=2, lanczos_mprime=2)
        out.append((m, opts))
    return out


def test_results_identical_alone_and_in_the_mix():
    import torch
    import paper_1809_07088_gb300 as ds
    ctx = ds.Context(0)
    reqs = _requests()
    models = [to_library(ctx, m) for m, _ in reqs]
    alone = []
    for lm, (m, o) in zip(models, reqs):
        got, _ = lm.intensity(qgrid_tuple(m.qgrid), **o)
        alone.append(got)
    outs, tickets = [], []
    for lm, (m, o) in zip(models, reqs):
        dt = torch.float64 if o["precision"] == 0 else torch.float32
        out = torch.full(m.qgrid.count, float("nan"), dtype=dt, device="cuda")
        outs.append(out)
        tickets.append(lm.submit(qgrid_tuple(m.qgrid), out, **o))
    infos = [ctx.wait(t, 120.0) for t in tickets]
    for a, out, info, (m, o) in zip(alone, outs, infos, reqs):
        assert np.array_equal(a, out.cpu().numpy())
        assert info.nvox == m.qgrid.nvox and info.latency_ms > 0 and info.gpu_ms > 0
    ctx.close()


def test_admission_by_footprint_and_refusal():
    import torch
    import paper_1809_07088_gb300 as ds
    m = syn.small_case(syn.SPIN, cells=(16, 16, 16), nsite=8, nmodels=1, seed=320)
    budget = 6 << 20          # a few MB: requests must take turns
    ctx = ds.Context(0, hbm_budget=budget)
    lm = to_library(ctx, m)
    want, _ = lm.intensity(qgrid_tuple(m.qgrid), disorder=1, mode=0, precision=1)
    outs = [torch.empty(m.qgrid.count, dtype=torch.float32, device="cuda") for _ in range(6)]
    ts = [lm.submit(qgrid_tuple(m.qgrid), o, disorder=1, mode=0, precision=1) for o in outs]
    for t in ts:
        ctx.wait(t, 60.0)
    for o in outs:
        assert np.array_equal(o.cpu().numpy(), want)
    big = syn.small_case(syn.SPIN, cells=(32, 32, 32), nsite=16, nmodels=1, seed=321)
    lb = to_library(ctx, big)
    out = torch.empty(big.qgrid.count, dtype=torch.float32, device="cuda")
    with pytest.raises(ds.DSError) as e:
        lb.submit(qgrid_tuple(big.qgrid), out, disorder=1, mode=0, precision=1)
    assert "DS_ERR_ADMISSION" in str(e.value)
    ctx.close()


def test_bounded_wait_and_poll_while_paused():
    import torch
    import paper_1809_07088_gb300 as ds
    ctx = ds.Context(0)
    m = syn.small_case(syn.OCC, cells=(8, 8, 8), nsite=2, nmodels=1, seed=330)
    lm = to_library(ctx, m)
    out = torch.empty(m.qgrid.count, dtype=torch.float32, device="cuda")
    ctx.pause_serving(True)
    t = lm.submit(qgrid_tuple(m.qgrid), out, disorder=0, mode=1, precision=1)
    st, _ = ctx.poll(t)
    assert st == ds._binding.DS_ERR_STATE
    with pytest.raises(ds.DSError) as e:
        ctx.wait(t, 0.2)
    assert "DS_ERR_TIMEOUT" in str(e.value)
    ctx.pause_serving(False)
    info = ctx.wait(t, 60.0)
    assert info.nvox == m.qgrid.nvox
    want, _ = lm.intensity(qgrid_tuple(m.qgrid), disorder=0, mode=1, precision=1)
    assert np.array_equal(out.cpu().numpy(), want)
    # malformed requests are refused at submission
    bad = syn.QGrid((0.0, 0.0, 0.0), (0.3, 0.125, 0.125), (2, 2, 2))
    with pytest.raises(ds.DSError):
        lm.submit(qgrid_tuple(bad), out, disorder=0)
    with pytest.raises(ds.DSError):
        lm.submit(qgrid_tuple(m.qgrid), out, disorder=1)   # no spins uploaded
    ctx.close()


def test_served_and_direct_displacive_requests_on_one_model_concurrently():
    """Displacive requests with several Taylor orders go through ds_submit (planned on the
    serving worker thread) while the caller thread runs ds_request_intensity on the same model
    with other orders: both threads fill the model's per-order table caches at the same time.
    Every result equals the same request run alone."""
    import torch
    import paper_1809_07088_gb300 as ds
    ctx = ds.Context(0)
    m = syn.small_case(syn.DISP, cells=(8, 6, 8), nsite=3, nmodels=1, seed=340, sigma=0.08)
    lm = to_library(ctx, m)
    q = qgrid_tuple(m.qgrid)
    served_P, direct_P = [3, 4, 5, 6, 7, 8], [9, 10, 11, 12]
    base = dict(disorder=2, mode=1, precision=1)
    # isolated results on a second model (empty caches), so the concurrent run builds its own
    ref = to_library(ctx, m)
    alone = {P: ref.intensity(q, taylor_order=P, **base)[0] for P in served_P + direct_P}
    outs = [torch.full(m.qgrid.count, float("nan"), dtype=torch.float32, device="cuda") for _ in served_P]
    tickets = [lm.submit(q, o, taylor_order=P, **base) for o, P in zip(outs, served_P)]
    direct = {P: lm.intensity(q, taylor_order=P, **base)[0] for P in direct_P}
    for t in tickets:
        ctx.wait(t, 120.0)
    for o, P in zip(outs, served_P):
        assert np.array_equal(o.cpu().numpy(), alone[P]), P
    for P in direct_P:
        assert np.array_equal(direct[P], alone[P]), P
    ctx.close()


def test_served_fp32_results_match_the_plain_fp64_path():
    """A mixed stream (occupancy, moments, displacive with automatic orders planned on the GPU,
    Lanczos) served in FP32 on concurrent streams: every result within 1e-5 of peak of the same
    request computed alone on the plain FP64 path, and the displacive ones with the FP64 path's
    Taylor order."""
    import torch
    import paper_1809_07088_gb300 as ds
    ctx = ds.Context(0)
    reqs = _requests()
    models = [to_library(ctx, m) for m, _ in reqs]
    outs, tickets = [], []
    for lm, (m, o) in zip(models, reqs):
        o32 = dict(o, precision=1)
        out = torch.full(m.qgrid.count, float("nan"), dtype=torch.float32, device="cuda")
        outs.append(out)
        tickets.append(lm.submit(qgrid_tuple(m.qgrid), out, **o32))
    infos = [ctx.wait(t, 120.0) for t in tickets]
    for lm, out, info, (m, o) in zip(models, outs, infos, reqs):
        want, info64 = lm.intensity(qgrid_tuple(m.qgrid), **dict(o, precision=0))
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want))
        if o["disorder"] == 2:
            assert info.taylor_order == info64["taylor_order"] and info.x_max == info64["x_max"]
    ctx.close()
