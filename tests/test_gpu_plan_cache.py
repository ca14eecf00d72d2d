"""The plan cache of sos_prepare: a channel whose raw coefficients, K and
length match those its tables were built from keeps them; any change
recomputes what depends on it.  Results must be those of a fresh plan, bit
for bit, through every change and back."""
import numpy as np
import pytest
import torch

import oracle
from synth import filters, rng, workloads
from test_gpu_forward import _lib, check, run_oracle

pytestmark = pytest.mark.gpu


def _case():
    lengths = [90_000, 40_001, 5, 4000]
    C, kmax = len(lengths), 6
    K = torch.tensor([6, 4, 2, 5], dtype=torch.int32)
    sos = workloads._random_bank(61, C, kmax, 0.4, 0.97, K.numpy())
    # channel 3: two identical low-pass sections (coincident poles) on a
    # channel too short for the partial-fraction-free horizon's eight
    # segments, so the look-back carries its state: the dispatch order is
    # part of the plan
    s1 = filters.butter_lowpass2_closed_form(0.05)
    sos[3, 3:5] = np.concatenate([s1, s1])
    x = rng.normal(61, rng.STREAM_SIGNAL, sum(lengths))
    zi = rng.normal(61, rng.STREAM_STATE, C * kmax * 2).view(C, kmax, 2)
    return x, torch.from_numpy(sos), K, torch.tensor(lengths), zi


def _fresh(P, x, sos, K, zi, L):
    plan = P.SosFilter(L, sos.shape[1])
    y, zf = plan(x, sos, K, zi)
    assert plan.device_status() == 0
    return y.clone(), zf.clone()


def test_plan_cache_keeps_and_recomputes_exactly_what_changed():
    P = _lib()
    x, sos, K, L, zi = _case()
    xd, sd, Kd, zid = x.cuda(), sos.cuda(), K.cuda(), zi.cuda()
    C = len(L)
    plan = P.SosFilter(L, sos.shape[1])
    y0, zf0 = plan(xd, sd, Kd, zid)
    assert plan.device_status() == 0 and plan.plan_recomputed() == C
    hz, _ = plan.plan_info()
    assert int(hz[3]) == -1  # carried by the look-back
    y_ref, zf_ref = run_oracle(x, sos, K, L, zi)
    check(y0.cpu().numpy(), zf0.cpu().numpy(), y_ref, zf_ref, L.numpy(), K.numpy(), 1e-5)
    y0, zf0 = y0.clone(), zf0.clone()

    # the same inputs: nothing recomputed, the same bits
    y1, zf1 = plan(xd, sd, Kd, zid)
    assert plan.plan_recomputed() == 0
    assert torch.equal(y1, y0) and torch.equal(zf1, zf0)

    # one coefficient of channel 1 moved by one ulp: only channel 1
    s2 = sos.clone()
    s2[1, 2, 4] = float(np.nextafter(s2[1, 2, 4].item(), 2.0))
    y2, zf2 = plan(xd, s2.cuda(), Kd, zid)
    assert plan.plan_recomputed() == 1
    yf, zff = _fresh(P, xd, s2.cuda(), Kd, zid, L)
    assert torch.equal(y2, yf) and torch.equal(zf2, zff)

    # K of channel 0 changed (and channel 1 back): two channels
    K3 = K.clone()
    K3[0] = 3
    y3, zf3 = plan(xd, sd, K3.cuda(), zid)
    assert plan.plan_recomputed() == 2
    yf, zff = _fresh(P, xd, sd, K3.cuda(), zid, L)
    assert torch.equal(y3, yf) and torch.equal(zf3, zff)
    y_ref, zf_ref = run_oracle(x, sos, K3, L, zi)
    check(y3.cpu().numpy(), zf3.cpu().numpy(), y_ref, zf_ref, L.numpy(), K3.numpy(), 1e-5)

    # back to the first inputs: the first results, bit for bit
    y4, zf4 = plan(xd, sd, Kd, zid)
    assert plan.plan_recomputed() == 1
    assert torch.equal(y4, y0) and torch.equal(zf4, zf0)

    # zi and x are not plan inputs: new ones reuse every table
    y5, _ = plan(xd * 2, sd, Kd, zid * 2)
    assert plan.plan_recomputed() == 0
    assert torch.allclose(y5, 2 * y0, rtol=1e-6, atol=1e-6)

    # the replan flag recomputes everything, with the same result
    planr = P.SosFilter(L, sos.shape[1], tuning=(0, 0, 0, P._abi.SOS_FLAG_REPLAN))
    for _ in range(2):
        yr, zfr = planr(xd, sd, Kd, zid)
        assert planr.plan_recomputed() == C
    assert torch.equal(yr, y0) and torch.equal(zfr, zf0)


def test_plan_cache_under_graph_replay_with_changing_coefficients():
    """A captured prepare + apply replayed while the coefficient buffer is
    rewritten between replays: each replay filters with the current rows."""
    P = _lib()
    x, sos, K, L, zi = _case()
    xd, Kd, zid = x.cuda(), K.cuda(), zi.cuda()
    sd = sos.cuda().clone()
    plan = P.SosFilter(L, sos.shape[1])
    y = torch.empty_like(xd)
    zf = torch.empty(len(L), sos.shape[1], 2, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan(xd, sd, Kd, zid, y=y, zf=zf)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan(xd, sd, Kd, zid, y=y, zf=zf)
    other = torch.from_numpy(workloads._random_bank(62, len(L), sos.shape[1], 0.4, 0.97,
                                                    K.numpy()))
    for rows in (sos, other, other, sos):
        sd.copy_(rows.cuda())
        g.replay()
        torch.cuda.synchronize()
        yf, zff = _fresh(P, xd, rows.cuda(), Kd, zid, L)
        assert torch.equal(y, yf) and torch.equal(zf, zff)
