"""GPU parity of the backward (adjoint) kernels against the FP64 oracle
adjoint, which the CPU pins tie to central finite differences and the
dot-product identity.

Tolerance: relative L2 error per parameter group <= 1e-4 for pole radius
<= 0.995, the accuracy target for gradients (the near-unit-circle stress
channels: 1e-3, as in the forward).  The ragged and special-case tests hold
every channel to it (dL/dx per channel; dL/db, dL/da over a channel's
sections; dL/dzi per channel); the differentiation workload is measured per
group over all its channels."""
import numpy as np
import pytest
import torch

import oracle
from synth import filters, rng, workloads

from test_gpu_forward import random_case

pytestmark = pytest.mark.gpu


def _lib():
    import paper_2607_14054_gb300 as P
    P.build()
    return P


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    n = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (n if n > 0 else 1.0))


def run_both(x, sos, K, lengths, zi, gy, gzf, tuning=None):
    P = _lib()
    plan = P.SosFilter(lengths, sos.shape[1], tuning=tuning)
    gx, gsos, gzi = plan.backward(x.cuda(), sos.cuda(), K.cuda(),
                                  zi.cuda() if zi is not None else None, gy.cuda(),
                                  gzf.cuda() if gzf is not None else None)
    st = plan.backward_status()
    assert st == 0, P._abi.STATUS_NAMES.get(st, st)
    ref = oracle.sosfilt_adjoint(x.double().numpy(), sos.numpy(), gy.double().numpy(),
                                 K=K.numpy(), lengths=lengths.numpy(),
                                 zi=zi.double().numpy() if zi is not None else None,
                                 g_zf=gzf.double().numpy() if gzf is not None else None)
    return (gx.cpu().numpy(), gsos.cpu().numpy(), gzi.cpu().numpy()), ref


def check_grads(got, ref, lengths, K, tol):
    gx, gsos, gzi = got
    rx, rsos, rzi = ref
    off = np.concatenate([[0], np.cumsum(lengths)])
    worst = {"x": 0.0, "b": 0.0, "a": 0.0, "zi": 0.0}
    for c in range(len(lengths)):
        k = int(K[c])
        if lengths[c] > 0:
            worst["x"] = max(worst["x"], _rel(gx[off[c]:off[c + 1]], rx[off[c]:off[c + 1]]))
        if k == 0:
            assert np.all(gsos[c] == 0)
            continue
        worst["b"] = max(worst["b"], _rel(gsos[c, :k, :3], rsos[c, :k, :3]))
        worst["a"] = max(worst["a"], _rel(gsos[c, :k, 3:], rsos[c, :k, 3:]))
        worst["zi"] = max(worst["zi"], _rel(gzi[c, :k], rzi[c, :k]))
        assert np.all(gsos[c, k:] == 0) and np.all(gzi[c, k:] == 0)
    assert all(v <= tol for v in worst.values()), worst
    return worst


@pytest.mark.parametrize("N", [16, 32, 64])
def test_adjoint_ragged_multichannel(N):
    """Ragged lengths around the group size, multi-segment channels, a0 != 1,
    random zi, dL/dy and dL/dzf."""
    G = 32 * N
    lengths = [1, 2, 3, G - 1, G, G + 1, 5 * G + 7, 0, 70_001, 200_000]
    x, sos, K, L, zi = random_case(300 + N, lengths, 8, rmax=0.95)
    gy = rng.normal(301 + N, rng.STREAM_SIGNAL, int(L.sum()))
    gzf = rng.normal(302 + N, rng.STREAM_STATE, len(lengths) * 16).view(len(lengths), 8, 2)
    got, ref = run_both(x, sos, K, L, zi, gy, gzf, tuning=(N, 8, 0, 0))
    print(check_grads(got, ref, np.array(lengths), K.numpy(), 1e-4))


def test_adjoint_general_mode_identity_and_no_state():
    """A section with b0 = 0 (no b0 factoring), a K = 0 channel, no zi, no
    dL/dzf, and an empty channel that passes dL/dzf through to dL/dzi."""
    lengths = [5000, 70000, 300, 0]
    x, sos, K, L, zi = random_case(7, lengths, 4, b0_zero_channel=1, with_zi=False)
    K[2] = 0
    gy = rng.normal(8, rng.STREAM_SIGNAL, int(L.sum()))
    got, ref = run_both(x, sos, K, L, None, gy, None)
    print(check_grads(got, ref, np.array(lengths), K.numpy(), 1e-4))
    off = np.concatenate([[0], np.cumsum(lengths)])
    assert np.array_equal(got[0][off[2]:off[3]], gy[off[2]:off[3]].numpy())
    # empty channel with dL/dzf: dL/dzi = dL/dzf
    gzf = torch.ones(len(lengths), 4, 2)
    got, ref = run_both(x, sos, K, L, zi, gy, gzf)
    assert np.allclose(got[2][3, :K[3]], 1.0)


def test_adjoint_long_memory_channels():
    """Poles at radius 0.999..0.9999 have no memory horizon: the backward runs
    each such channel as one segment; mixed with short-memory channels."""
    lengths = [150_000, 60_000, 90_000]
    C, kmax = 3, 8
    K = np.array([8, 4, 6], dtype=np.int32)
    sos = np.zeros((C, kmax, 6))
    sos[:, :, 0] = 1.0
    sos[:, :, 3] = 1.0
    for c, k in enumerate(K):
        rmin, rmax = (0.999, 0.9999) if c != 1 else (0.5, 0.95)
        sos[c, :k] = filters.random_sections(60 + c, int(k), rmin, rmax)
    x = rng.normal(61, rng.STREAM_SIGNAL, sum(lengths))
    zi = rng.normal(61, rng.STREAM_STATE, C * kmax * 2).view(C, kmax, 2)
    gy = rng.normal(62, rng.STREAM_SIGNAL, sum(lengths))
    gzf = rng.normal(63, rng.STREAM_STATE, C * kmax * 2).view(C, kmax, 2)
    got, ref = run_both(x, torch.from_numpy(sos), torch.from_numpy(K), torch.tensor(lengths), zi,
                        gy, gzf)
    print(check_grads(got, ref, np.array(lengths), K, 1e-3))


def test_autograd_function_matches_oracle_adjoint():
    """torch.autograd through sosfilt_diff: L = <y, w> + <zf, v>."""
    P = _lib()
    lengths = [40_000, 9_000]
    x, sos, K, L, zi = random_case(70, lengths, 8, rmax=0.97)
    w = rng.normal(71, rng.STREAM_SIGNAL, int(L.sum()))
    v = rng.normal(72, rng.STREAM_STATE, 2 * 16).view(2, 8, 2)
    xg = x.cuda().requires_grad_(True)
    sg = sos.cuda().requires_grad_(True)
    zg = zi.cuda().requires_grad_(True)
    y, zf = P.sosfilt_diff(xg, sg, K.cuda(), lengths=L, zi=zg)
    loss = (y * w.cuda()).sum() + (zf * v.cuda()).sum()
    loss.backward()
    rx, rsos, rzi = oracle.sosfilt_adjoint(x.double().numpy(), sos.numpy(), w.double().numpy(),
                                           K=K.numpy(), lengths=L.numpy(), zi=zi.double().numpy(),
                                           g_zf=v.double().numpy())
    assert _rel(xg.grad.cpu().numpy(), rx) <= 1e-4
    assert _rel(sg.grad.cpu().numpy(), rsos) <= 1e-4
    assert _rel(zg.grad.cpu().numpy(), rzi) <= 1e-4


def test_differentiation_workload_full_size():
    """256 channels x 2^16, K = 8 random sections (radius <= 0.995), MSE loss
    against the same input through a second random cascade (the oracle's
    output is the target); every gradient against the oracle adjoint."""
    P = _lib()
    wl = workloads.differentiation()
    L = wl.lengths
    xn = wl.x.double().numpy()
    target, _ = oracle.sosfilt(xn, wl.sos_target.numpy(), K=wl.K.numpy(), lengths=L.numpy(),
                               zi=wl.zi.double().numpy())
    xg = wl.x.cuda().requires_grad_(True)
    sg = wl.sos.cuda().requires_grad_(True)
    zg = wl.zi.cuda().requires_grad_(True)
    y, zf = P.sosfilt_diff(xg, sg, wl.K.cuda(), lengths=L, zi=zg)
    tgt = torch.from_numpy(target).float().cuda()
    loss = ((y - tgt) ** 2).mean()
    loss.backward()
    # the oracle's gradient of the same loss at the oracle's own y
    y_ref, _ = oracle.sosfilt(xn, wl.sos.numpy(), K=wl.K.numpy(), lengths=L.numpy(),
                              zi=wl.zi.double().numpy())
    g_y = 2.0 * (y_ref - target) / y_ref.size
    rx, rsos, rzi = oracle.sosfilt_adjoint(xn, wl.sos.numpy(), g_y, K=wl.K.numpy(),
                                           lengths=L.numpy(), zi=wl.zi.double().numpy())
    gx, gsos, gzi = (xg.grad.cpu().numpy(), sg.grad.cpu().numpy(), zg.grad.cpu().numpy())
    # relative L2 per parameter group over all channels (x, zi, b, a).  A few
    # of these random cascades have a total gain near 1e-12 (eight unit-peak
    # sections that cancel each other): there even a sequential FP32 DF2T is
    # off by ~1e-3 relative, but their gradients are as small as their gain,
    # so they do not move the group norms.
    groups = {"x": _rel(gx, rx), "zi": _rel(gzi, rzi), "b": _rel(gsos[..., :3], rsos[..., :3]),
              "a": _rel(gsos[..., 3:], rsos[..., 3:])}
    print(groups)
    assert all(v <= 1e-4 for v in groups.values()), groups


def test_adjoint_long_memory_several_segments():
    """Channels with poles at radius 0.99..0.995 (memory horizons of a few
    thousand samples) long enough to be cut into many backward segments
    (each warmed up over its horizon on both sides): every gradient group
    within 1e-4 of the oracle adjoint, and the plan really cut them."""
    from synth import filters
    P = _lib()
    C, kmax, n = 6, 4, 1 << 19
    lengths = torch.full((C,), n, dtype=torch.int64)
    K = torch.full((C,), kmax, dtype=torch.int32)
    sos = np.zeros((C, kmax, 6))
    for c in range(C):
        sos[c] = filters.random_sections(700 + c, kmax, 0.99, 0.995)
    sos = torch.from_numpy(sos)
    x = rng.normal(701, rng.STREAM_SIGNAL, C * n)
    zi = rng.normal(701, rng.STREAM_STATE, C * kmax * 2).view(C, kmax, 2)
    gy = rng.normal(702, rng.STREAM_SIGNAL, C * n)
    gzf = rng.normal(703, rng.STREAM_STATE, C * kmax * 2).view(C, kmax, 2)
    got, ref = run_both(x, sos, K, lengths, zi, gy, gzf)
    worst = check_grads(got, ref, lengths.numpy(), K.numpy(), 1e-4)
    # the backward plan's segments: the channel table of the backward
    # workspace (its channel table follows the header, as in the forward's)
    plan = P.SosFilter(lengths, kmax)
    plan.backward(x.cuda(), sos.cuda(), K.cuda(), zi.cuda(), gy.cuda(), gzf.cuda())
    h = torch.empty(C, dtype=torch.int32)
    t = torch.empty(C, dtype=torch.int32)
    st = P._abi.sos_plan_query(plan._bws.data_ptr(), 0, C, h.data_ptr(), t.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert st == 0
    assert (h > 1000).all() and (t >= 4).all(), (h, t)
    print("long-memory adjoint", worst, "horizons", h.tolist(), "segments", t.tolist())


def test_adjoint_repeated_poles_several_segments():
    """Cascades whose sections come in identical pairs (repeated poles, as
    in Linkwitz-Riley filters) have no partial-fraction memory horizon; the
    backward plan bounds their memory without one (C(n + 2K - 1, 2K - 1) r^n
    over the largest pole radius r) and still cuts long channels into
    segments: every gradient group within 1e-4 of the oracle adjoint."""
    from synth import filters
    P = _lib()
    C, kmax, n = 4, 4, 1 << 19
    lengths = torch.full((C,), n, dtype=torch.int64)
    K = torch.full((C,), kmax, dtype=torch.int32)
    sos = np.zeros((C, kmax, 6))
    for c in range(C):
        half = filters.random_sections(800 + c, kmax // 2, 0.95, 0.99)
        sos[c, 0::2] = half
        sos[c, 1::2] = half
    sos = torch.from_numpy(sos)
    x = rng.normal(801, rng.STREAM_SIGNAL, C * n)
    zi = rng.normal(801, rng.STREAM_STATE, C * kmax * 2).view(C, kmax, 2)
    gy = rng.normal(802, rng.STREAM_SIGNAL, C * n)
    gzf = rng.normal(803, rng.STREAM_STATE, C * kmax * 2).view(C, kmax, 2)
    got, ref = run_both(x, sos, K, lengths, zi, gy, gzf)
    worst = check_grads(got, ref, lengths.numpy(), K.numpy(), 1e-4)
    plan = P.SosFilter(lengths, kmax)
    plan.backward(x.cuda(), sos.cuda(), K.cuda(), zi.cuda(), gy.cuda(), gzf.cuda())
    h = torch.empty(C, dtype=torch.int32)
    t = torch.empty(C, dtype=torch.int32)
    st = P._abi.sos_plan_query(plan._bws.data_ptr(), 0, C, h.data_ptr(), t.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert st == 0
    assert (h > 0).all() and (t >= 4).all(), (h, t)
    # the forward plan of the same (long) channels takes the same horizons
    plan.prepare(sos.cuda(), K.cuda())
    hf, _ = plan.plan_info()
    assert torch.equal(hf, h), (hf, h)
    print("repeated-pole adjoint", worst, "horizons", h.tolist(), "segments", t.tolist())
