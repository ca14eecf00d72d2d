"""The allocation-free entry point (sos_filter_static) against sos_filter.

Some callers cannot allocate device memory (real-time callbacks, plug-ins
inside an application that owns the allocator); sos_filter_static serves
them with a fixed library-owned scratch array.  This file is collected last
on purpose: if it fails, a run that stops at the first failure has already
run every other test.  It must pass both alone in a fresh process and after
the other tests (the scratch array keeps the previous call's contents)."""
import numpy as np
import pytest
import torch

import oracle
from synth import rng, workloads

pytestmark = pytest.mark.gpu


def _case(seed, lengths, kmax=8):
    C = len(lengths)
    L = torch.tensor(lengths, dtype=torch.int64)
    K = rng.randint(seed, rng.STREAM_SECTIONS, C, 1, kmax).to(torch.int32)
    sos = torch.from_numpy(workloads._random_bank(seed, C, kmax, 0.3, 0.97, K.numpy()))
    x = rng.normal(seed, rng.STREAM_SIGNAL, int(L.sum()))
    zi = rng.normal(seed, rng.STREAM_STATE, C * kmax * 2).view(C, kmax, 2)
    return x, sos, K, L, zi


def _static(P, x, sos, K, L, zi):
    C, kmax = sos.shape[0], sos.shape[1]
    xd, sd, Kd, Ld, zid = x.cuda(), sos.cuda().contiguous(), K.cuda(), L.cuda(), zi.cuda()
    y = torch.empty_like(xd)
    zf = torch.empty(C, kmax, 2, device="cuda")
    Lh = L.contiguous()
    st, dev_st = P._abi.sos_filter_static(xd.data_ptr(), sd.data_ptr(), Kd.data_ptr(), C, kmax,
                                          Ld.data_ptr(), Lh.data_ptr(), zid.data_ptr(), y.data_ptr(),
                                          zf.data_ptr(), None,
                                          torch.cuda.current_stream().cuda_stream)
    return st, dev_st, y, zf


def test_static_entry_point_matches_sos_filter_twice():
    import paper_2607_14054_gb300 as P
    P.build()
    for seed, lengths in ((21, [70_000, 3, 120_001]), (22, [9_999, 250_000])):
        x, sos, K, L, zi = _case(seed, lengths)
        st, dev_st, y, zf = _static(P, x, sos, K, L, zi)
        assert st == 0 and dev_st == 0, (st, dev_st)
        y_ref, zf_ref = P.sosfilt(x.cuda(), sos.cuda(), K=K.cuda(), lengths=L, zi=zi.cuda(),
                                  check=True)
        torch.cuda.synchronize()
        yo, _ = oracle.sosfilt(x.double().numpy(), sos.numpy(), K=K.numpy(), lengths=L.numpy(),
                               zi=zi.double().numpy())
        err_static = oracle.rel_l2_per_channel(y.cpu().numpy(), yo, L.numpy())
        err_ref = oracle.rel_l2_per_channel(y_ref.cpu().numpy(), yo, L.numpy())
        assert err_static.max() <= 1e-5 and err_ref.max() <= 1e-5
        assert torch.allclose(y, y_ref, rtol=1e-5, atol=1e-6)
        assert torch.allclose(zf, zf_ref, rtol=1e-4, atol=1e-6)


def test_static_entry_point_rejects_oversized_requests():
    import paper_2607_14054_gb300 as P
    P.build()
    lengths = torch.full((4096,), 1 << 20, dtype=torch.int64)  # workspace far beyond 8 MiB
    st, _ = P._abi.sos_filter_static(0, 0, 0, 4096, 8, 0, lengths.data_ptr(), 0, 0, 0, None, 0,
                                     want_status=False)
    assert st == -5  # SOS_ERR_WORKSPACE, nothing enqueued


_FIRST_CALL_ON_SIDE_STREAM = r'''
import sys, torch
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
import paper_2607_14054_gb300 as P
from test_zz_no_alloc import _case
x, sos, K, L, zi = _case(23, [50_000, 7, 160_003])
s = torch.cuda.Stream()          # created non-blocking, like every torch stream
C, kmax = sos.shape[0], sos.shape[1]
xd, sd, Kd, Ld, zid = x.cuda(), sos.cuda().contiguous(), K.cuda(), L.cuda(), zi.cuda()
torch.cuda.synchronize()
with torch.cuda.stream(s):
    y = torch.empty_like(xd)
    zf = torch.empty(C, kmax, 2, device="cuda")
    # the first call of this process on the device: the set-up zeroes the
    # array on this stream before the call's own kernels
    st, _ = P._abi.sos_filter_static(xd.data_ptr(), sd.data_ptr(), Kd.data_ptr(), C, kmax,
                                     Ld.data_ptr(), L.data_ptr(), zid.data_ptr(), y.data_ptr(),
                                     zf.data_ptr(), None, s.cuda_stream, want_status=False)
    assert st == 0, st
s.synchronize()
y_ref, zf_ref = P.sosfilt(xd, sd, K=Kd, lengths=L, zi=zid, check=True)
torch.cuda.synchronize()
assert torch.allclose(y, y_ref, rtol=1e-5, atol=1e-6), float((y - y_ref).abs().max())
assert torch.allclose(zf, zf_ref, rtol=1e-4, atol=1e-6)
print("side-stream first call ok")
'''


def test_static_first_call_on_a_non_blocking_stream():
    """A fresh process whose very first sos_filter_static call is made on a
    non-blocking stream: the array's zeroing must be complete before that
    call's kernels run, whatever the stream."""
    import os
    import subprocess
    import sys
    import paper_2607_14054_gb300 as P
    P.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL_ON_SIDE_STREAM, root],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "side-stream first call ok" in r.stdout


def test_static_refuses_status_read_under_capture():
    """device_status needs a stream wait, which a capture forbids: the call
    is refused (SOS_ERR_ARG) before anything is enqueued."""
    import paper_2607_14054_gb300 as P
    P.build()
    x, sos, K, L, zi = _case(24, [4096])
    _static(P, x, sos, K, L, zi)  # set-up done outside the capture
    C, kmax = sos.shape[0], sos.shape[1]
    xd, sd, Kd, Ld = x.cuda(), sos.cuda().contiguous(), K.cuda(), L.cuda()
    y = torch.empty_like(xd)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        st, _ = P._abi.sos_filter_static(xd.data_ptr(), sd.data_ptr(), Kd.data_ptr(), C, kmax,
                                         Ld.data_ptr(), L.data_ptr(), 0, y.data_ptr(), 0, None,
                                         s.cuda_stream, want_status=True)
    assert st == -1
