"""The comparison algorithms of the paper's evaluation (sos_apply_baseline):
the scalar recursion and block filtering (Sec. IV, Eq.
block_filtering_equation), on the same tables and segmentation as the
method, against the oracle on ragged packed channels (outputs and final
states)."""
import numpy as np
import pytest
import torch

from test_gpu_forward import _lib, check, random_case, run_oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("algorithm", ["scalar", "block"])
@pytest.mark.parametrize("seg_len", [64, 1000, 8192])
def test_baseline_algorithms_match_oracle(algorithm, seg_len):
    P = _lib()
    lengths = [1, 2, 31, 32, 33, 1000, 0, 70_001, 5, 250_000]
    x, sos, K, L, zi = random_case(151 + seg_len, lengths, 8, rmax=0.95)
    K[3] = 0
    plan = P.SosFilter(L, 8)
    xd, sd, Kd, zid = x.cuda(), sos.cuda(), K.cuda(), zi.cuda()
    plan.prepare(sd, Kd)
    y = torch.empty_like(xd)
    zf = torch.empty(len(lengths), 8, 2, device="cuda")
    plan.apply_baseline(algorithm, xd, y, seg_len, zid, zf)
    assert plan.device_status() == 0
    y_ref, zf_ref = run_oracle(x, sos, K, L, zi)
    check(y.cpu().numpy(), zf.cpu().numpy(), y_ref, zf_ref, L.numpy(), K.numpy(), 1e-5)
