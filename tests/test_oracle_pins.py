"""The FP64 oracle against its pins (see tests/pins.py for what each fixes)."""
import pytest

import oracle
import pins


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(orc, pin):
    if pin is pins.pin_scipy_sosfilt:
        pytest.importorskip("scipy.signal")
    pin(orc)


def test_golden_block_permutation():
    """Paper Fig. block_permutation (L = 4, N = 8): after the permutation, block
    m holds samples m, m+N, ..., m+(L-1)N, i.e. element l of block m is sample
    l*N + m.  The CUDA path keeps exactly this layout with L = 32 warp lanes:
    lane l holds the contiguous samples [l*N, l*N + N) of a group, one per
    register m."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "block_permutation_L4_N8.txt")
    sec = None
    data = {"original": [], "permuted": []}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line in data:
            sec = line
            continue
        data[sec].append([int(v) for v in line.split()])
    L, N = 4, 8
    assert data["original"] == [[b * L + l for l in range(L)] for b in range(N)]
    assert data["permuted"] == [[l * N + m for l in range(L)] for m in range(N)]
