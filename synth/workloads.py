"""The five synthetic workloads (signals, filters, lengths, states).

Each builder returns a :class:`Workload` on the requested device.  Signals
are i.i.d. N(0, 1) FP32 (Box-Muller on SplitMix64 draws, see ``rng``);
filters come from ``filters``.  The paper states no signal length or
distribution for its 16th-order runs, so these shapes follow the workload
descriptions: a 2nd-order Butterworth low-pass on 8,192 samples, a 16th-order
(8-section) Butterworth band-pass on 2^24 samples, a batch of 4,096 channels
of uneven length with 1..8 random sections each, a near-unit-circle stress
batch, and a differentiation batch.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import torch

from . import filters, rng


@dataclasses.dataclass
class Workload:
    name: str
    x: torch.Tensor            # float32 [sum(lengths)] packed
    sos: torch.Tensor          # float64 [C, kmax, 6]
    K: torch.Tensor            # int32 [C]
    lengths: torch.Tensor      # int64 [C] (CPU copy)
    zi: Optional[torch.Tensor]  # float32 [C, kmax, 2] or None
    target: Optional[torch.Tensor] = None   # float32 like x (differentiation workload)
    sos_target: Optional[torch.Tensor] = None

    @property
    def n_channels(self) -> int:
        return int(self.sos.shape[0])

    @property
    def kmax(self) -> int:
        return int(self.sos.shape[1])

    @property
    def total(self) -> int:
        return int(self.x.numel())

    def describe(self) -> dict:
        return {"workload": self.name, "channels": self.n_channels, "kmax": self.kmax,
                "samples": self.total}


def _signal(seed: int, n: int, device) -> torch.Tensor:
    return rng.normal(seed, rng.STREAM_SIGNAL, n, device=device, dtype=torch.float32)


def plain_lowpass(n: int = 8192, seed: int = 1, device="cpu") -> Workload:
    """1 channel, K = 1: 2nd-order Butterworth low-pass, cutoff 0.1, zero state."""
    sos = torch.from_numpy(filters.butter_lowpass2_closed_form(0.1))[None].contiguous()
    return Workload("butter_lp2_wn0.1_1x%d" % n, _signal(seed, n, device), sos.to(device),
                    torch.ones(1, dtype=torch.int32, device=device),
                    torch.tensor([n], dtype=torch.int64), None)


def plain_bandpass16(n: int = 1 << 24, seed: int = 2, device="cpu") -> Workload:
    """1 channel, K = 8: 16th-order Butterworth band-pass 0.1-0.2, zero state."""
    sos = torch.from_numpy(filters.butter_bandpass(8, 0.1, 0.2))[None].contiguous()
    return Workload("butter_bp16_0.1-0.2_1x%d" % n, _signal(seed, n, device), sos.to(device),
                    torch.full((1,), 8, dtype=torch.int32, device=device),
                    torch.tensor([n], dtype=torch.int64), None)


def _random_bank(seed: int, C: int, kmax: int, rmin: float, rmax: float,
                 K: np.ndarray) -> np.ndarray:
    sos = np.zeros((C, kmax, 6))
    sos[:, :, 0] = 1.0
    sos[:, :, 3] = 1.0  # unused rows: identity sections (never read)
    total = int(K.sum())
    rows = filters.random_sections(seed, total, rmin, rmax)
    o = 0
    for c in range(C):
        sos[c, :K[c]] = rows[o:o + K[c]]
        o += K[c]
    return sos


def batched(n_channels: int = 4096, min_len: int = 1 << 10, max_len: int = 1 << 20,
            kmax: int = 8, seed: int = 3, device="cpu", rmin=0.5, rmax=0.995,
            with_state: bool = True) -> Workload:
    """Channels with lengths U-int[min_len, max_len], K U{1..kmax}, random
    stable sections (radius U[rmin, rmax], angles U[0, pi], zeros on the unit
    circle, unit peak gain per section) and N(0, 1) initial states."""
    lengths = rng.randint(seed, rng.STREAM_LENGTHS, n_channels, min_len, max_len)
    K = rng.randint(seed, rng.STREAM_SECTIONS, n_channels, 1, kmax).to(torch.int32)
    sos = _random_bank(seed, n_channels, kmax, rmin, rmax, K.numpy())
    zi = (rng.normal(seed, rng.STREAM_STATE, n_channels * kmax * 2, device=device)
          .view(n_channels, kmax, 2) if with_state else None)
    if zi is not None:
        # sections beyond K[c] carry no state
        mask = (torch.arange(kmax, device=device)[None, :] < K.to(device)[:, None])
        zi = zi * mask[:, :, None].to(zi.dtype)
    x = _signal(seed, int(lengths.sum()), device)
    return Workload("batched_%dch_len%d-%d_K1-%d" % (n_channels, min_len, max_len, kmax),
                    x, torch.from_numpy(sos).to(device), K.to(device), lengths, zi)


def precision_stress(n_channels: int = 64, length: int = 1 << 26, seed: int = 4,
                     device="cpu") -> Workload:
    """K = 8 sections per channel with poles at radius U[0.999, 0.9999],
    angles U[0, pi], zero initial state."""
    lengths = torch.full((n_channels,), length, dtype=torch.int64)
    K = torch.full((n_channels,), 8, dtype=torch.int32)
    sos = _random_bank(seed, n_channels, 8, 0.999, 0.9999, K.numpy())
    x = _signal(seed, n_channels * length, device)
    return Workload("stress_%dx%d_r0.999-0.9999_K8" % (n_channels, length), x,
                    torch.from_numpy(sos).to(device), K.to(device), lengths, None)


def differentiation(n_channels: int = 256, length: int = 1 << 16, seed: int = 5,
                    target_seed: int = 6, device="cpu") -> Workload:
    """K = 8 random sections as in the batched workload, N(0, 1) states; the
    regression target is the same input through a second random cascade
    (seed ``target_seed``), filtered by whichever implementation is under test
    or by the oracle in parity tests (``sos_target`` is returned for that)."""
    lengths = torch.full((n_channels,), length, dtype=torch.int64)
    K = torch.full((n_channels,), 8, dtype=torch.int32)
    sos = _random_bank(seed, n_channels, 8, 0.5, 0.995, K.numpy())
    sos_t = _random_bank(target_seed, n_channels, 8, 0.5, 0.995, K.numpy())
    zi = rng.normal(seed, rng.STREAM_STATE, n_channels * 8 * 2, device=device).view(n_channels, 8, 2)
    x = _signal(seed, n_channels * length, device)
    return Workload("diff_%dx%d_K8" % (n_channels, length), x, torch.from_numpy(sos).to(device),
                    K.to(device), lengths, zi, None, torch.from_numpy(sos_t).to(device))


BUILDERS = {
    "plain_lowpass": plain_lowpass,
    "plain_bandpass16": plain_bandpass16,
    "batched": batched,
    "precision_stress": precision_stress,
    "differentiation": differentiation,
}
