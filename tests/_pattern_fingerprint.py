"""Fingerprint of an assembled block pattern on the device: the number of
entries and the sum mod 2^64 of splitmix64(l M + j) over the entries (l, j)
of the CSR (row_ptr, col), with the output function of Steele, Lea and
Flood's SplitMix64 written out here in torch int64 arithmetic (two's
complement, wrapping multiplication; logical shifts by masking). The oracle
computes the same fingerprint from its own pattern (Oracle.pattern_hash)."""
import numpy as np

MASK64 = (1 << 64) - 1


def _signed(c):
    return c - (1 << 64) if c >= 1 << 63 else c


C1, C2 = _signed(0xbf58476d1ce4e5b9), _signed(0x94d049bb133111eb)


def _lsr(z, s):
    return (z >> s) & ((1 << (64 - s)) - 1)


def splitmix64_out(z):
    z = (z ^ _lsr(z, 30)) * C1
    z = (z ^ _lsr(z, 27)) * C2
    return z ^ _lsr(z, 31)


def device_fingerprint(rp, col, M):
    """(hash as a Python int in [0, 2^64), nnz) of one CSR on the device."""
    import torch
    counts = rp[1:] - rp[:-1]
    nnz = int(rp[-1].item() - rp[0].item())
    if nnz == 0:
        return 0, 0
    rows = torch.repeat_interleave(torch.arange(M, device=rp.device, dtype=torch.int64), counts)
    h = splitmix64_out(rows * M + col.to(torch.int64))
    return int(h.sum().item()) & MASK64, nnz
