"""The pattern fingerprint used by the full-size GPU parity tests, checked on
the CPU: the torch SplitMix64 output function against the first outputs of
the published generator (seed 0), and the oracle's per-block fingerprint over
all rows against the same fingerprint computed from the oracle's own rows."""
import numpy as np

from _pattern_fingerprint import MASK64, device_fingerprint, splitmix64_out
from oracle.oracle import Oracle
from paper_1503_07221_gb300 import inputs


def test_splitmix64_published_sequence():
    import torch
    # SplitMix64, seed 0: state advances by the golden gamma, outputs are mix(state)
    gamma = 0x9e3779b97f4a7c15
    want = [0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f]
    st = [((k + 1) * gamma) & MASK64 for k in range(3)]
    z = torch.tensor([s - (1 << 64) if s >= 1 << 63 else s for s in st], dtype=torch.int64)
    got = [int(v) & MASK64 for v in splitmix64_out(z)]
    assert got == want


def test_oracle_fingerprint_matches_its_rows():
    import torch
    V, F = inputs.icosphere(1)
    t = inputs.equidistant_grid(9, 2.0)
    o = Oracle(V, F, t)
    nb, M = o.num_blocks(), o.M
    hs, nz = o.pattern_hash(np.arange(nb))
    res = o.assemble_rows(np.arange(M), np.arange(nb))
    for b in range(nb):
        cols = [c for (c, f, n) in res[b]]
        rp = torch.tensor(np.concatenate([[0], np.cumsum([len(c) for c in cols])]), dtype=torch.int64)
        col = torch.tensor(np.concatenate(cols), dtype=torch.int32)
        h, n = device_fingerprint(rp, col, M)
        assert n == nz[b] and h == int(hs[b]), b
