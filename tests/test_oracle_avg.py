"""Pins of the oracle's channel-averaging weights (Sec. 2.6) against hand-derived tables."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "avg_weights.txt")


def _cases():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, body, tot = (s.strip() for s in line.split("|"))
        N, F, dc, j = (int(v) for v in head.split())
        w = {int(c): float(x) for c, x in (kv.split(":") for kv in body.split())}
        out.append((N, F, dc, j, w, float(tot)))
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: f"N{c[0]}F{c[1]}dc{c[2]}j{c[3]}")
def test_weights_golden(case):
    N, F, dc, j, expect, tot = case
    w, s = oracle.avg_weights(N, F, dc, j)
    full = np.zeros(N)
    for c, x in expect.items():
        full[c] = x
    assert np.array_equal(w, full)
    assert s == tot


@pytest.mark.parametrize("N,F", [(128, 4), (6400, 50), (6400, 200), (1280, 10), (1280, 40), (32, 1), (20, 4), (10, 5)])
def test_weights_partition_of_unity(N, F):
    # Sec. 2.6: away from the coarse-channel edges every frequency contributes equally:
    # summed over the output channels, each interior bin has total weight exactly 1,
    # DC excepted (excluded from the centre channel when F > 1).  Near the edges the
    # totals can only be 0, 1/2 or 1 (half-channels).
    M = N // F
    tot = np.zeros(N)
    for j in range(M):
        tot += oracle.avg_weights(N, F, 1, j)[0]
    u = np.arange(N) - N // 2
    interior = np.abs(u) <= N // 2 - F
    dc = (u == 0) & (F > 1)
    assert np.all(tot[interior & ~dc] == 1.0)
    assert np.all(tot[dc] == 0.0)
    assert set(np.unique(tot[~interior])) <= {0.0, 0.5, 1.0}
