"""The benchmark's model of the tensor-core convolution's executed work
(bench.k2_live_chunks), checked by brute force: every column of every
chunk of every tile is tested for a source sample inside the signal."""
import pytest

import bench


def brute_force(ts, lh, kc=64, nn=256, phases=16):
    n_chunks = (lh + phases - 1 + kc - 1) // kc
    n_tiles = -(-(ts + lh - 1) // (phases * nn))
    tot = 0.0
    for t in range(n_tiles):
        c0 = t * phases * nn - lh + 1
        first = True
        for ch in range(n_chunks):
            live = [n for n in range(nn)
                    if any(0 <= c0 + kc * ch + phases * n + e < ts for e in range(kc))]
            if not live:
                continue  # the kernel skips chunks whose window is all padding
            if first:
                width = nn
                first = False
            else:
                width = ((max(live) | 31) + 1) - (min(live) & ~31)
            tot += width / nn
    return tot


@pytest.mark.parametrize("ts, lh", [(16000, 8192), (3000, 700), (1, 1), (5000, 4097),
                                    (100, 9000), (4096, 4096)])
def test_executed_work_model_matches_brute_force(ts, lh):
    assert bench.k2_live_chunks(ts, lh) == pytest.approx(brute_force(ts, lh), abs=1e-12)
