"""The library's host clustering (word-parallel Berger-Rigoutsos on flag
bitmaps, the code every regrid runs) gives the oracle's boxes, box for box,
on exhaustive small fields and on random fields with nesting masks (no GPU)."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_1511_03645_gb300 import adjamr as A


def _same(flags, mc, eff, nest=None):
    got = A.cluster_boxes(flags, mc=mc, eff=eff, nest=nest)
    want = O.cluster(flags, mc=mc, eff=eff, nest=nest)
    assert np.array_equal(got, want), (flags, got, want)


def test_all_3x4_fields():
    for bits in itertools.product((0, 1), repeat=12):
        f = np.array(bits, dtype=np.uint8).reshape(3, 4)
        _same(f, 1, 0.7)


@pytest.mark.parametrize("seed", range(6))
def test_random_fields_with_nesting_masks(seed):
    rng = np.random.default_rng(seed)
    for _ in range(60):
        M = 1 if rng.random() < 0.2 else int(rng.integers(1, 130))
        N = int(rng.integers(1, 200))
        dens = rng.random() * 0.3
        flags = (rng.random((M, N)) < dens).astype(np.uint8)
        # blobs: several flagged discs
        yy, xx = np.mgrid[0:M, 0:N]
        for _ in range(int(rng.integers(0, 4))):
            cx, cy, r = rng.integers(0, N), rng.integers(0, M), rng.integers(1, 20)
            flags |= (((xx - cx) ** 2 + (yy - cy) ** 2) < r * r).astype(np.uint8)
        nest = None
        if rng.random() < 0.6:
            nest = (rng.random((M, N)) > 0.03).astype(np.uint8)
        _same(flags, int(rng.integers(1, 5)), float(rng.uniform(0.5, 0.9)), nest)


def test_rejects_bad_arguments():
    with pytest.raises(A.AdjamrError):
        A.cluster_boxes(np.zeros((2, 3), np.uint8), mc=0)
