"""Launch configuration and the column tile autotuner: the chosen path per
grid, and bit-identical results for every column tile width."""
import os

import numpy as np
import pytest

import paper_1804_02883_gb300 as P
from paper_1804_02883_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(r, nsteps, width=None):
    old = os.environ.get("EPD_LB_COLUMN_TILE")
    if width is None:
        os.environ.pop("EPD_LB_COLUMN_TILE", None)
    else:
        os.environ["EPD_LB_COLUMN_TILE"] = str(width)
    try:
        h = P.EpdLb([r])
    finally:
        if old is None:
            os.environ.pop("EPD_LB_COLUMN_TILE", None)
        else:
            os.environ["EPD_LB_COLUMN_TILE"] = old
    tiles = h.tiles(0)
    h.step(nsteps)
    phi, q = h.densities(0)
    om, pop, vel = h.get_state(0)
    h.close()
    return tiles, phi, q, om, pop, vel


@pytest.mark.parametrize("ny,nx,path", [(64, 64, 2), (256, 512, 2), (64, 1024, 1)])
def test_column_tile_width_does_not_change_results(ny, nx, path):
    r = W.with_(W.plain_small(), nx=nx, ny=ny, ns=16, precision=P.MIXED_FP32, f0=1.0)
    ref = None
    for w in (4, 8, 16):
        tiles, *state = _run(r, 3, w)
        assert tiles["path"] == path
        assert tiles["column_tile"] == w
        assert tiles["stream_column_tile"] == (w if path == 1 else 0)
        if ref is None:
            ref = state
        else:
            for a, b in zip(state, ref):
                assert np.array_equal(a, b)


def test_autotuner_picks_a_width_and_paths():
    r = W.with_(W.plain_small(), precision=P.MIXED_FP32)
    tiles, *_ = _run(r, 1)
    assert tiles["path"] == 2 and tiles["cluster_ctas"] >= 2 and tiles["differential"]
    assert tiles["column_tile"] in (4, 8, 16)
    t64, *_ = _run(W.plain_small(), 1)
    assert t64 == {"path": 0, "cluster_ctas": 0, "column_tile": 0, "differential": False, "stream_column_tile": 0,
                   "chain_launches": 0}
    assert tiles["chain_launches"] == 1  # one run: both chains in one launch
    ts, *_ = _run(W.with_(r, nx=1024, ny=64, ns=8), 1)
    assert ts["path"] == 1 and ts["stream_column_tile"] in (4, 8, 16) and ts["differential"]
