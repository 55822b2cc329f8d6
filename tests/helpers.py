"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle as O
from paper_1804_02883_gb300.binding import RunParams


def oracle_params(r: RunParams) -> O.Params:
    d = {f.name: getattr(r, f.name) for f in dataclasses.fields(O.Params)}
    return O.Params(**d)


def rel_err(got, want) -> float:
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = np.abs(want).max()
    if scale == 0:
        return float(np.abs(got).max())
    return float(np.abs(got - want).max() / scale)


def fluct_err(got, want) -> float:
    """Error relative to the spread of `want` around its mean (for fields whose
    mean carries no information, e.g. omega around 0 or Phi around phi_p)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    spread = np.abs(want - want.mean()).max()
    return float(np.abs(got - want).max() / spread) if spread > 0 else float(np.abs(got - want).max())


def vel_err(got, want, rtol: float, floor: float = 1e-15) -> float:
    """Velocity error in units of the tolerance rtol * max|u| + floor (pass if
    < 1).  The floor reflects that the oracle forms j = sum_i n_i c_i from O(1)
    populations, which resolves the velocity only to ~1e-16 absolute."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    return float(np.abs(got - want).max() / (rtol * np.abs(want).max() + floor))
