"""Merge of prediction times into training times (Sec. 4.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The M prediction times are inserted into the sorted N training times and
treated as missing measurements.  Reading for ties (the paper does not discuss
them): a stable merge, training point first at equal times.  A library stable
sort serves as the merge step.
"""
from __future__ import annotations

import numpy as np


def merge(t_train: np.ndarray, y_train: np.ndarray, t_test: np.ndarray):
    """Returns (t, y, mask, test_pos): merged times, observations (0 at test
    steps), mask (1 = observed) and the merged index of each test point."""
    N, M = t_train.size, t_test.size
    t_all = np.concatenate([t_train, t_test])
    order = np.argsort(t_all, kind="stable")     # ties keep training first
    t = t_all[order]
    y = np.concatenate([y_train, np.zeros(M)])[order]
    mask = np.concatenate([np.ones(N, np.uint8), np.zeros(M, np.uint8)])[order]
    inv = np.empty(N + M, np.int64)
    inv[order] = np.arange(N + M)
    test_pos = inv[N:]
    return t, y, mask, test_pos
