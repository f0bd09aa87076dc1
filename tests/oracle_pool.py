"""Run many independent FP64 oracle evaluations of one large cell in parallel (test infrastructure).

The workers are spawned processes (never forked from a process that has touched the GPU).  Each
worker receives the potential and the grid once, through the pool initialiser, then evaluates one
probe or one S-matrix beam per task with the oracle's own functions.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

from oracle import prism_oracle as O

_V = None
_G = None


def _init(V, g):
    global _V, _G
    _V, _G = V, g


def _multislice_probe(args):
    probe, det, x0, y0 = args
    return O.multislice_probe(_V, _G, probe, det, x0, y0)


def _prism_probe(args):
    probe, det, x0, y0 = args
    return O.prism_probe_direct(_V, _G, probe, det, x0, y0)


def _smatrix_beam(args):
    m, n = args
    S, _, _ = O.smatrix_build(_V, _G, beams=(np.array([m]), np.array([n])))
    return S[0]


_KINDS = {"multislice": _multislice_probe, "prism": _prism_probe, "beam": _smatrix_beam}


def evaluate(kind, V, g, items, workers=None):
    """[oracle result of each item] for kind "multislice" / "prism" (items: (probe, det, x0, y0))
    or "beam" (items: (m, n) of one plane wave; returns its stored S-matrix beam)."""
    items = list(items)
    workers = workers or max(1, min(len(items), (os.cpu_count() or 2) // 2, 8))
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"), initializer=_init,
                             initargs=(V, g)) as ex:
        return list(ex.map(_KINDS[kind], items))
