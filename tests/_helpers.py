"""Shared test helpers (no method arithmetic: comparisons only)."""
import numpy as np

import oracle as O

TIE_REL = 1e-6   # blocks whose measure lies within this relative band of tau may go either way


def states_within_tie_band(gpu_states, measure, tau, cfg, classifier=None):
    """True if every GPU block state lies between the oracle's states with the
    tie-band blocks all inactive and all active (states are monotone in the
    active set, so any valid choice for the tie-band blocks lands in between).
    `classifier`: the oracle's classify (default) or classify_half."""
    classifier = classifier or O.classify
    measure = np.asarray(measure, dtype=np.float64)
    tie = np.abs(measure - tau) <= TIE_REL * tau
    lo = classifier(np.where(tie, -np.inf, measure), tau, force_dc=cfg.force_dc, transitions=cfg.transitions)
    hi = classifier(np.where(tie, np.inf, measure), tau, force_dc=cfg.force_dc, transitions=cfg.transitions)
    g = np.asarray(gpu_states)
    return bool(np.all((g >= lo) & (g <= hi))), int(np.count_nonzero(tie))


def rel_l2(a, b):
    return O.rel_l2(a, b)
