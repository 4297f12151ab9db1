"""The paper's early-stopping rule (App. B, "Early Stop") (TEST INFRASTRUCTURE ONLY).

GaBP stops after iteration t once mean|m_t - m_{t-1}| < tau * mean|m_2 - m_1|, the mean
running over all messages (Sec. 3.2 "Early stopping", Alg. 2).  Readings: m_i is the message
set after i iterations from the start of the run (m_0 = the initialisation); the mean runs over
both components (eta, Lambda) of every factor-variable edge; with check_every = k the rule is
evaluated after iterations 2 + k, 2 + 2k, ... (k = 1 is the paper's every-iteration check).
"""
from __future__ import annotations

import numpy as np

from . import gabp, init_messages


def message_change(new, old) -> float:
    """mean over both components of every edge of |m_new - m_old| (messages as (eta, Lambda) arrays)."""
    de = np.abs(np.asarray(new[0], np.float64) - np.asarray(old[0], np.float64))
    dl = np.abs(np.asarray(new[1], np.float64) - np.asarray(old[1], np.float64))
    return float((de.sum() + dl.sum()) / (de.size + dl.size))


def gabp_early_stop(fl, beta: float, tau: float, max_iters: int, check_every: int = 1, init: str = "cold"):
    """Run GaBP under the rule.  Returns (t, history, messages): the stopping iteration (None if
    max_iters came first), the checked changes [(t, change)] with (2, reference) first, and the
    final messages."""
    msg = init_messages(fl, init)
    _, _, m1 = gabp(fl, beta, 1, messages=msg)
    _, _, m2 = gabp(fl, beta, 1, messages=m1)
    ref = message_change(m2, m1)
    hist = [(2, ref)]
    t, cur = 2, m2
    while t < max_iters:
        chunk = min(check_every, max_iters - t)
        prev = cur
        if chunk > 1:
            _, _, prev = gabp(fl, beta, chunk - 1, messages=cur)
        _, _, cur = gabp(fl, beta, 1, messages=prev)
        t += chunk
        d = message_change(cur, prev)
        hist.append((t, d))
        if d < tau * ref:
            return t, hist, cur
    return None, hist, cur
