"""FP64 estimators of the oracle (TEST INFRASTRUCTURE; see oracle/__init__.py).

Per bin b with k_b samples tallied as (q0, q1, q2, q3) by Alg. Phase 4c:
  c_hat_b = (q1 + q2 + q3) / k_b                         (Thm 3.2)
  t_hat_b = p_b * (q1 + q2/2 + q3/3) / k_b               (Thm 3.3)
  eps_b   = sqrt(ln(2/delta) / (2 k_b))                  (Thm 3.1 solved for eps)
Global from bins, Eq. (global_est), Sec. 4.6:
  c_hat = sum_b (p_b / p) c_hat_b,   t_hat = c_hat * p / 3
Global stream (one bin of every degree >= 2, Sec. 4.2 special case):
  c_hat_g = closed / k_g,   t_hat_g = c_hat_g * p / 3     (Eq. (CC): c = 3t/p)
Bins with k_b = 0 report c_hat_b = t_hat_b = 0.
"""
from __future__ import annotations

import math

import numpy as np


def estimate(p_b, counts, glob, delta: float):
    p_b = [int(x) for x in p_b]
    counts = np.asarray(counts, dtype=np.uint64)
    p = sum(p_b)
    c_b, t_b, e_b = [], [], []
    for b, pb in enumerate(p_b):
        k, q0, q1, q2, q3 = (int(x) for x in counts[b])
        if k == 0:
            c_b.append(0.0)
            t_b.append(0.0)
            e_b.append(0.0)
            continue
        c_b.append((q1 + q2 + q3) / k)
        t_b.append(pb * (q1 + q2 / 2.0 + q3 / 3.0) / k)
        e_b.append(math.sqrt(math.log(2.0 / delta) / (2.0 * k)))
    c_hat = sum((pb / p) * cb for pb, cb in zip(p_b, c_b)) if p > 0 else 0.0
    kg, closed = int(glob[0]), int(glob[1])
    c_g = closed / kg if kg > 0 else 0.0
    return {
        "p": p,
        "c_b": c_b,
        "t_b": t_b,
        "eps_b": e_b,
        "c_hat": c_hat,
        "t_hat": c_hat * p / 3.0,
        "c_hat_global": c_g,
        "t_hat_global": c_g * p / 3.0,
        "eps_global": math.sqrt(math.log(2.0 / delta) / (2.0 * kg)) if kg > 0 else 0.0,
    }
