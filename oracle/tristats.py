"""Triangle statistics of sampled wedges (TEST INFRASTRUCTURE; see
oracle/__init__.py).

Sec. 5.7: with one bin of all degrees, the closed wedges among uniform wedge
samples are uniform triangles (Thm 3.4). Each sampled triangle has a smallest
and a largest vertex degree. Triangles are grouped by the bin of the smallest
degree, BinId of Eq. (binid) with tau = 2 and omega = 2, and every group's
largest degrees are summarised as a box plot.

The paper does not define its box plot's quantiles or whiskers. Readings
taken here:
  * quartiles by nearest rank: the ceil(p c)-th smallest of the group's c
    values, p = 1/4, 1/2, 3/4 (exact rational arithmetic);
  * whiskers at 1.5 times the interquartile range beyond the box: a value v
    is an outlier iff v < q1 - 1.5 (q3 - q1) or v > q3 + 1.5 (q3 - q1); the
    whiskers are the smallest and largest values that are not outliers;
  * the max/min degree ratio of a triangle is the FP64 quotient d_max / d_min
    (one correctly rounded division), summarised over all sampled triangles
    by the same nearest-rank rule (min, q1, median, q3, max).
Plain Python over sorted lists; no blocking or reordering.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from . import STAT_BINS, bin_id, sample

BOX_FIELDS = ("count", "min", "q1", "median", "q3", "max", "whisker_lo", "whisker_hi", "outliers")


def nearest_rank(sorted_vals, p: Fraction):
    """The ceil(p c)-th smallest (1-based) of c sorted values (at least the 1st)."""
    c = len(sorted_vals)
    r = max(1, math.ceil(p * c))
    return sorted_vals[r - 1]


def box(values):
    """Box-plot summary of a list of integers, as a dict over BOX_FIELDS."""
    vals = sorted(int(v) for v in values)
    if not vals:
        return {f: 0 for f in BOX_FIELDS}
    q1 = nearest_rank(vals, Fraction(1, 4))
    med = nearest_rank(vals, Fraction(1, 2))
    q3 = nearest_rank(vals, Fraction(3, 4))
    iqr = Fraction(q3 - q1)
    lo_bound = q1 - Fraction(3, 2) * iqr
    hi_bound = q3 + Fraction(3, 2) * iqr
    inside = [v for v in vals if lo_bound <= v <= hi_bound]
    return {"count": len(vals), "min": vals[0], "q1": q1, "median": med, "q3": q3, "max": vals[-1],
            "whisker_lo": min(inside), "whisker_hi": max(inside), "outliers": len(vals) - len(inside)}


def summarise(records):
    """Summary of the closed samples among records (rows v0, v1, v2, closed,
    d0, d1, d2, 0): box[STAT_BINS, 9] by BinId(d_min) (tau = 2, omega = 2),
    ratio_q[5] of d_max / d_min, hist[STAT_BINS, STAT_BINS] of
    (BinId(d_min), BinId(d_max)), and the number of closed samples."""
    groups = {}
    ratios = []
    hist = np.zeros((STAT_BINS, STAT_BINS), np.uint64)
    closed = 0
    rec = np.asarray(records)
    for row in rec[rec[:, 3] != 0]:
        closed += 1
        ds = sorted(int(x) for x in row[4:7])
        dmin, dmax = ds[0], ds[2]
        bmin, bmax = bin_id(dmin, 2, 2), bin_id(dmax, 2, 2)
        groups.setdefault(bmin, []).append(dmax)
        ratios.append(float(dmax) / float(dmin))
        hist[bmin, bmax] += 1
    out = np.zeros((STAT_BINS, len(BOX_FIELDS)), np.uint64)
    for b, vals in groups.items():
        s = box(vals)
        out[b] = [s[f] for f in BOX_FIELDS]
    ratio_q = np.zeros(5, np.float64)
    if ratios:
        r = sorted(ratios)
        ratio_q[:] = [r[0], nearest_rank(r, Fraction(1, 4)), nearest_rank(r, Fraction(1, 2)),
                      nearest_rank(r, Fraction(3, 4)), r[-1]]
    return {"closed": closed, "box": out, "ratio_q": ratio_q, "hist": hist}


def triangle_stats(off, adj, seed: int, k: int):
    """Samples [0, k) of the global stream (uniform over all wedges, Sec. 3.2),
    then summarise(): the paper's single-bin triangle-sampling run."""
    s = sample(off, adj, 1, 2, seed, 0, k, records=True)
    out = summarise(s["records"])
    out["records"] = s["records"]
    out["stats"] = s["stats"]
    return out
