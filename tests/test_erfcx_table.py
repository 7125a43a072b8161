"""The piecewise-polynomial erfcx table used by the kernels for the half-line Maxwellian moments
(erfc(t) = exp(-t^2) erfcx(t)) agrees with scipy's erfcx to a few ulp on [0, 28)."""
import os
import re

import numpy as np
from scipy import special

from conftest import ROOT


def _table():
    src = open(os.path.join(ROOT, "paper_2001_01570_gb300", "csrc", "cgks_erfcx_table.h")).read()
    body = src[src.index("= {") + 3: src.rindex("};")]
    rows = re.findall(r"\{([^{}]*)\}", body)
    return np.array([[float(x) for x in r.split(",")] for r in rows])


def _eval(tab, t):
    k = np.minimum((np.minimum(t, 27.9) * 4.0).astype(int), tab.shape[0] - 1)
    z = t - (0.25 * k + 0.125)
    r = tab[k, 0].copy()
    for m in range(1, tab.shape[1]):
        r = r * z + tab[k, m]
    return r


def test_erfcx_table_accuracy():
    tab = _table()
    assert tab.shape == (112, 12)
    rng = np.random.default_rng(0)
    t = np.concatenate([rng.uniform(0, 28, 20000), rng.uniform(0, 1, 5000), np.arange(0, 28, 0.25)])
    rel = np.abs(_eval(tab, t) / special.erfcx(t) - 1.0)
    assert rel.max() < 1e-15, rel.max()
    # erfc itself through the scaled form, against scipy, where it does not underflow
    t2 = rng.uniform(0, 26, 5000)
    erfc = np.exp(-t2 * t2) * _eval(tab, t2)
    ok = special.erfc(t2) > 1e-300
    assert np.max(np.abs(erfc[ok] / special.erfc(t2[ok]) - 1.0)) < 1e-13
