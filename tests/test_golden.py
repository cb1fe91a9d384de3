"""The stored expected values under tests/golden/ still follow from the current
generator and oracle (CPU): config 0 in full, and the two smallest problems of
the config-2 batch.  Config 1 (N = 10000) takes about ten minutes of dense
work and is left to tests/golden/make_golden.py."""
import os

import numpy as np

import oracle as O
from synthetic import CONFIGS, batched_specs, make_problem

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_config0_golden_reproduces():
    spec = CONFIGS[0]
    lam, _ = O.tda_lowest(make_problem(spec)["A"], spec.nev)
    gold = np.loadtxt(os.path.join(GOLD, "config0_lambda.txt"))
    np.testing.assert_allclose(lam, gold, rtol=1e-13, atol=0)


def test_config2_golden_reproduces_for_the_smallest_problems():
    specs = batched_specs()
    gold = np.loadtxt(os.path.join(GOLD, "config2_omega.txt")).reshape(len(specs), -1)
    for i in np.argsort([s.n for s in specs])[:2]:
        p = make_problem(specs[i])
        om = O.ph_lowest_shao(p["A"], p["B"], specs[i].nev)
        np.testing.assert_allclose(om, gold[i], rtol=1e-12, atol=0)
