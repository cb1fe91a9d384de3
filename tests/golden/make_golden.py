"""Write the stored expected values under tests/golden/ from the FP64 oracle.

Calls only oracle/ (and the seeded generator in synthetic/).  Run from the
repository root:  python tests/golden/make_golden.py [config ...]

  config0_lambda.txt   TDA, N = 2000, lowest 20 eigenvalues of A (zheevd)
  config1_omega.txt    PH, N = 10000, lowest 100 positive omega of H, by the
                       paper's dense reduction (Sec. 2.1.1, Eqs. 4-6), which
                       tests/test_oracle_pins.py pins against zgeev
  config2_omega.txt    the 64-problem uneven batch, 16 omega each (same method)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from synthetic import CONFIGS, batched_specs, make_problem  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _write(name, header, values):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        for line in header.strip().splitlines():
            f.write("# " + line + "\n")
        for v in np.atleast_1d(values).ravel():
            f.write(f"{v:.17e}\n")
    print("wrote", path)


def config0():
    spec = CONFIGS[0]
    t = time.time()
    p = make_problem(spec)
    lam, _ = O.tda_lowest(p["A"], spec.nev)
    _write("config0_lambda.txt", f"""
TDA, N={spec.n}, N_G={spec.n_g}, seed={spec.seed}, complex128 (synthetic generator)
lowest {spec.nev} eigenvalues of A (eV), oracle.tda_lowest (dense zheevd), {time.time() - t:.1f} s
""", lam)


def config1():
    spec = CONFIGS[1]
    t = time.time()
    p = make_problem(spec)
    om = O.ph_lowest_shao(p["A"], p["B"], spec.nev)
    _write("config1_omega.txt", f"""
pseudo-Hermitian, N={spec.n}, N_G={spec.n_g}, seed={spec.seed}, complex128 (synthetic generator)
lowest {spec.nev} positive omega of H = [[A, B], [-conj B, -conj A]] (eV),
oracle.ph_lowest_shao: Cholesky of M_r and Hermitian -iW (Sec. 2.1.1, Eqs. 4-6), {time.time() - t:.1f} s
""", om)


def config2():
    specs = batched_specs()
    t = time.time()
    rows = []
    for s in specs:
        p = make_problem(s)
        rows.append(O.ph_lowest_shao(p["A"], p["B"], s.nev))
    _write("config2_omega.txt", f"""
uneven batch of {len(specs)} pseudo-Hermitian problems, N_i = {[s.n for s in specs]}
N_G=400, complex64 storage, lowest {specs[0].nev} positive omega each (problem-major), eV
oracle.ph_lowest_shao on the stored complex64 values promoted to FP64, {time.time() - t:.1f} s
""", np.array(rows))


if __name__ == "__main__":
    which = sys.argv[1:] or ["0", "1", "2"]
    for w in which:
        {"0": config0, "1": config1, "2": config2}[w]()
