"""Write the stored expected values under tests/golden/ from the FP64 oracle.

Calls only oracle/ (and the seeded generator in synthetic/).  Run from the
repository root:  python tests/golden/make_golden.py [config ...]

  config0_lambda.txt   TDA, N = 2000, lowest 20 eigenvalues of A (zheevd)
  config1_omega.txt    PH, N = 10000, lowest 100 positive omega of H, by the
                       paper's dense reduction (Sec. 2.1.1, Eqs. 4-6), which
                       tests/test_oracle_pins.py pins against zgeev
  config2_omega.txt    the 64-problem uneven batch, 16 omega each (same method)
  config3r_omega.txt   the config-3 recipe (PH, N_G = 1000, complex64) at N = 4000:
                       lowest 50 omega (same method)
  config3r_grad.txt    dL/dA and dL/dB of that problem at 64 seeded entries for the
                       loss L = sum w_i omega_i + sum (omega_i - t_i)^2 with
                       t_i = omega_i + noise_i (synthetic.loss_draws), i.e.
                       dL/domega_i = w_i - 2 noise_i: Hellmann-Feynman with the
                       left eigenvectors of Eq. 7 (oracle.hf_gradient_ph) on the
                       eigenvectors of the dense reduction
  config4r_omega.txt   the config-4 recipe (PH, energies U[1, 12] eV, N_G = 2000,
                       complex64) at N = 4000: lowest 200 omega (same method)
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


REDUCED_N = 4000


def config3r():
    from synthetic import gradient_probe_entries, loss_draws, reduced_spec
    spec = reduced_spec(3, REDUCED_N)
    t = time.time()
    p = make_problem(spec)
    om, X, Y = O.ph_lowest_shao(p["A"], p["B"], spec.nev, vectors=True)
    t_eig = time.time() - t
    _write("config3r_omega.txt", f"""
pseudo-Hermitian, config-3 recipe at N={spec.n}, N_G={spec.n_g}, seed={spec.seed}, complex64 storage
lowest {spec.nev} positive omega (eV), oracle.ph_lowest_shao on the stored values promoted to FP64, {t_eig:.1f} s
""", om)
    w, noise = loss_draws(spec.nev)
    g = w - 2.0 * noise
    GA, GB = O.hf_gradient_ph(X, Y, g)
    rows = []
    for kind, i, j in gradient_probe_entries(spec.n, 2 * spec.nev):
        G = GA if kind.startswith("A") else GB
        rows.append((i, j, G[i, j].real, G[i, j].imag))
    path = os.path.join(HERE, "config3r_grad.txt")
    with open(path, "w") as f:
        f.write(f"# config-3 recipe at N={spec.n}: oracle gradient entries for dL/domega = w - 2 noise\n")
        f.write("# (synthetic.loss_draws(50)); entries from synthetic.gradient_probe_entries(N, 2 nev), in order;\n")
        f.write("# columns: i j Re(G_ij) Im(G_ij), G = G_A for the A_* kinds, G_B for the B_* kinds\n")
        f.write("# oracle.hf_gradient_ph on the Omega-normalised eigenvectors of oracle.ph_lowest_shao\n")
        for i, j, re, im in rows:
            f.write(f"{i} {j} {re:.17e} {im:.17e}\n")
    print("wrote", path)


def config4r():
    from synthetic import reduced_spec
    spec = reduced_spec(4, REDUCED_N)
    t = time.time()
    p = make_problem(spec)
    om = O.ph_lowest_shao(p["A"], p["B"], spec.nev)
    _write("config4r_omega.txt", f"""
pseudo-Hermitian, config-4 recipe at N={spec.n}, N_G={spec.n_g}, seed={spec.seed}, energies U[{spec.e_lo}, {spec.e_hi}] eV,
complex64 storage; lowest {spec.nev} positive omega (eV), oracle.ph_lowest_shao on the stored values
promoted to FP64, {time.time() - t:.1f} s
""", om)


if __name__ == "__main__":
    which = sys.argv[1:] or ["0", "1", "2", "3r", "4r"]
    for w in which:
        {"0": config0, "1": config1, "2": config2, "3r": config3r, "4r": config4r}[w]()
