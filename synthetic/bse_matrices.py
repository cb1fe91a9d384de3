"""Seeded synthetic BSE matrices with the shapes of the paper's test workloads.

The paper builds its matrices from a TD-DFT kernel of monolayer CrI3 (Sec. 3.1,
Eqs. 8-9): R = diag(transition energies) + v + f_xc and C = v + f_xc, stored
as single-precision complex.  Those matrices are not available, so this module
draws stand-ins of the same structure:

    A = diag(E) + K_x - W        (Hermitian, "R" of Eq. 1)
    B = s_B * rho^H diag(v) conj(rho)   (complex symmetric, "C" of Eq. 1, C = C^T)

with K_x = s_x * rho^H diag(v) rho and W = s_W * rhoW^H diag(v) rhoW, v_G =
1/(|G|^2 + 0.1) over the first N_G integer G-vectors, and the scales chosen so
that ||K_x||_2, ||W||_2 and ||B||_2 take prescribed values.  Because
lambda_min(A) >= E_min - ||W||_2 > ||B||_2, the matrix M of Eq. 2 is positive
definite and the spectrum of H is real (Sec. 1, after Eq. 3).

This module holds no arithmetic of the eigensolver.  Both the FP64 oracle and
the CUDA path consume the bytes it produces; random numbers are drawn with
numpy's PCG64 so the host and a device generator see the same draws.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "BSEProblemSpec",
    "CONFIGS",
    "g_vectors",
    "coulomb_weights",
    "complex_gaussian",
    "make_problem",
    "make_problem_torch",
    "batched_specs",
    "loss_draws",
    "random_start",
    "reduced_spec",
    "gradient_probe_entries",
]


@dataclasses.dataclass(frozen=True)
class BSEProblemSpec:
    """Recipe for one synthetic problem (sizes in transitions, energies in eV)."""

    n: int                      # resonant block order N
    n_g: int                    # number of G-vectors N_G
    seed: int | np.random.SeedSequence
    form: str = "ph"            # "tda" (A only) or "ph" (A and B)
    e_lo: float = 1.5           # transition energies ~ U[e_lo, e_hi], sorted
    e_hi: float = 10.0
    kx_norm: float = 0.3        # ||K_x||_2
    w_norm: float = 0.2         # ||W||_2
    b_norm: float = 0.15        # ||B||_2
    dtype: str = "c128"         # storage type: "c128" or "c64"
    nev: int = 20


# The five workloads (index = seed).  Config 2 is a batch drawn by batched_specs().
CONFIGS = {
    0: BSEProblemSpec(n=2000, n_g=300, seed=0, form="tda", dtype="c128", nev=20),
    1: BSEProblemSpec(n=10000, n_g=600, seed=1, form="ph", dtype="c128", nev=100),
    3: BSEProblemSpec(n=20000, n_g=1000, seed=3, form="ph", dtype="c64", nev=50),
    4: BSEProblemSpec(n=50000, n_g=2000, seed=4, form="ph", e_lo=1.0, e_hi=12.0,
                      dtype="c64", nev=200),
}
BATCH_COUNT = 64
BATCH_N_RANGE = (500, 6000)
BATCH_NG = 400
BATCH_NEV = 16


def g_vectors(n_g: int) -> np.ndarray:
    """First n_g integer triples ordered by (|n|^2, lexicographic); G = 0 first."""
    r = 1
    while (2 * r + 1) ** 3 < 4 * n_g + 64:
        r += 1
    # all triples with |n_i| <= r; the ball of radius r is complete, keep only it
    ax = np.arange(-r, r + 1)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    n2 = (g * g).sum(axis=1)
    g, n2 = g[n2 <= r * r], n2[n2 <= r * r]
    order = np.lexsort((g[:, 2], g[:, 1], g[:, 0], n2))
    g = g[order]
    if g.shape[0] < n_g:
        raise ValueError("g-vector ball too small")
    return g[:n_g]


def coulomb_weights(n_g: int) -> np.ndarray:
    """v_G = 1 / (|G|^2 + 0.1) in units where |G| = |n|."""
    g = g_vectors(n_g)
    return 1.0 / ((g * g).sum(axis=1).astype(np.float64) + 0.1)


def complex_gaussian(rng: np.random.Generator, shape) -> np.ndarray:
    """(N(0,1) + i N(0,1)) / sqrt(2), real part drawn first as one block."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) / math.sqrt(2.0)


def _rng(seed) -> np.random.Generator:
    if isinstance(seed, np.random.SeedSequence):
        return np.random.Generator(np.random.PCG64(seed))
    return np.random.default_rng(seed)


def _draws(spec: BSEProblemSpec):
    rng = _rng(spec.seed)
    energies = np.sort(rng.uniform(spec.e_lo, spec.e_hi, spec.n))
    rho = complex_gaussian(rng, (spec.n_g, spec.n))
    rho_w = complex_gaussian(rng, (spec.n_g, spec.n))
    return rng, energies, rho, rho_w


def _scales(rho, rho_w, v, spec):
    """Scale factors so that ||K_x||_2, ||W||_2, sigma_max(B) hit the spec (FP64)."""
    sq = np.sqrt(v)[:, None]
    f = sq * rho                         # D^{1/2} rho, N_G x N
    fw = sq * rho_w
    lam_x = np.linalg.eigvalsh(f @ f.conj().T)[-1]
    lam_w = np.linalg.eigvalsh(fw @ fw.conj().T)[-1]
    s_x = spec.kx_norm / lam_x
    s_w = spec.w_norm / lam_w
    s_b = 0.0
    if spec.form == "ph":
        # B = F^H conj(F): sigma_max from QR of F^H and conj(F)^H (N x N_G each)
        _, r1 = np.linalg.qr(f.conj().T)
        _, r2 = np.linalg.qr(f.T)
        s_b = spec.b_norm / np.linalg.svd(r1 @ r2.conj().T, compute_uv=False)[0]
    return s_x, s_w, s_b


def _store(x: np.ndarray, dtype: str) -> np.ndarray:
    return np.ascontiguousarray(x.astype(np.complex64 if dtype == "c64" else np.complex128))


def make_problem(spec: BSEProblemSpec):
    """Host generation.  Returns dict(A, B, energies) with A exactly Hermitian and
    B exactly complex symmetric in the storage dtype (row-major, full N x N)."""
    _, energies, rho, rho_w = _draws(spec)
    v = coulomb_weights(spec.n_g)
    s_x, s_w, s_b = _scales(rho, rho_w, v, spec)
    vr = v[:, None] * rho
    a = s_x * (rho.conj().T @ vr) - s_w * (rho_w.conj().T @ (v[:, None] * rho_w))
    a[np.diag_indices(spec.n)] += energies
    a = _store(a, spec.dtype)
    a = _hermitian(a)
    b = None
    if spec.form == "ph":
        b = s_b * (rho.conj().T @ (v[:, None] * rho.conj()))
        b = _symmetric(_store(b, spec.dtype))
    return {"A": a, "B": b, "energies": energies}


def _hermitian(a: np.ndarray) -> np.ndarray:
    """Exact Hermitian completion from the upper triangle (diagonal made real)."""
    n = a.shape[0]
    step = 2048
    for i0 in range(0, n, step):
        i1 = min(n, i0 + step)
        a[i0:i1, :i0] = a[:i0, i0:i1].conj().T
        d = a[i0:i1, i0:i1]
        low = np.tril(np.ones(d.shape, dtype=bool), -1)
        d[low] = d.conj().T[low]
    a[np.diag_indices(n)] = a.diagonal().real
    return a


def _symmetric(b: np.ndarray) -> np.ndarray:
    n = b.shape[0]
    step = 2048
    for i0 in range(0, n, step):
        i1 = min(n, i0 + step)
        b[i0:i1, :i0] = b[:i0, i0:i1].T
        d = b[i0:i1, i0:i1]
        low = np.tril(np.ones(d.shape, dtype=bool), -1)
        d[low] = d.T[low]
    return b


def make_problem_torch(spec: BSEProblemSpec, device="cuda"):
    """Device generation for the large workloads: the same numpy draws, the
    N_G-contractions done with torch on `device` in the storage precision.
    A and B are made exactly Hermitian / symmetric from their upper triangles."""
    import torch

    _, energies, rho, rho_w = _draws(spec)
    v = coulomb_weights(spec.n_g)
    cdt = torch.complex64 if spec.dtype == "c64" else torch.complex128
    vt = torch.from_numpy(v).to(device)
    out = {"energies": energies}
    # scale factors on the host, with the same code as make_problem (the
    # device only runs plain matrix products)
    s_x, s_w, s_b = _scales(rho, rho_w, v, spec)
    rc = torch.from_numpy(rho).to(device=device, dtype=cdt)
    rwc = torch.from_numpy(rho_w).to(device=device, dtype=cdt)
    vc = vt.to(cdt)
    a = (s_x * rc.conj().T) @ (vc[:, None] * rc)
    a -= (s_w * rwc.conj().T) @ (vc[:, None] * rwc)
    del rwc
    a.diagonal().add_(torch.from_numpy(energies).to(device=device, dtype=cdt))
    out["A"] = _hermitian_torch(a)
    if spec.form == "ph":
        b = (s_b * rc.conj().T) @ (vc[:, None] * rc.conj())
        out["B"] = _symmetric_torch(b)
    else:
        out["B"] = None
    return out


def _hermitian_torch(a):
    import torch

    n = a.shape[0]
    step = 4096
    for i0 in range(0, n, step):           # lower := conj(upper), block rows
        i1 = min(n, i0 + step)
        blk = a[i0:i1, :]
        up = a[:, i0:i1].conj().T          # rows i0:i1 of conj(A^T)
        low = torch.arange(n, device=a.device)[None, :] < torch.arange(i0, i1, device=a.device)[:, None]
        blk.copy_(torch.where(low, up, blk))
    a.diagonal().copy_(a.diagonal().real.to(a.dtype))
    return a


def _symmetric_torch(b):
    import torch

    n = b.shape[0]
    step = 4096
    for i0 in range(0, n, step):
        i1 = min(n, i0 + step)
        blk = b[i0:i1, :]
        up = b[:, i0:i1].T
        low = torch.arange(n, device=b.device)[None, :] < torch.arange(i0, i1, device=b.device)[:, None]
        blk.copy_(torch.where(low, up, blk))
    return b


def batched_specs(seed: int = 2, count: int = BATCH_COUNT):
    """The uneven batch: N_i ~ U{500..6000} drawn first, then one spawned
    stream per problem (N_G = 400, complex64, 16 eigenpairs each)."""
    ss = np.random.SeedSequence(seed)
    rng = np.random.Generator(np.random.PCG64(ss))
    sizes = rng.integers(BATCH_N_RANGE[0], BATCH_N_RANGE[1] + 1, size=count)
    children = ss.spawn(count)
    return [BSEProblemSpec(n=int(n), n_g=BATCH_NG, seed=c, form="ph", dtype="c64",
                           nev=BATCH_NEV) for n, c in zip(sizes, children)]


def loss_draws(nev: int, seed: int = 3):
    """Weights w_i ~ U[0,1] and target noise ~ N(0, 0.01 eV) for the
    differentiable workload, from a stream separate from the matrices."""
    rng = np.random.default_rng([seed, 1])
    w = rng.uniform(0.0, 1.0, nev)
    noise = rng.normal(0.0, 0.01, nev)
    return w, noise


def reduced_spec(index: int, n: int) -> BSEProblemSpec:
    """The recipe of workload `index` (seed, N_G, energy window, kernel norms,
    storage type, nev) at a smaller order n, for the dense oracle to reach."""
    return dataclasses.replace(CONFIGS[index], n=int(n))


# the seven perturbation directions of a Hermitian A / symmetric B entry
PROBE_KINDS = ("A_re", "A_im", "A_diag", "B_re", "B_im", "B_diag_re", "B_diag_im")


def gradient_probe_entries(n: int, focus: int, counts=(10, 10, 8, 10, 10, 8, 8), seed: int = 31):
    """Seeded entries (kind, i, j) at which a gradient is probed: off-diagonal
    entries (i < j) for the *_re / *_im kinds, diagonal ones (i == j) for the
    *_diag kinds; `counts` per kind in the order of PROBE_KINDS (64 in all).
    Three in four indices are drawn from [0, focus) -- with the transition
    energies sorted ascending, the lowest eigenvectors live mostly there, so
    those entries carry gradients well above rounding -- the rest from [0, n)."""
    rng = np.random.default_rng([seed, n])
    out = []
    for kind, c in zip(PROBE_KINDS, counts):
        for t in range(c):
            hi = n if t % 4 == 3 else min(n, focus)
            if "diag" in kind:
                i = int(rng.integers(0, hi))
                out.append((kind, i, i))
            else:
                i, j = sorted(int(v) for v in rng.choice(hi, 2, replace=False))
                out.append((kind, i, j))
    return out


def random_start(n: int, seed: int = 12345) -> np.ndarray:
    """Complex Gaussian start vector for a Krylov iteration (passed as input)."""
    return complex_gaussian(np.random.default_rng(seed), (n,))
