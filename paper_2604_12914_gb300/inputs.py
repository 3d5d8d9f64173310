"""Seeded synthetic inputs for the LR-CCSD response path.

This module only draws random numbers and shapes them (Hermitian symmetrisation,
antisymmetrisation of amplitude-like arrays, the exponential decay of the Cholesky
vectors).  It contains none of the method's arithmetic: no integrals, no amplitudes
derived from integrals, no residuals.  Both the CUDA path (through the C ABI) and
the CPU oracle consume what it returns.

Recipe (the paper's systems are real molecules; these stand in for them):

* orbital (spinor) energies: occupied ~ U[-2, -0.3], virtual ~ U[0.1, 5] Hartree;
* Cholesky vectors L^P (P = 0..naux-1): L^P = (G + G^H)/sqrt(2) * exp(-P/decay) * scale,
  with Re G, Im G i.i.d. N(0, 1/2), so every L^P is Hermitian, off-diagonal
  E|L_pq|^2 = scale^2 * exp(-2P/decay), diagonal real N(0, scale^2 exp(-2P/decay));
* dipole integrals mu^x, mu^y, mu^z: the same Hermitian recipe without decay;
* optional T1 = t1_scale * CN(0, 1).

Generation order (one numpy PCG64 stream per seed): eps_occ, eps_vir, L, mu_x, mu_y,
mu_z, T1.  Sizes follow the paper's active spaces: o occupied and v virtual spinors
after frozen core and natural-spinor truncation (Sec. 4.6), naux Cholesky vectors
(Sec. 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Named workloads: o, v, naux and the frequencies (a.u.) each is solved at.
CONFIGS = {
    "C1": dict(o=10, v=40, naux=200, omegas=(0.0,)),
    "C2": dict(o=32, v=240, naux=1200, omegas=(0.0, 0.0428)),
    "C3": dict(o=40, v=320, naux=1600, omegas=(0.0, 0.02, 0.0428, 0.0656)),
    "C4": dict(o=24, v=160, naux=800, omegas=(0.0,)),
    "C5": dict(o=56, v=480, naux=3000, omegas=(0.0, 0.0428)),
}


@dataclass
class System:
    o: int
    v: int
    naux: int
    eps: np.ndarray          # [n] float64, occupied first
    L: np.ndarray            # [naux, n, n] complex128, each L[P] Hermitian
    mu: np.ndarray           # [3, n, n] complex128, Hermitian
    t1: np.ndarray           # [o, v] complex128
    seed: int = 0
    scale: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.o + self.v


def _hermitian(rng: np.random.Generator, shape) -> np.ndarray:
    """(G + G^H)/sqrt(2) over the last two axes, Re G, Im G ~ N(0, 1/2)."""
    g = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * math.sqrt(0.5)
    return (g + np.conj(np.swapaxes(g, -1, -2))) / math.sqrt(2.0)


def make_system(o: int, v: int, naux: int, seed: int = 1, scale: float = 1.0,
                t1_scale: float = 0.0, decay: float = 60.0) -> System:
    """Draw one synthetic system; see the module docstring for the recipe."""
    rng = np.random.default_rng(seed)
    eps_occ = rng.uniform(-2.0, -0.3, o)
    eps_vir = rng.uniform(0.1, 5.0, v)
    n = o + v
    L = np.empty((naux, n, n), dtype=np.complex128)
    chunk = max(1, int(2e7 // max(1, n * n)))
    for p0 in range(0, naux, chunk):
        p1 = min(naux, p0 + chunk)
        blk = _hermitian(rng, (p1 - p0, n, n))
        blk *= (np.exp(-np.arange(p0, p1) / decay) * scale)[:, None, None]
        L[p0:p1] = blk
    mu = _hermitian(rng, (3, n, n))
    t1 = np.zeros((o, v), dtype=np.complex128)
    if t1_scale != 0.0:
        t1 = t1_scale * (rng.standard_normal((o, v)) + 1j * rng.standard_normal((o, v))) * math.sqrt(0.5)
    eps = np.concatenate([eps_occ, eps_vir])
    return System(o, v, naux, eps, L, mu, t1, seed=seed, scale=scale,
                  meta=dict(decay=decay, t1_scale=t1_scale))


def make_config(name: str, seed: int | None = None, scale: float = 1.0,
                t1_scale: float = 0.0) -> System:
    c = CONFIGS[name]
    if seed is None:
        seed = int(name[1:])
    s = make_system(c["o"], c["v"], c["naux"], seed=seed, scale=scale, t1_scale=t1_scale)
    s.meta["config"] = name
    s.meta["omegas"] = c["omegas"]
    return s


def antisym_pairs(x: np.ndarray) -> np.ndarray:
    """Project a [o,o,v,v] array onto the part antisymmetric in (0,1) and in (2,3)."""
    y = x - np.swapaxes(x, 0, 1)
    return 0.5 * 0.5 * (y - np.swapaxes(y, 2, 3))


def random_amplitudes(o: int, v: int, seed: int, s1: float = 1.0, s2: float = 1.0,
                      nvec: int | None = None):
    """Random singles [.., o, v] and antisymmetric doubles [.., o, o, v, v] (complex128)."""
    rng = np.random.default_rng(seed)
    lead = () if nvec is None else (nvec,)
    x1 = s1 * (rng.standard_normal(lead + (o, v)) + 1j * rng.standard_normal(lead + (o, v))) * math.sqrt(0.5)
    z = (rng.standard_normal(lead + (o, o, v, v)) + 1j * rng.standard_normal(lead + (o, o, v, v))) * math.sqrt(0.5)
    if nvec is None:
        x2 = s2 * 2.0 * antisym_pairs(z)
    else:
        x2 = s2 * 2.0 * np.stack([antisym_pairs(zz) for zz in z])
    return x1, x2


def subspace_mask(o: int, v: int, occ_idx, vir_idx):
    """Boolean masks selecting amplitude entries whose indices all lie in a subspace."""
    mo = np.zeros(o, bool)
    mo[list(occ_idx)] = True
    mv = np.zeros(v, bool)
    mv[list(vir_idx)] = True
    m1 = mo[:, None] & mv[None, :]
    m2 = mo[:, None, None, None] & mo[None, :, None, None] & mv[None, None, :, None] & mv[None, None, None, :]
    return m1, m2
