"""Seeded synthetic binary-glass spring networks: the shared input generator.

This package produces inputs only (positions, types, masses, bonds with spring constants and
unit vectors). It contains none of the eigensolver's arithmetic; the CPU oracle and the GPU
library each assemble the mass-weighted Hessian H_ij = Delta_ij / sqrt(m_i m_j) (Sec. 1,
eqs. (1)-(2) of arXiv 1902.07041) from these arrays with their own code.

The C source ``glassgen.c`` is compiled on first use with the system C compiler into
``_glassgen.so`` next to it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glassgen.c")
_LIB = os.path.join(_HERE, "_glassgen.so")
_lib = None

# Binary-glass recipe shared by every workload (masses in amu, lengths in Angstrom,
# spring constants in eV/A^2).
DENSITY = 0.06
D_MIN = 2.2
R_CUT = 3.5
FRAC_A = 0.64
MASS_A = 63.546
MASS_B = 91.224
K_MEDIAN = 1.0
K_SIGMA = 0.3


def build(force: bool = False) -> str:
    """Compile glassgen.c into a shared object (idempotent unless ``force``)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.gg_generate.restype = ctypes.c_int
        lib.gg_generate.argtypes = [
            ctypes.c_int32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p,
        ]
        lib.gg_subseed.restype = ctypes.c_uint64
        lib.gg_subseed.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        _lib = lib
    return _lib


@dataclass
class Glass:
    """One synthetic glass: N atoms, their masses and the bond network."""

    n_atoms: int
    seed: int
    box: float
    pos: np.ndarray  # (N, 3) float64
    mass: np.ndarray  # (N,) float64
    types: np.ndarray  # (N,) int32, 0 = A, 1 = B
    bi: np.ndarray  # (nb,) int32, bi < bj
    bj: np.ndarray  # (nb,) int32
    k: np.ndarray  # (nb,) float64 spring constants
    rhat: np.ndarray  # (nb, 3) float64 unit vectors from atom bi to atom bj (minimum image)

    @property
    def n_bonds(self) -> int:
        return int(self.bi.shape[0])

    @property
    def n(self) -> int:
        """Matrix order 3N."""
        return 3 * self.n_atoms


_ERRORS = {-1: "bad arguments", -3: "random sequential addition gave up (packing too dense)",
           -4: "out of memory"}


def generate(n_atoms: int, seed: int, *, density: float = DENSITY, d_min: float = D_MIN,
             r_cut: float = R_CUT, frac_a: float = FRAC_A, mass_a: float = MASS_A,
             mass_b: float = MASS_B, k_median: float = K_MEDIAN, k_sigma: float = K_SIGMA,
             spatial_sort: bool = True) -> Glass:
    """Generate a seeded glass. Same arguments give bit-identical arrays on every machine."""
    lib = _load()
    n_atoms = int(n_atoms)
    pos = np.zeros((n_atoms, 3), np.float64)
    mass = np.zeros(n_atoms, np.float64)
    types = np.zeros(n_atoms, np.int32)
    box = ctypes.c_double(0.0)
    nb = ctypes.c_int64(0)
    cap = max(64, 12 * n_atoms)
    for _ in range(3):
        bi = np.zeros(cap, np.int32)
        bj = np.zeros(cap, np.int32)
        kk = np.zeros(cap, np.float64)
        rh = np.zeros((cap, 3), np.float64)
        rc = lib.gg_generate(n_atoms, ctypes.c_uint64(seed), density, d_min, r_cut, frac_a, mass_a,
                             mass_b, k_median, k_sigma, int(bool(spatial_sort)),
                             pos.ctypes.data, mass.ctypes.data, types.ctypes.data,
                             ctypes.byref(box), cap, ctypes.byref(nb), bi.ctypes.data,
                             bj.ctypes.data, kk.ctypes.data, rh.ctypes.data)
        if rc == -2:
            cap = int(nb.value) + 16
            continue
        if rc != 0:
            raise RuntimeError(f"glassgen: {_ERRORS.get(rc, rc)}")
        m = int(nb.value)
        return Glass(n_atoms, seed, box.value, pos, mass, types, bi[:m].copy(), bj[:m].copy(),
                     kk[:m].copy(), rh[:m].copy())
    raise RuntimeError("glassgen: bond buffer sizing failed")


def subseed(seed: int, index: int) -> int:
    """Per-sample sub-seed for batches: SplitMix64(seed XOR index)."""
    return int(_load().gg_subseed(ctypes.c_uint64(seed), ctypes.c_uint64(index)))


def batch_sizes(n_samples: int, seed: int, lo: int = 5000, hi: int = 40000) -> list[int]:
    """Atom counts of a batch of independent samples, uniform integers in [lo, hi]."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    return [int(x) for x in rng.integers(lo, hi + 1, size=n_samples)]
