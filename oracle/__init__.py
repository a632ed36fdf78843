"""FP64 CPU oracle for statistical multi-resolution projection (arXiv 1503.03492).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  The
product library (``paper_1503_03492_gb300``) never imports it, and the two
share no code: this package wraps the plain C file ``smre_oracle.c`` with
ctypes and adds the Python-side helpers the tests need (default set order of
Sec. 2.3 reading R4, weights of Sec. 2.1, KKT residuals).

The C library is compiled on first use (``build()``), with ``gcc -O2`` and
OpenMP when the compiler has it; nothing here depends on a GPU.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smre_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``smre_oracle.c`` into ``oracle/lib/liboracle.so`` (plain C, FP64)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:] + ["-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.oracle_normal_quantile.restype = ctypes.c_double
            lib.oracle_normal_quantile.argtypes = [ctypes.c_double]
            lib.oracle_chi2_quantile.restype = ctypes.c_double
            lib.oracle_chi2_quantile.argtypes = [ctypes.c_double, ctypes.c_int]
            lib.oracle_bound_from_quantile.restype = ctypes.c_double
            lib.oracle_bound_from_quantile.argtypes = [ctypes.c_double, ctypes.c_int]
            lib.oracle_normal_sample.restype = ctypes.c_double
            lib.oracle_normal_sample.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.oracle_maxstat_quantile.restype = ctypes.c_double
            lib.oracle_maxstat_quantile.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ip,
                                                    ctypes.c_double, ctypes.c_int, ctypes.c_uint64]
            lib.oracle_dykstra.restype = ctypes.c_int
            lib.oracle_dykstra.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ip, ip, ip,
                                           dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int, dp, dp, dp]
            lib.oracle_icd.restype = ctypes.c_int
            lib.oracle_icd.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp,
                                       ctypes.c_double, ctypes.c_int, dp, ip]
            lib.oracle_max_violation.restype = ctypes.c_double
            lib.oracle_max_violation.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ip, dp]
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.oracle_max_threads.argtypes = []
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# ---------------------------------------------------------------- weights (Sec. 2.1)

def normal_quantile(alpha: float) -> float:
    """alpha-quantile of N(0, 1) (bisection on the CDF)."""
    return _load().oracle_normal_quantile(float(alpha))


def chi2_quantile(alpha: float, k: int) -> float:
    """alpha-quantile of chi^2 with k degrees of freedom (finite-sum CDF + bisection)."""
    return _load().oracle_chi2_quantile(float(alpha), int(k))


def bound_from_quantile(q: float, L: int) -> float:
    """cS = 1 / c_s(alpha) = (q sigma_s + mu_s)^4 for an L x L window (Sec. 2.1)."""
    return _load().oracle_bound_from_quantile(float(q), int(L))


def normal_sample(seed: int, j: int) -> float:
    """The j-th N(0,1) number of the SplitMix64 + Box-Muller stream ``seed``."""
    return _load().oracle_normal_sample(int(seed) & (2**64 - 1), int(j))


def maxstat_quantile(H, W, sides, alpha, draws, seed) -> float:
    """Monte Carlo alpha-quantile of Q_Omega (Sec. 2.1) on H x W N(0,1) images."""
    s = np.ascontiguousarray(sides, dtype=np.int32)
    return _load().oracle_maxstat_quantile(int(H), int(W), len(s), _ip(s), float(alpha),
                                           int(draws), int(seed) & (2**64 - 1))


PERSET, CHI2, MAXSTAT = "perset", "chi2", "maxstat"


def bounds(sides, alpha: float, mode: str = PERSET, H: int = 0, W: int = 0,
           draws: int = 1000, seed: int = 0) -> np.ndarray:
    """Bound cS (= r_s^2 = 1/c_s(alpha)) per side, FP64.

    ``perset``: q = Phi^{-1}(alpha) in c_s(alpha) = 1/(q sigma_s + mu_s)^4
    (the paper's fourth-root normal approximation of the per-window chi^2
    alpha-quantile).  ``chi2``: the exact chi^2_{L^2} alpha-quantile.
    ``maxstat``: q = Monte Carlo alpha-quantile of Q_Omega on H x W noise.
    """
    sides = [int(L) for L in sides]
    if mode == PERSET:
        q = normal_quantile(alpha)
        return np.array([bound_from_quantile(q, L) for L in sides])
    if mode == CHI2:
        return np.array([chi2_quantile(alpha, L * L) for L in sides])
    if mode == MAXSTAT:
        q = maxstat_quantile(H, W, sides, alpha, draws, seed)
        return np.array([bound_from_quantile(q, L) for L in sides])
    raise ValueError(mode)


# ------------------------------------------------------- set order (reading R4)

def default_tilings(sides):
    """Tilings (L, a, b) of one cycle: sides descending, a outer, b inner."""
    out = []
    for L in sorted(set(int(s) for s in sides), reverse=True):
        for a in range(L):
            for b in range(L):
                out.append((L, a, b))
    return out


def n_windows(H, W, sides) -> int:
    """Number of sets of one cycle: sum_L (H - L + 1)(W - L + 1)."""
    return sum((H - L + 1) * (W - L + 1) for L in set(int(s) for s in sides))


# ------------------------------------------------------ Algorithm 2 (Sec. 2.3)

class DykstraResult:
    def __init__(self, x, cycles, hist, q, tilings):
        self.x = x
        self.cycles = cycles
        self.hist = hist            # (cycles, 2): L2 change d, |x_prev|
        self.q = q                  # (n_tilings, H, W) paper sign convention, or None
        self.tilings = tilings


def dykstra(x0, sides, cS, max_cycles=200, tol=-1.0, tol_relative=False, tilings=None,
            n_threads=1, want_q=False) -> DykstraResult:
    """Dykstra's cyclic projection of ``x0`` onto the intersection of the balls
    sum_{i in s} x_i^2 <= cS[L] of every L x L window (Algorithm 2).

    ``cS`` maps each side to its bound (dict, or a sequence aligned with ``sides``).
    ``tilings`` is the order of one cycle (default: reading R4).
    ``tol < 0`` runs exactly ``max_cycles`` cycles.
    """
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    H, W = x0.shape
    if not isinstance(cS, dict):
        cS = {int(L): float(c) for L, c in zip(sides, cS)}
    til = list(tilings) if tilings is not None else default_tilings(sides)
    Ls = np.array([t[0] for t in til], dtype=np.int32)
    As = np.array([t[1] for t in til], dtype=np.int32)
    Bs = np.array([t[2] for t in til], dtype=np.int32)
    ck = np.array([cS[int(t[0])] for t in til], dtype=np.float64)
    x = np.empty_like(x0)
    hist = np.zeros((max(max_cycles, 1), 2))
    q = np.empty((len(til), H, W)) if want_q else None
    n = _load().oracle_dykstra(H, W, _dp(x0), len(til), _ip(Ls), _ip(As), _ip(Bs), _dp(ck),
                               int(max_cycles), float(tol), int(bool(tol_relative)),
                               int(n_threads), _dp(x), _dp(hist),
                               _dp(q) if q is not None else None)
    if n < 0:
        raise MemoryError("oracle_dykstra: out of memory")
    return DykstraResult(x, n, hist[:n].copy(), q, til)


# ------------------------------------------------------------- ICD (Sec. 3.2)

def icd_K(sides) -> int:
    """K = floor(log2 max side) (Eq. k-smre with the largest window side)."""
    return int(np.floor(np.log2(max(sides))))


def icd_tile_grid(H, W, K):
    """(off, n_tiles_i, n_tiles_j) of each pass i = 0..K (reading R7)."""
    B = 1 << K
    out = []
    for i in range(K + 1):
        off = (1 << i) % B
        out.append((off, (H - off) // B if H - off >= B else 0,
                    (W - off) // B if W - off >= B else 0))
    return out


class ICDResult:
    def __init__(self, x, sweeps, grid):
        self.x = x
        self.sweeps = sweeps        # list per pass of (n_ti, n_tj) int arrays
        self.grid = grid


def icd(x0, K, cS_level, tol=1e-3, max_sweeps=1000) -> ICDResult:
    """Incomplete Dykstra P_incomplete = prod_i P_{Omega^i} (Sec. 3.2).

    ``cS_level[k]`` is the bound of side 2^k, k = 0..K.
    """
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    H, W = x0.shape
    c = np.ascontiguousarray(cS_level, dtype=np.float64)
    assert len(c) == K + 1
    grid = icd_tile_grid(H, W, K)
    total = sum(g[1] * g[2] for g in grid)
    sw = np.zeros(max(total, 1), dtype=np.int32)
    x = np.empty_like(x0)
    n = _load().oracle_icd(H, W, _dp(x0), int(K), _dp(c), float(tol), int(max_sweeps),
                           _dp(x), _ip(sw))
    if n < 0:
        raise ValueError("oracle_icd: bad arguments or out of memory")
    per_pass, o = [], 0
    for (_, ni, nj) in grid:
        per_pass.append(sw[o:o + ni * nj].reshape(ni, nj).copy())
        o += ni * nj
    return ICDResult(x, per_pass, grid)


# ------------------------------------------------------------------- checkers

def icd_reach_mask(H, W, K, differ):
    """Pixels that tiles with a different sweep count can influence (Sec. 3.2).

    ``differ`` holds one boolean (n_ti, n_tj) array per pass i = 0..K (True:
    the two runs took a different number of sweeps on that tile).  Such a
    tile's pixels may differ; a tile of a later pass that overlaps a pixel
    that may differ starts from different values, so all of its pixels may
    differ as well.  Returns the H x W boolean mask of those pixels; outside
    it both runs computed the same arithmetic on the same inputs.
    """
    B = 1 << K
    mask = np.zeros((H, W), bool)
    for i, (off, ni, nj) in enumerate(icd_tile_grid(H, W, K)):
        d = np.asarray(differ[i]).reshape(ni, nj)
        for ti in range(ni):
            for tj in range(nj):
                sl = (slice(off + B * ti, off + B * (ti + 1)), slice(off + B * tj, off + B * (tj + 1)))
                if d[ti, tj] or mask[sl].any():
                    mask[sl] = True
    return mask



def max_violation(x, sides, cS) -> float:
    """max over all windows of (sum x^2 - cS) / cS (Eq. geq); <= 0 means feasible."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    H, W = x.shape
    s = np.ascontiguousarray(sides, dtype=np.int32)
    if isinstance(cS, dict):
        c = np.array([cS[int(L)] for L in s], dtype=np.float64)
    else:
        c = np.ascontiguousarray(cS, dtype=np.float64)
    return _load().oracle_max_violation(H, W, _dp(x), len(s), _ip(s), _dp(c))


def max_threads() -> int:
    return _load().oracle_max_threads()
