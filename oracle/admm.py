"""FP64 oracle of the ADMM outer loop (Sec. 2.2, Algorithm 1 with Eq. 3).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle``): only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s oracle legs may use it.

The estimator (Eq. 1 with the splitting of Eq. 3) is

    min_{x, eps, z}  G(eps) + R(z)   s.t.   I = A x + eps,   z = x,

with G the indicator of the multi-resolution set (Eq. geq; all L x L windows
of every side, sum of squares <= cS[L]), R the total variation of Sec. 2
(anisotropic: sum over pixels of |forward difference| along each axis) and A
the convolution with a normalised, truncated Gaussian point-spread function.
The augmented Lagrangian (Eq. 2 with the two constraints of Eq. 3) has
multipliers Y1 (for I = A x + eps) and Y2 (for z = x) and penalties rho1,
rho2.  One iteration, in the paper's order (x, then eps, then the
multipliers; z is the second primal block of Eq. 3):

  x   <- x - (1/gamma) * grad_x L   (the linearised x-step: a gradient step of
          length 1/gamma on the smooth part, gamma >= rho1 |A|^2 + rho2)
  eps <- P_G(I - A x + Y1/rho1)    (Sec. 2.2: the projection onto the
          multi-resolution set, by Dykstra's algorithm, Algorithm 2)
  z   <- prox_{R/rho2}(x + Y2/rho2) (dual projected gradient, fixed count)
  Y1  <- Y1 + rho1 (I - A x - eps),  Y2 <- Y2 + rho2 (x - z)

and the loop stops once both |x_r - x_{r-1}|_2 <= delta and
|I - (A x_r + eps_r)|_2 <= delta, or at the iteration cap.  Every choice the
paper leaves open (the x-step, R, the z-step solver, the multiplier step
length, the stopping rule, the start values) is taken as stated here.

Plain numpy, FP64; the eps-step calls the FP64 C oracle of Algorithm 2.
"""
from __future__ import annotations

import math

import numpy as np

from . import dykstra as _dykstra
from . import icd as _icd
from . import icd_K as _icd_K


# ------------------------------------------------------------------ operator A

def gaussian_kernel(sigma: float, radius: int = 0) -> np.ndarray:
    """1-D weights w_k, k = -r..r, of exp(-k^2 / (2 sigma^2)), summing to 1.

    ``radius <= 0`` takes r = ceil(3 sigma).  The 2-D point-spread function is
    the outer product w_u w_v (separable Gaussian).
    """
    r = int(radius) if radius > 0 else int(math.ceil(3.0 * sigma))
    k = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-k * k / (2.0 * sigma * sigma))
    return w / w.sum()


def blur(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """(A x)_{i,j} = sum_{u,v} w_u w_v x_{i+u, j+v}, x = 0 outside the image.

    The kernel is symmetric, so A is its own adjoint.
    """
    x = np.asarray(x, dtype=np.float64)
    H, W = x.shape
    r = (len(w) - 1) // 2
    pad = np.zeros((H + 2 * r, W + 2 * r))
    pad[r:r + H, r:r + W] = x
    rows = np.zeros((H + 2 * r, W))
    for t in range(2 * r + 1):          # along each row: columns j + (t - r)
        rows += w[t] * pad[:, t:t + W]
    out = np.zeros((H, W))
    for t in range(2 * r + 1):          # then along each column
        out += w[t] * rows[t:t + H, :]
    return out


# ------------------------------------------------------------------------- TV

def grad(z: np.ndarray):
    """Forward differences D z = (d1, d2): d1[i,j] = z[i+1,j] - z[i,j] (0 on the
    last row), d2[i,j] = z[i,j+1] - z[i,j] (0 on the last column)."""
    d1 = np.zeros_like(z)
    d2 = np.zeros_like(z)
    d1[:-1, :] = z[1:, :] - z[:-1, :]
    d2[:, :-1] = z[:, 1:] - z[:, :-1]
    return d1, d2


def grad_adj(p1: np.ndarray, p2: np.ndarray) -> np.ndarray:
    """D^T p (minus the divergence): the adjoint of ``grad``."""
    out = np.zeros_like(p1)
    out[:-1, :] -= p1[:-1, :]
    out[1:, :] += p1[:-1, :]
    out[:, :-1] -= p2[:, :-1]
    out[:, 1:] += p2[:, :-1]
    return out


def tv(z: np.ndarray) -> float:
    """R(z) = sum_i sum_k |(grad z)_{i,k}| (Sec. 2, d = 2, anisotropic)."""
    d1, d2 = grad(np.asarray(z, dtype=np.float64))
    return float(np.abs(d1).sum() + np.abs(d2).sum())


def tv_prox(f, rho, iters, p1=None, p2=None, tau=None):
    """argmin_z R(z) + rho/2 |z - f|^2 by projected gradient on the dual.

    R(z) = max_{|p|_inf <= 1} <p, D z>, so for a dual point p the primal point
    is z = f - D^T p / rho, and the dual ascends along D z:
        p <- clip(p + tau D(f - D^T p / rho), -1, 1),   tau = rho / 8
    (|D|^2 <= 8 for the 2-D forward differences).  Starts from the given p
    (zero if None); returns (z, p1, p2) after ``iters`` steps.
    """
    f = np.asarray(f, dtype=np.float64)
    p1 = np.zeros_like(f) if p1 is None else np.array(p1, dtype=np.float64)
    p2 = np.zeros_like(f) if p2 is None else np.array(p2, dtype=np.float64)
    if tau is None:
        tau = rho / 8.0
    for _ in range(int(iters)):
        t = f - grad_adj(p1, p2) / rho
        g1, g2 = grad(t)
        p1 = np.clip(p1 + tau * g1, -1.0, 1.0)
        p2 = np.clip(p2 + tau * g2, -1.0, 1.0)
    z = f - grad_adj(p1, p2) / rho
    return z, p1, p2


# ----------------------------------------------------------------------- ADMM

class AdmmResult:
    def __init__(self, x, z, eps, Y1, Y2, p1, p2, iters, hist, dykstra_cycles):
        self.x, self.z, self.eps = x, z, eps
        self.Y1, self.Y2 = Y1, Y2
        self.p1, self.p2 = p1, p2
        self.iters = iters
        self.hist = hist                    # (iters, 2): |x_r - x_{r-1}|, |I - A x_r - eps_r|
        self.dykstra_cycles = dykstra_cycles


def admm(I, sides, cS, sigma, radius=0, rho1=1.0, rho2=1.0, gamma=0.0, tv_iters=20,
         max_iters=100, delta=-1.0, dyk_cycles=200, dyk_tol=-1.0, dyk_relative=False,
         n_threads=1, eps_incomplete=False, icd_K=-1, icd_tol=1e-3, icd_max_sweeps=1000) -> AdmmResult:
    """Algorithm 1 on Eq. 3 as read in the module docstring.

    ``gamma <= 0`` takes 1.01 (rho1 + rho2) (|A| <= 1 for a normalised
    non-negative kernel).  ``delta < 0`` runs exactly ``max_iters``
    iterations.  The eps-step runs Dykstra from q = 0 with ``dyk_cycles`` /
    ``dyk_tol`` / ``dyk_relative`` (``dyk_tol < 0``: exactly dyk_cycles).
    Start: x = z = eps = Y1 = Y2 = 0, TV dual p = 0 (carried across
    iterations).  ``eps_incomplete`` replaces the eps-step by the incomplete
    Dykstra of Sec. 3.2 (K = ``icd_K``, floor(log2 max side) if < 0; bound of
    side 2^k from ``cS``), the approximation the paper times the estimator with.
    """
    I = np.asarray(I, dtype=np.float64)
    H, W = I.shape
    w = gaussian_kernel(sigma, radius)
    cmap = cS if isinstance(cS, dict) else {int(L): float(c) for L, c in zip(sides, cS)}
    if eps_incomplete:
        K = icd_K if icd_K >= 0 else _icd_K(sides)
        c_level = [cmap[1 << k] for k in range(K + 1)]
    if gamma <= 0:
        gamma = 1.01 * (rho1 + rho2)
    x = np.zeros((H, W))
    z = np.zeros((H, W))
    eps = np.zeros((H, W))
    Y1 = np.zeros((H, W))
    Y2 = np.zeros((H, W))
    p1 = np.zeros((H, W))
    p2 = np.zeros((H, W))
    hist = []
    cycles = []
    it = 0
    while it < max_iters:
        # x-step: gradient of the smooth part of the augmented Lagrangian in x
        g = -blur(rho1 * (I - blur(x, w) - eps) + Y1, w) + rho2 * (x - z) + Y2
        x_new = x - g / gamma
        # eps-step: projection of I - A x + Y1 / rho1 onto the multi-resolution set
        Ax = blur(x_new, w)
        if eps_incomplete:
            r = _icd(I - Ax + Y1 / rho1, K, c_level, tol=icd_tol, max_sweeps=icd_max_sweeps)
            cycles.append(int(sum(int(sw.sum()) for sw in r.sweeps)))
        else:
            r = _dykstra(I - Ax + Y1 / rho1, sides, cS, max_cycles=dyk_cycles, tol=dyk_tol,
                         tol_relative=dyk_relative, n_threads=n_threads)
            cycles.append(r.cycles)
        eps = r.x
        # z-step: prox of R / rho2 at x + Y2 / rho2
        z, p1, p2 = tv_prox(x_new + Y2 / rho2, rho2, tv_iters, p1, p2)
        # multipliers
        res1 = I - Ax - eps
        Y1 = Y1 + rho1 * res1
        Y2 = Y2 + rho2 * (x_new - z)
        dx = float(np.sqrt(((x_new - x) ** 2).sum()))
        e = float(np.sqrt((res1 ** 2).sum()))
        hist.append((dx, e))
        x = x_new
        it += 1
        if delta >= 0 and dx <= delta and e <= delta:
            break
    return AdmmResult(x, z, eps, Y1, Y2, p1, p2, it, np.array(hist).reshape(-1, 2), cycles)
