"""ADMM outer loop (Sec. 2.2, Algorithm 1 on Eq. 3) through the C ABI against
the FP64 oracle.

Tolerance.  One iteration composes the eps-step (the projection, within
1e-5 max-abs relative of FP64), two FP32 blurs (<= 49 taps a pixel) and
FP32 TV steps (relative rounding ~1e-7 each).  The iteration map is
nonexpansive, so rounding does not grow from one iteration to the next;
it only adds up: after K iterations the max-abs relative error stays below
K * 2e-5.  The tests run K <= 4 and check 1e-4."""
import numpy as np
import pytest

import oracle
from oracle import admm as OA

torch = pytest.importorskip("torch")
smre = pytest.importorskip("paper_1503_03492_gb300")

pytestmark = pytest.mark.gpu

TOL_PER_ITER = 2e-5


def _image(H, W, sigma, seed, n_emitters=None):
    rng = np.random.default_rng(seed)
    truth = np.zeros((H, W))
    n = n_emitters if n_emitters is not None else max(3, H * W // 300)
    ii = rng.integers(0, H, n)
    jj = rng.integers(0, W, n)
    np.add.at(truth, (ii, jj), rng.uniform(4.0, 10.0, n))
    I = OA.blur(truth, OA.gaussian_kernel(sigma)) + rng.normal(size=(H, W))
    return I.astype(np.float32)


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def _run(I32, sides, sigma, iters, radius=0, rho1=1.0, rho2=1.0, tv_iters=10, dyk_cycles=30):
    H, W = I32.shape
    cS = oracle.bounds(sides, 0.9)
    Id = torch.from_numpy(I32).cuda()
    x = torch.empty_like(Id)
    z = torch.empty_like(Id)
    e = torch.empty_like(Id)
    with smre.Admm(H, W, sides, sigma, radius=radius, rho1=rho1, rho2=rho2, tv_iters=tv_iters,
                   max_iters=iters, delta=-1.0, cmode=smre.SMRE_C_EXPLICIT, c_explicit=list(cS),
                   max_cycles=dyk_cycles, tol=-1.0) as A:
        res = A.solve(Id, x, z, e)
        launches = A.kernel_launches()
    torch.cuda.synchronize()
    ref = OA.admm(I32.astype(np.float64), sides, cS, sigma=sigma, radius=radius, rho1=rho1, rho2=rho2,
                  tv_iters=tv_iters, max_iters=iters, dyk_cycles=dyk_cycles, dyk_tol=-1.0,
                  n_threads=oracle.max_threads())
    return res, launches, x.cpu().numpy(), z.cpu().numpy(), e.cpu().numpy(), ref


@pytest.mark.parametrize("H,W,sides,sigma,radius,iters,tv_iters", [
    (40, 72, [1, 2, 4], 1.0, 0, 4, 10),     # ragged tiles in both directions
    (33, 31, [1, 3], 0.8, 0, 3, 0),         # one tile with a ragged edge; z-step = identity
    (70, 45, [2, 5], 4.0, 16, 2, 6),        # widest halo (radius 16) over a small image
])
def test_admm_matches_oracle(H, W, sides, sigma, radius, iters, tv_iters):
    I = _image(H, W, sigma, seed=H * 1000 + W)
    res, launches, x, z, e, ref = _run(I, sides, sigma, iters, radius=radius, tv_iters=tv_iters)
    assert res.iters == iters and res.status == smre.SMRE_OK
    assert res.dykstra_cycles == iters * 30
    assert launches == iters * (3 + -(-tv_iters // 4))   # four TV steps a launch
    tol = TOL_PER_ITER * iters
    assert _rel(x, ref.x) <= tol
    assert _rel(z, ref.z) <= tol
    assert _rel(e, ref.eps) <= tol
    # the reported norms are those of the last iteration
    assert res.dx == pytest.approx(ref.hist[-1, 0], rel=1e-3)
    assert res.residual == pytest.approx(ref.hist[-1, 1], rel=1e-3, abs=1e-6)


def test_admm_incomplete_eps_step_matches_oracle():
    # the eps-step by the incomplete Dykstra (Sec. 3.2), K = 2, tol 0 (every
    # tile sweeps to the cap of 4 unless a sweep changes nothing)
    H, W, sides, sigma, iters = 40, 72, [1, 2, 4], 1.0, 3
    I = _image(H, W, sigma, seed=99)
    cS = oracle.bounds(sides, 0.9)
    Id = torch.from_numpy(I).cuda()
    x, z, e = (torch.empty_like(Id) for _ in range(3))
    with smre.Admm(H, W, sides, sigma, tv_iters=5, max_iters=iters, delta=-1.0, eps_incomplete=True,
                   icd_K=2, icd_tol=0.0, cmode=smre.SMRE_C_EXPLICIT, c_explicit=list(cS),
                   icd_max_sweeps=4) as A:
        res = A.solve(Id, x, z, e)
    ref = OA.admm(I.astype(np.float64), sides, cS, sigma=sigma, tv_iters=5, max_iters=iters,
                  eps_incomplete=True, icd_K=2, icd_tol=0.0, icd_max_sweeps=4)
    assert abs(res.dykstra_cycles - sum(ref.dykstra_cycles)) <= 0.01 * sum(ref.dykstra_cycles)
    tol = TOL_PER_ITER * iters
    assert _rel(x.cpu().numpy(), ref.x) <= tol
    assert _rel(z.cpu().numpy(), ref.z) <= tol
    assert _rel(e.cpu().numpy(), ref.eps) <= tol


def test_admm_full_size_emitter_image():
    # the 512 x 512 emitter residual with the PSF of its generator (sigma 2),
    # sides 1..8, three iterations of 20 projection cycles
    from synthetic import emitter_residual
    I = np.ascontiguousarray(emitter_residual(), np.float32)
    res, _, x, z, e, ref = _run(I, list(range(1, 9)), 2.0, 3, tv_iters=20, dyk_cycles=20)
    tol = TOL_PER_ITER * 3
    assert _rel(x, ref.x) <= tol
    assert _rel(z, ref.z) <= tol
    assert _rel(e, ref.eps) <= tol


def test_admm_stopping_rule():
    # the loop stops once both norms are <= delta (the FP64 oracle needs a few
    # hundred iterations here), and reports ENOTCONVERGED at the cap
    I = _image(24, 40, 0.6, seed=7)
    sides = [1, 2]
    cS = oracle.bounds(sides, 0.9)
    Id = torch.from_numpy(I).cuda()
    x = torch.empty_like(Id)
    e = torch.empty_like(Id)
    with smre.Admm(24, 40, sides, 0.6, tv_iters=20, max_iters=3000, delta=2e-2,
                   cmode=smre.SMRE_C_EXPLICIT, c_explicit=list(cS), max_cycles=100, tol=1e-7) as A:
        r = A.solve(Id, x, None, e)
        assert r.status == smre.SMRE_OK and r.iters < 3000
        assert r.dx <= 2e-2 and r.residual <= 2e-2
        # eps comes from the projection (at most 100 cycles): inside the set up to
        # what those cycles leave (the FP64 oracle: 3e-6 here)
        assert oracle.max_violation(e.cpu().numpy().astype(np.float64), sides, cS) < 1e-4
    with smre.Admm(24, 40, sides, 0.6, tv_iters=20, max_iters=2, delta=1e-12,
                   cmode=smre.SMRE_C_EXPLICIT, c_explicit=list(cS), max_cycles=20, tol=-1.0) as A:
        r = A.solve(Id, x)
        assert r.status == smre.SMRE_ENOTCONVERGED and r.iters == 2


@pytest.mark.parametrize("q_dtype,u", [(1, 2.0 ** -8), (2, 2.0 ** -11)])
def test_admm_with_16bit_increments(q_dtype, u):
    """The eps-step through a projection with BF16 / FP16 increments (a
    one-image batch), against the FP64 oracle of the same loop: the FP32 loop
    within K * 2e-5 of it, the 16-bit loop within K times the 16-bit envelope
    (4 u a projection) plus that.  The envelope is measured, not a proven
    bound: each set update perturbs the exact projection by at most u |q_i| a
    pixel, and nothing here bounds how those perturbations add up."""
    H, W, sides, sigma, iters = 40, 72, [1, 2, 4], 1.0, 3
    I = _image(H, W, sigma, seed=5)
    cS = oracle.bounds(sides, 0.9)
    Id = torch.from_numpy(I).cuda()
    outs = []
    for qd in (0, q_dtype):
        x = torch.empty_like(Id)
        with smre.Admm(H, W, sides, sigma, tv_iters=5, max_iters=iters, delta=-1.0, q_dtype=qd,
                       cmode=smre.SMRE_C_EXPLICIT, c_explicit=list(cS), max_cycles=20, tol=-1.0) as A:
            A.solve(Id, x)
        outs.append(x.cpu().numpy())
    ref = OA.admm(I.astype(np.float64), sides, cS, sigma=sigma, tv_iters=5, max_iters=iters,
                  dyk_cycles=20, dyk_tol=-1.0, n_threads=oracle.max_threads())
    e32, e16 = _rel(outs[0], ref.x), _rel(outs[1], ref.x)
    print(f"q_dtype {q_dtype}: x vs FP64 oracle, FP32 increments {e32:.2e}, 16-bit {e16:.2e} "
          f"({e16 / u:.2f} u)")
    assert e32 <= iters * TOL_PER_ITER
    assert e16 <= iters * (4 * u + TOL_PER_ITER)
    assert _rel(outs[1], outs[0]) <= iters * 4 * u


def test_admm_rejects_host_images():
    # the solver's kernels use the images directly: host memory is an EINVAL
    I = _image(32, 40, 1.0, seed=3)
    cS = oracle.bounds([1, 2], 0.9)
    with smre.Admm(32, 40, [1, 2], 1.0, max_iters=1, cmode=smre.SMRE_C_EXPLICIT,
                   c_explicit=list(cS), max_cycles=2, tol=-1.0) as A:
        x = np.empty_like(I)
        with pytest.raises(smre.SmreError) as ei:
            A.solve(I, x)
        assert ei.value.status == smre.SMRE_EINVAL
        Id = torch.from_numpy(I).cuda()
        with pytest.raises(smre.SmreError):
            A.solve(Id, x)
        xd = torch.empty_like(Id)
        A.solve(Id, xd)   # still usable
