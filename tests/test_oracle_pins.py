"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test fixes one piece of the oracle to a closed form, a textbook routine,
a convex-analysis property or a brute-force solution, chosen so that a
plausible mistake (a dropped term, a wrong sign or index, a transposed operand,
a wrong set order or offset) fails at least one of them.

Paper passages: weights Sec. 2.1; projection p_s of Sec. 2.3 and Algorithm 2
(Sec. 2.3); incomplete Dykstra Sec. 3.2.
"""
import numpy as np
import pytest

from synthetic import blobs_residual, random_image

scipy_stats = pytest.importorskip("scipy.stats")


# ----------------------------------------------------------------- Sec. 2.1

@pytest.mark.parametrize("alpha", [0.5, 0.9, 0.95, 0.99, 0.999])
def test_normal_quantile_matches_textbook(oracle_mod, alpha):
    assert abs(oracle_mod.normal_quantile(alpha) - scipy_stats.norm.ppf(alpha)) < 1e-12


@pytest.mark.parametrize("L", list(range(1, 13)))
@pytest.mark.parametrize("alpha", [0.5, 0.9, 0.99])
def test_chi2_quantile_matches_textbook(oracle_mod, L, alpha):
    ref = scipy_stats.chi2.ppf(alpha, L * L)
    assert abs(oracle_mod.chi2_quantile(alpha, L * L) - ref) <= 1e-10 * ref


def test_perset_bound_is_fourth_root_normal_approximation(oracle_mod):
    """The fourth-root transform of Sec. 2.1 approximates chi^2_{|s|}: the bound
    (Phi^{-1}(alpha) sigma_s + mu_s)^4 lies within 5 % of the exact quantile and
    the gap shrinks as |s| grows."""
    sides = list(range(1, 13))
    perset = oracle_mod.bounds(sides, 0.9)
    exact = np.array([scipy_stats.chi2.ppf(0.9, L * L) for L in sides])
    rel = np.abs(perset - exact) / exact
    assert rel.max() < 0.05
    assert rel[-1] < rel[0] / 10
    # mu_s and sigma_s enter as stated: |s| = 1 gives (1.28155*8^-1/2 + 0.5^1/4)^4
    z = scipy_stats.norm.ppf(0.9)
    assert abs(perset[0] - (z / np.sqrt(8.0) + 0.5 ** 0.25) ** 4) < 1e-12


def test_perset_bound_has_coverage_alpha(oracle_mod):
    """P(sum over an L x L window of N(0,1)^2 <= cS) ~= alpha (Monte Carlo with
    numpy's generator, independent of the oracle)."""
    rng = np.random.default_rng(7)
    for L, c in zip([2, 4, 8], oracle_mod.bounds([2, 4, 8], 0.9)):
        t = (rng.standard_normal((200000, L * L)) ** 2).sum(axis=1)
        assert abs((t <= c).mean() - 0.9) < 0.02


def test_normal_sample_stream_is_standard_normal(oracle_mod):
    v = np.array([oracle_mod.normal_sample(123, j) for j in range(20000)])
    assert abs(v.mean()) < 0.03 and abs(v.std() - 1.0) < 0.03
    assert scipy_stats.kstest(v, "norm").pvalue > 1e-3


def test_maxstat_quantile_brute_force(oracle_mod):
    """Q_Omega on a tiny image: the oracle's Monte Carlo quantile equals the
    quantile of maxima recomputed here from the same normal stream."""
    H, W, sides, draws, seed = 5, 4, [1, 2], 40, 99
    maxima = []
    for d in range(draws):
        img = np.array([oracle_mod.normal_sample(seed, d * H * W + p) for p in range(H * W)])
        img = img.reshape(H, W)
        best = -np.inf
        for L in sides:
            n = L * L
            mu, sg = (n - 0.5) ** 0.25, (1.0 / (8 * np.sqrt(n))) ** 0.5
            for r in range(H - L + 1):
                for c in range(W - L + 1):
                    t = (img[r:r + L, c:c + L] ** 2).sum()
                    best = max(best, (t ** 0.25 - mu) / sg)
        maxima.append(best)
    ref = np.sort(maxima)[int(np.ceil(0.9 * draws)) - 1]
    got = oracle_mod.maxstat_quantile(H, W, sides, 0.9, draws, seed)
    assert abs(got - ref) < 1e-12
    # the maximum over many windows is a larger quantile than a single window's
    assert got > scipy_stats.norm.ppf(0.9)


# --------------------------------------------------- Sec. 2.3 closed forms

@pytest.mark.parametrize("L", [1, 2, 3, 5])
def test_single_ball_closed_form(oracle_mod, L):
    """Image exactly L x L, sides {L}: one set, projection = radial scaling."""
    x0 = random_image(L, L, scale=3.0, seed=L)
    c = 0.5 * (x0 ** 2).sum()
    r = oracle_mod.dykstra(x0, [L], [c], max_cycles=3, tol=-1)
    ref = x0 * np.sqrt(c / (x0 ** 2).sum())
    assert np.abs(r.x - ref).max() < 1e-14
    # already inside: identity
    r2 = oracle_mod.dykstra(x0, [L], [2.0 * (x0 ** 2).sum()], max_cycles=2, tol=-1)
    assert np.array_equal(r2.x, x0)


def test_feasible_input_is_identity(oracle_mod):
    sides = [1, 2, 3, 4]
    x0 = random_image(17, 13, scale=0.2, seed=3)
    c = oracle_mod.bounds(sides, 0.9)
    assert oracle_mod.max_violation(x0, sides, c) < 0
    r = oracle_mod.dykstra(x0, sides, c, max_cycles=50, tol=0.0, want_q=True)
    assert r.cycles == 1 and r.hist[0, 0] == 0.0
    assert np.array_equal(r.x, x0)
    assert not r.q.any()


def test_all_sets_disjoint_is_elementwise_clamp(oracle_mod):
    """sides {1}: every set is one pixel; exact after one cycle."""
    x0 = random_image(9, 11, scale=3.0, seed=4)
    c = 2.0
    r = oracle_mod.dykstra(x0, [1], [c], max_cycles=4, tol=-1)
    ref = x0 * np.minimum(1.0, np.sqrt(c) / np.abs(x0))
    assert np.abs(r.x - ref).max() < 1e-15


def test_window_count_closed_form(oracle_mod):
    for (H, W, sides) in [(64, 64, [1, 2, 4]), (512, 512, range(1, 9)), (37, 23, [3, 5, 7])]:
        count = 0
        for (L, a, b) in oracle_mod.default_tilings(sides):
            count += ((H - a) // L) * ((W - b) // L)
        assert count == oracle_mod.n_windows(H, W, sides)
        assert count == sum((H - L + 1) * (W - L + 1) for L in set(sides))


def test_default_order_is_sides_descending_a_outer_b_inner(oracle_mod):
    til = oracle_mod.default_tilings([1, 3, 2])
    assert til[0] == (3, 0, 0) and til[1] == (3, 0, 1) and til[3] == (3, 1, 0)
    assert til[9] == (2, 0, 0) and til[-1] == (1, 0, 0) and len(til) == 14


# ------------------------------------------- Algorithm 2 invariants / KKT

def test_invariant_x_minus_sum_q_is_x0(oracle_mod):
    """With the listing's q (q_s = p_s(s1) - s1, s1 = e - q_s) every set update
    keeps e - sum_s q_s unchanged, so it equals x0 after any number of cycles."""
    sides = [1, 2, 3]
    x0 = blobs_residual(20, 18, n_blobs=2, seed=5)
    c = oracle_mod.bounds(sides, 0.9)
    for cyc in (1, 2, 7):
        r = oracle_mod.dykstra(x0, sides, c, max_cycles=cyc, tol=-1, want_q=True)
        assert np.abs(r.x - r.q.sum(axis=0) - x0).max() < 1e-12


def _tiny_solution(oracle_mod, x0, sides, c, tilings=None, cycles=20000):
    return oracle_mod.dykstra(x0, sides, c, max_cycles=cycles, tol=1e-15,
                              tilings=tilings, want_q=True)


def _windows(H, W, L):
    for r in range(H - L + 1):
        for cc in range(W - L + 1):
            yield r, cc


def test_kkt_at_convergence(oracle_mod):
    """KKT of min 1/2|x - x0|^2 s.t. |x_s|^2 <= cS: x0 - x = sum_s mu_s x|_s with
    mu_s >= 0, mu_s (|x_s|^2 - cS) = 0, and feasibility.  The increments of the
    converged iteration give the multipliers: q_s = -mu_s x|_s."""
    sides = [1, 2, 3]
    x0 = blobs_residual(9, 8, n_blobs=1, sigma=1.5, amplitude=6, seed=6)
    c = oracle_mod.bounds(sides, 0.9)
    r = _tiny_solution(oracle_mod, x0, sides, c)
    x = r.x
    assert oracle_mod.max_violation(x, sides, c) < 1e-9
    cmap = dict(zip(sides, c))
    n_active = 0
    for k, (L, a, b) in enumerate(r.tilings):
        for u in range((x.shape[0] - a) // L):
            for v in range((x.shape[1] - b) // L):
                sl = (slice(a + L * u, a + L * u + L), slice(b + L * v, b + L * v + L))
                qs, xs = r.q[k][sl], x[sl]
                nx = (xs ** 2).sum()
                mu = -(qs * xs).sum() / nx if nx > 0 else 0.0
                assert np.abs(qs + mu * xs).max() < 1e-8          # q_s parallel to x_s
                assert mu > -1e-10                                  # dual feasibility
                assert abs(mu * (nx - cmap[L])) < 1e-7 * cmap[L]   # complementary slackness
                n_active += mu > 1e-6
    assert n_active > 0
    # stationarity: x0 - x = -sum q
    assert np.abs(x0 - x + r.q.sum(axis=0)).max() < 1e-12


def _feasible_scale(z, sides, c):
    s = 1.0
    for L, cl in zip(sides, c):
        for (r, cc) in _windows(*z.shape, L):
            t = (z[r:r + L, cc:cc + L] ** 2).sum()
            if t > 0:
                s = min(s, np.sqrt(cl / t))
    return s


def test_variational_inequality(oracle_mod):
    """x* = P(x0) iff <x0 - x*, z - x*> <= 0 for every feasible z."""
    sides = [1, 2, 3]
    x0 = blobs_residual(6, 6, n_blobs=1, sigma=1.0, amplitude=5, seed=8)
    c = oracle_mod.bounds(sides, 0.9)
    xs = _tiny_solution(oracle_mod, x0, sides, c).x
    rng = np.random.default_rng(9)
    g = x0 - xs
    worst = -np.inf
    for i in range(3000):
        z = rng.standard_normal(x0.shape) * rng.uniform(0.1, 3.0)
        z *= _feasible_scale(z, sides, c) * 0.999999
        if i % 2:
            z = xs + rng.uniform(0, 1) * (z - xs)   # points between x* and z stay feasible
        worst = max(worst, (g * (z - xs)).sum())
    assert worst <= 1e-10


def test_limit_does_not_depend_on_set_order(oracle_mod):
    """Dykstra converges to the unique projection for any cyclic order."""
    sides = [1, 2, 3]
    x0 = blobs_residual(8, 7, n_blobs=1, sigma=1.2, amplitude=6, seed=10)
    c = oracle_mod.bounds(sides, 0.9)
    ref = _tiny_solution(oracle_mod, x0, sides, c).x
    til = oracle_mod.default_tilings(sides)
    asc = sorted(til, key=lambda t: (t[0], t[2], t[1]))
    rnd = [til[i] for i in np.random.default_rng(11).permutation(len(til))]
    for order in (asc, rnd):
        other = _tiny_solution(oracle_mod, x0, sides, c, tilings=order).x
        assert np.abs(other - ref).max() < 1e-10
    # but the iterates after one cycle do depend on the order
    one = oracle_mod.dykstra(x0, sides, c, max_cycles=1, tol=-1).x
    one_asc = oracle_mod.dykstra(x0, sides, c, max_cycles=1, tol=-1, tilings=asc).x
    assert np.abs(one - one_asc).max() > 1e-6


def test_matches_slsqp_on_tiny_qcqp(oracle_mod):
    """Brute force: a general-purpose constrained solver on the same QCQP."""
    from scipy.optimize import minimize
    sides = [1, 2, 3]
    x0 = blobs_residual(5, 5, n_blobs=1, sigma=1.0, amplitude=5, seed=12)
    c = oracle_mod.bounds(sides, 0.9)
    ref = _tiny_solution(oracle_mod, x0, sides, c).x
    cons = []
    for L, cl in zip(sides, c):
        for (r, cc) in _windows(5, 5, L):
            idx = [(r + i) * 5 + cc + j for i in range(L) for j in range(L)]
            cons.append({"type": "ineq",
                         "fun": (lambda v, idx=idx, cl=cl: cl - (v[idx] ** 2).sum()),
                         "jac": (lambda v, idx=idx: _grad(v, idx))})
    res = minimize(lambda v: 0.5 * ((v - x0.ravel()) ** 2).sum(), np.zeros(25),
                   jac=lambda v: v - x0.ravel(), constraints=cons, method="SLSQP",
                   options={"ftol": 1e-12, "maxiter": 1000})
    assert res.success
    assert np.abs(res.x.reshape(5, 5) - ref).max() < 1e-6


def _grad(v, idx):
    g = np.zeros_like(v)
    g[idx] = -2.0 * v[idx]
    return g


def test_stopping_rule_absolute_and_relative(oracle_mod):
    sides = [1, 2]
    x0 = blobs_residual(16, 16, n_blobs=2, seed=13)
    c = oracle_mod.bounds(sides, 0.9)
    full = oracle_mod.dykstra(x0, sides, c, max_cycles=60, tol=-1)
    d, n = full.hist[:, 0], full.hist[:, 1]
    tol = float(d[10] * 1.0000001)
    ra = oracle_mod.dykstra(x0, sides, c, max_cycles=60, tol=tol)
    assert ra.cycles == int(np.argmax(d <= tol)) + 1
    rel = float(d[12] / n[12] * 1.0000001)
    rr = oracle_mod.dykstra(x0, sides, c, max_cycles=60, tol=rel, tol_relative=True)
    assert rr.cycles == int(np.argmax(d <= rel * n)) + 1
    assert np.array_equal(rr.x, oracle_mod.dykstra(x0, sides, c, max_cycles=rr.cycles,
                                                   tol=-1).x)
    # |x_prev| of cycle 1 is |x0|
    assert abs(n[0] - np.sqrt((x0 ** 2).sum())) < 1e-12


def test_threads_bitwise_identical(oracle_mod):
    sides = [1, 2, 3, 4]
    x0 = blobs_residual(40, 33, n_blobs=3, seed=14)
    c = oracle_mod.bounds(sides, 0.9)
    a = oracle_mod.dykstra(x0, sides, c, max_cycles=3, tol=-1, n_threads=1).x
    b = oracle_mod.dykstra(x0, sides, c, max_cycles=3, tol=-1, n_threads=4).x
    assert np.array_equal(a, b)


# ------------------------------------------------------------ Sec. 3.2 (ICD)

def test_icd_K0_is_elementwise_clamp(oracle_mod):
    x0 = random_image(7, 9, scale=3.0, seed=15)
    r = oracle_mod.icd(x0, 0, [2.0], tol=0.0, max_sweeps=10)
    ref = x0 * np.minimum(1.0, np.sqrt(2.0) / np.abs(x0))
    assert np.abs(r.x - ref).max() < 1e-15
    # one set per tile: a feasible pixel ends after one sweep; otherwise the
    # second sweep changes nothing and ends the tile
    assert np.array_equal(r.sweeps[0], np.where(np.abs(x0) > np.sqrt(2.0), 2, 1))


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5])
def test_icd_stop_threshold_is_tol_times_B_squared(oracle_mod, K):
    """The tile's sweep loop ends when one sweep changes e by at most tol * B^2
    in L1 (Sec. 3.2 listing: tol * 1024 for B = 32).  A B x B image of one
    constant v has a single tile, in the last pass, holding a single set (the
    whole tile): the first sweep projects it onto the ball and changes it by
    B^2 v - B sqrt(c) in L1, the second sweep changes nothing.  So the tile
    takes two sweeps when v is a little above tol + sqrt(c) / B and one when
    it is a little below -- a threshold of tol * B or tol * B^4 would give the
    same count on both sides."""
    B = 1 << K
    c = oracle_mod.bounds([1 << k for k in range(K + 1)], 0.9)
    tol = 1e-3
    for f, want in ((1.01, 2), (0.99, 1)):
        v = np.sqrt(c[K]) / B + f * tol
        x0 = np.full((B, B), v)
        r = oracle_mod.icd(x0, K, c, tol=tol, max_sweeps=100)
        assert all(s.size == 0 for s in r.sweeps[:K])      # shifted tiles do not fit
        assert r.sweeps[K].shape == (1, 1) and int(r.sweeps[K][0, 0]) == want, (f, r.sweeps[K])
        # the change of the first sweep is f * tol * B^2 by construction
        assert abs(np.abs(x0 - r.x).sum() - f * tol * B * B) < 1e-9 * B * B
        # and the result is the projection of the tile onto its ball
        assert np.abs(r.x - x0 * np.sqrt(c[K] / (B * B * v * v))).max() < 1e-14


def test_icd_reach_mask(oracle_mod):
    """A tile with a different sweep count taints its pixels and, through
    them, every later-pass tile that overlaps them (and nothing else)."""
    H, W, K = 20, 20, 2        # B = 4: pass 0 offset 1, pass 1 offset 2, pass 2 offset 0
    grid = oracle_mod.icd_tile_grid(H, W, K)
    differ = [np.zeros((ni, nj), bool) for (_, ni, nj) in grid]
    differ[0][1, 1] = True     # pass 0 tile at rows/cols 5..8
    m = oracle_mod.icd_reach_mask(H, W, K, differ)
    ref = np.zeros((H, W), bool)
    ref[5:9, 5:9] = True                 # the tile itself
    ref[2:10, 2:10] = True               # pass 1 tiles (offset 2) overlapping rows/cols 5..8: 2..5, 6..9
    ref[0:12, 0:12] = True               # pass 2 tiles (offset 0) overlapping 2..9: 0..3, 4..7, 8..11
    assert np.array_equal(m, ref)
    assert not oracle_mod.icd_reach_mask(H, W, K, [np.zeros_like(d) for d in differ]).any()


def test_icd_tile_grid_offsets(oracle_mod):
    """Pass i uses offset (1 << i) mod B; the last pass is the aligned one."""
    g = oracle_mod.icd_tile_grid(40, 35, 3)
    assert [x[0] for x in g] == [1, 2, 4, 0]
    assert g[0][1:] == ((40 - 1) // 8, (35 - 1) // 8)
    assert g[3][1:] == (5, 4)


def test_icd_feasible_is_identity(oracle_mod):
    x0 = random_image(24, 16, scale=0.1, seed=16)
    c = oracle_mod.bounds([1, 2, 4], 0.9)
    r = oracle_mod.icd(x0, 2, c, tol=1e-3)
    assert np.array_equal(r.x, x0)
    assert all((s == 1).all() for s in r.sweeps)


def test_icd_pass_equals_exact_projection_per_tile(oracle_mod):
    """At a tight tolerance every ICD pass is the exact projection of each tile
    onto the intersection of its aligned dyadic squares, which the generic
    Dykstra routine computes with the tile as an image and tilings (2^k, 0, 0)
    (here in ascending level order, unlike the ICD's descending one)."""
    K = 2
    B = 1 << K
    sides = [1, 2, 4]
    x0 = blobs_residual(19, 22, n_blobs=2, sigma=1.5, amplitude=6, seed=17)
    c = oracle_mod.bounds(sides, 0.9)
    got = oracle_mod.icd(x0, K, c, tol=1e-15, max_sweeps=100000).x
    ref = x0.copy()
    for i, (off, ni, nj) in enumerate(oracle_mod.icd_tile_grid(*x0.shape, K)):
        lv = [1 << k for k in range(i, K + 1)]
        for ti in range(ni):
            for tj in range(nj):
                sl = (slice(off + B * ti, off + B * ti + B), slice(off + B * tj, off + B * tj + B))
                sub = oracle_mod.dykstra(ref[sl], lv, [c[int(np.log2(L))] for L in lv],
                                         max_cycles=100000, tol=1e-15,
                                         tilings=[(L, 0, 0) for L in lv])
                ref[sl] = sub.x
    assert np.abs(got - ref).max() < 1e-10


def test_icd_last_pass_sets_are_feasible_and_untouched_border(oracle_mod):
    K = 3
    x0 = blobs_residual(27, 30, n_blobs=3, seed=18)
    c = oracle_mod.bounds([1, 2, 4, 8], 0.9)
    r = oracle_mod.icd(x0, K, c, tol=1e-12, max_sweeps=100000)
    # the last pass (aligned 8 x 8 squares) leaves each of its squares feasible
    for ti in range(27 // 8):
        for tj in range(30 // 8):
            t = (r.x[8 * ti:8 * ti + 8, 8 * tj:8 * tj + 8] ** 2).sum()
            assert t <= c[3] * (1 + 1e-9)
    # pixels covered by no tile of any pass are never changed
    covered = np.zeros(x0.shape, bool)
    for (off, ni, nj) in oracle_mod.icd_tile_grid(27, 30, K):
        covered[off:off + 8 * ni, off:off + 8 * nj] = True
    assert np.array_equal(r.x[~covered], x0[~covered])


def test_max_violation_brute_force(oracle_mod):
    x = random_image(6, 5, seed=19)
    sides, c = [1, 3], [1.5, 7.0]
    ref = -np.inf
    for L, cl in zip(sides, c):
        for (r, cc) in _windows(6, 5, L):
            ref = max(ref, ((x[r:r + L, cc:cc + L] ** 2).sum() - cl) / cl)
    assert abs(oracle_mod.max_violation(x, sides, c) - ref) < 1e-14


def test_golden_bounds_table(oracle_mod):
    """Regression lock on the stored bound table (written by
    tests/golden/make_golden.py from the oracle)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "bounds_alpha0.9.txt")
    tab = np.loadtxt(path)
    L = tab[:, 0].astype(int)
    assert np.allclose(oracle_mod.bounds(L, 0.9, "perset"), tab[:, 1], rtol=1e-13, atol=0)
    assert np.allclose(oracle_mod.bounds(L, 0.9, "chi2"), tab[:, 2], rtol=1e-13, atol=0)
    # 2.8037 for L = 1 and 79.188 for L = 8, to the digits of the usual table
    assert abs(tab[0, 1] - 2.8037) < 1e-4 and abs(tab[7, 1] - 79.188) < 1e-3
