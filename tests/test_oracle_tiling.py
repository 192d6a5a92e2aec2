"""Pins of the oracle's tiled proposal (Sec. II; App. A) against the likelihood's own inner
products, the Fisher metric, brute force and exact identities of the mixture."""
import math

import numpy as np
import pytest

import oracle
import workloads
from workloads import MC, Q, PHIC

F_LO, DF, NB = 20.0, 0.25, 1969


@pytest.fixture(scope="module")
def grid():
    f = F_LO + DF * np.arange(NB)
    return f, oracle.psd_aligo(f)


@pytest.fixture(scope="module")
def demo(grid):
    """The demonstration space: Mc = 24 + mod(x, 4) over x in [20, 28), q in [1/6, 6]."""
    return oracle.Tiling(F_LO, DF, NB, grid[1], 20.0, 28.0, 4.0, 24.0, 1 / 6, 6.0)


def single_detector_event(psd):
    v, x, y = workloads.network(["H1"])
    return oracle.OracleEvent(F_LO, DF, NB, psd.reshape(1, -1), v, x, y, gmst=0.0, marg=0)


def params(mc, q):
    p = np.zeros(11)
    p[MC], p[Q] = mc, q
    p[workloads.RA], p[workloads.DEC], p[workloads.PSI], p[workloads.IOTA] = 1.0, 0.5, 0.3, 0.4
    p[workloads.DL] = 100.0
    return p


def test_match_equals_the_normalised_overlap_of_the_likelihood_inner_product(grid, demo):
    """match(a, b) = |(h_a|h_b)| / sqrt((h_a|h_a)(h_b|h_b)) with (.|.) the likelihood's
    inner product (Eq. 1) of detector strains: data h_a without noise, template h_b."""
    ev = single_detector_event(grid[1])
    rng = np.random.default_rng(5)
    for _ in range(6):
        xa, xb = rng.uniform(20, 28, 2)
        qa, qb = rng.uniform(1 / 6, 6, 2)
        mca, qpa = demo.physical(xa, qa)
        mcb, qpb = demo.physical(xb, qb)
        ev.set_strain(oracle.make_strain(ev, params(mca, qpa)))
        z, hb = oracle.overlaps(ev, params(mcb, qpb))
        ha = oracle.optimal_snr2(ev, params(mca, qpa))
        want = abs(z) / math.sqrt(ha * hb)
        assert demo.match(xa, qa, xb, qb) == pytest.approx(want, rel=1e-12, abs=1e-14)


def test_mismatch_follows_the_phase_projected_fisher_metric(grid, demo):
    """1 - match(theta, theta + d) = d^T g d / 2 + O(|d|^3), g the Fisher matrix over (Mc, q)
    with the phase projected out (Schur complement), divided by (h|h)."""
    ev = single_detector_event(grid[1])
    th = params(25.0, 3.5)
    steps = np.array([25e-6, 3.5e-6, 1e-6])
    G = oracle.fisher(ev, th, [MC, Q, PHIC], steps)
    g = (G[:2, :2] - np.outer(G[:2, 2], G[2, :2]) / G[2, 2]) / oracle.optimal_snr2(ev, th)
    for d in ([2e-3, 0.0], [0.0, 4e-3], [1.5e-3, -2e-3], [-1e-3, -3e-3]):
        d = np.array(d)
        mm = 1.0 - demo.match(25.0, 3.5, 25.0 + d[0], 3.5 + d[1])
        assert mm == pytest.approx(0.5 * d @ g @ d, rel=2e-2)


def test_coordinate_map_and_its_images(demo):
    assert demo.physical(21.0, 3.5) == (25.0, 3.5)
    mc, qp = demo.physical(25.0, 1 / 3.5)
    assert mc == 25.0 and qp == pytest.approx(3.5, rel=1e-15)
    assert demo.physical(27.5, 0.25) == (27.5, 4.0)
    # the four images of one binary have one waveform
    for x, q in ((25.0, 3.5), (21.0, 1 / 3.5), (25.0, 1 / 3.5)):
        assert demo.match(21.0, 3.5, x, q) == pytest.approx(1.0, abs=1e-13)
    u, live = demo.waveform(21.0, 3.5)
    assert live == int(np.ceil((oracle.f_isco(25.0, 3.5) - F_LO) / DF))
    assert np.vdot(u, u).real == pytest.approx(1.0, abs=1e-14)
    assert np.all(u[live:] == 0)


def test_bank_packs_below_and_covers_above_the_minimal_match(grid):
    """Template pairs match below the minimal match; every rejected candidate matches some
    earlier template at or above it; placement stops after the stated run of rejections."""
    t = oracle.Tiling(F_LO, DF, NB, grid[1], 24.0, 26.0, 0.0, 0.0, 1.0, 3.0)
    cand = workloads.uniform_points(3000, 24.0, 26.0, 1.0, 3.0, seed=11)
    mm, stop = 0.97, 300
    idx, used, margin = t.bank(cand, mm, stop, 4096)
    assert len(idx) >= 5 and idx[0] == 0 and margin > 0
    tx, tq = cand[0][idx], cand[1][idx]
    for a in range(len(idx)):
        for b in range(a):
            assert t.match(tx[a], tq[a], tx[b], tq[b]) < mm
    accepted = set(idx.tolist())
    for i in range(used):
        if i in accepted:
            continue
        earlier = [j for j in idx if j < i]
        assert max(t.match(cand[0][i], cand[1][i], cand[0][j], cand[1][j]) for j in earlier) >= mm
    if used < cand.shape[1]:
        assert used - 1 - idx[-1] >= stop  # the last `stop` candidates visited were rejected


def test_assignment_is_the_best_template(grid):
    t = oracle.Tiling(F_LO, DF, NB, grid[1], 20.0, 28.0, 4.0, 24.0, 1 / 6, 6.0)
    cand = workloads.uniform_points(2000, 20.0, 28.0, 1 / 6, 6.0, seed=12)
    idx, _, _ = t.bank(cand, 0.95, 200, 4096)
    tpl = cand[:, idx]
    pts = workloads.uniform_points(40, 20.0, 28.0, 1 / 6, 6.0, seed=13)
    tile, match, second = t.assign(pts, tpl)
    for i in range(pts.shape[1]):
        m = np.array([t.match(pts[0, i], pts[1, i], tpl[0, j], tpl[1, j]) for j in range(tpl.shape[1])])
        assert tile[i] == int(np.argmax(m)) and match[i] == pytest.approx(m.max(), abs=1e-13)
        assert second[i] == pytest.approx(np.sort(m)[-2], abs=1e-13)
    # a template and its images land in its own tile with match one
    j = len(idx) // 2
    img = np.array([[tpl[0, j], tpl[0, j] + 4.0 if tpl[0, j] < 24.0 else tpl[0, j] - 4.0], [tpl[1, j], 1 / tpl[1, j]]])
    tile, match, _ = t.assign(img, tpl)
    assert list(tile) == [j, j] and np.allclose(match, 1.0, atol=1e-13)


def test_lists_group_members_by_tile_in_sample_order():
    rng = np.random.default_rng(3)
    tile = rng.integers(-1, 7, 500).astype(np.int32)
    count, offset, members = oracle.tiling_lists(tile, 7)
    assert count.sum() == np.sum(tile >= 0)
    for j in range(7):
        got = members[offset[j]:offset[j] + count[j]]
        assert np.array_equal(got, np.flatnonzero(tile == j))


def mixture_case(seed=4, N=600, T=9):
    rng = np.random.default_rng(seed)
    tile = rng.integers(0, T, N).astype(np.int32)
    tile[tile == 3] = 4                     # tile 3 has no members
    ll_tpl = rng.normal(5.0, 3.0, T)
    count, offset, members = oracle.tiling_lists(tile, T)
    c, m = oracle.tiling_mixture(count, ll_tpl)
    return tile, ll_tpl, count, offset, members, c, m


def test_mixture_weights_and_the_exact_expectation_of_the_weights():
    """Over the discrete proposal, E_g[w] = sum_i P(i) L_i pi_i / g_i = (1/N) sum_i L_i
    exactly, whatever the per-sample likelihood; p_j = n_j L_j / sum_k n_k L_k."""
    tile, ll_tpl, count, offset, members, c, m = mixture_case()
    N = len(tile)
    p = count * np.exp(ll_tpl - ll_tpl[count > 0].max())
    p /= p.sum()
    assert np.allclose(np.diff(np.concatenate([[0.0], c])) / c[-1], p, rtol=1e-13, atol=1e-16)
    ll_i = np.random.default_rng(9).normal(4.0, 2.0, N)
    log_ratio = ll_tpl[tile] - m - math.log(c[-1]) + math.log(N)   # ln g - ln pi of each pool member
    prob = p[tile] / count[tile]                                   # P(draw member i)
    assert np.sum(prob) == pytest.approx(1.0, rel=1e-13)
    e_w = np.sum(prob * np.exp(ll_i - log_ratio))
    assert e_w == pytest.approx(np.mean(np.exp(ll_i)), rel=1e-12)
    # the oracle's draw reports the same ln g - ln pi
    _, tile_d, lr = oracle.tiling_draw(7, 0, 200, c, m, ll_tpl, count, offset, members, N)
    assert np.allclose(lr, ll_tpl[tile_d] - m - math.log(c[-1]) + math.log(N), rtol=0, atol=1e-13)


def test_likelihood_constant_per_tile_gives_equal_weights():
    """When L(theta) equals the likelihood at its tile's template, every weight is the same:
    ESS = n and log Z = ln sum_j (n_j / N) L_j (proposal proportional to the target)."""
    tile, ll_tpl, count, offset, members, c, m = mixture_case()
    N = len(tile)
    idx, tile_d, lr = oracle.tiling_draw(21, 100, 5000, c, m, ll_tpl, count, offset, members, N)
    assert np.array_equal(tile[idx], tile_d)
    r = oracle.reduce(ll_tpl[tile_d], np.zeros(len(idx)), lr)
    assert r["ess"] == pytest.approx(len(idx), rel=1e-12)
    want = math.log(np.sum(count * np.exp(ll_tpl)) / N)
    assert r["log_z"] == pytest.approx(want, rel=1e-12)


def test_draw_frequencies_counters_and_members():
    tile, ll_tpl, count, offset, members, c, m = mixture_case(N=400, T=5)
    N = len(tile)
    n = 200000
    idx, tile_d, _ = oracle.tiling_draw(1234, 0, n, c, m, ll_tpl, count, offset, members, N)
    p = np.diff(np.concatenate([[0.0], c])) / c[-1]
    obs = np.bincount(tile_d, minlength=len(count))
    assert obs[3] == 0
    live = p > 0
    chi2 = np.sum((obs[live] - n * p[live]) ** 2 / (n * p[live]))
    assert chi2 < 30.0                                  # 3 or 4 dof
    # members drawn uniformly within the most probable tile
    j = int(np.argmax(p))
    sub = idx[tile_d == j]
    hist = np.bincount(np.searchsorted(members[offset[j]:offset[j] + count[j]], sub), minlength=count[j])
    e = len(sub) / count[j]
    assert np.sum((hist - e) ** 2 / e) < count[j] + 6 * math.sqrt(2 * count[j])
    # a draw is named by its counter
    a, ta, la = oracle.tiling_draw(99, 5, 10, c, m, ll_tpl, count, offset, members, N)
    b, tb, lb = oracle.tiling_draw(99, 0, 15, c, m, ll_tpl, count, offset, members, N)
    assert np.array_equal(a, b[5:]) and np.array_equal(ta, tb[5:]) and np.array_equal(la, lb[5:])
