"""The tiled proposal (Sec. II; App. A) on the device, through the C ABI, against the FP64
oracle on the two-parameter demonstration space.

* FP64 matches and template placement: identical banks (every accept decision of the
  oracle lies far from the minimal match compared with FP64 rounding).
* Tile assignment (FP16 tensor-core contraction): the chosen template's match is within
  MATCH_TOL of the best one, and equals the oracle's choice wherever the two best
  templates differ by more than 2 MATCH_TOL; the reported match is within MATCH_TOL.
* Member lists, mixture and draws: bitwise the oracle's on a pool without near ties.
* End to end: ESS and log Z of the tiled proposal against the oracle's on the same draws.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle.events import make_event
from gpu_common import LOGL_TOL, m, torch, gpu_context, set_metric  # noqa: F401

pytestmark = pytest.mark.gpu

# FP16 operands round to 2^-11 relative: with unit-norm waveforms the match error is at most
# ~1e-3 (all roundings aligned) and ~3e-5 for independent roundings over 100-240 live bins;
# the largest seen over a few thousand points is 7.6e-5.
MATCH_TOL = 2e-4


@pytest.fixture(scope="module")
def demo():
    return workloads.tiled_demo()


@pytest.fixture(scope="module")
def psd(demo):
    w = demo.workload
    return oracle.psd_aligo(w.f_lo + w.df * np.arange(w.n_bins))


@pytest.fixture(scope="module")
def otl(demo, psd):
    w = demo.workload
    return oracle.Tiling(w.f_lo, w.df, w.n_bins, psd, demo.x_lo, demo.x_hi, demo.mc_period, demo.mc_base, demo.q_lo,
                         demo.q_hi)


@pytest.fixture(scope="module")
def gtl(m, torch, demo, psd):
    w = demo.workload
    t = m.mbis_tiling_create(w.f_lo, w.df, w.n_bins, psd, demo.x_lo, demo.x_hi, demo.mc_period, demo.mc_base,
                             demo.q_lo, demo.q_hi)
    yield t
    m.mbis_tiling_destroy(t)


@pytest.fixture(scope="module")
def banks(m, demo, otl, gtl):
    cand = workloads.uniform_points(demo.n_candidates, demo.x_lo, demo.x_hi, demo.q_lo, demo.q_hi,
                                    demo.candidate_seed)
    idx_o, used_o, margin = otl.bank(cand, demo.min_match, demo.stop_after, demo.max_templates)
    T, used = m.mbis_tiling_bank(gtl, cand, demo.min_match, demo.stop_after, demo.max_templates)
    coords, phys, idx_g = m.mbis_tiling_templates(gtl)
    return dict(cand=cand, idx_o=idx_o, used_o=used_o, margin=margin, T=T, used=used, coords=coords, phys=phys,
                idx_g=idx_g, tpl=cand[:, idx_o])


def dev(torch, a, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def test_fp64_pair_match_equals_the_oracle(m, torch, demo, otl, gtl):
    a = workloads.uniform_points(300, demo.x_lo, demo.x_hi, demo.q_lo, demo.q_hi, 101)
    b = a + np.array([[0.01], [0.02]]) * workloads.uniform_points(300, -1, 1, -1, 1, 102)
    b[0] = np.clip(b[0], demo.x_lo, demo.x_hi - 1e-9)
    b[1] = np.clip(b[1], demo.q_lo, demo.q_hi)
    b[:, :5] = a[:, :5]                                     # identical points: match 1
    b[:, 5] = [a[0, 5] + 4.0 if a[0, 5] < 24 else a[0, 5] - 4.0, 1.0 / a[1, 5]]  # an image: match 1
    out = torch.empty(300, dtype=torch.float64, device="cuda")
    m.mbis_tiling_match(gtl, 300, dev(torch, a), dev(torch, b), out)
    got = out.cpu().numpy()
    want = np.array([otl.match(a[0, i], a[1, i], b[0, i], b[1, i]) for i in range(300)])
    assert np.abs(got - want).max() <= 1e-12
    assert np.allclose(got[:6], 1.0, atol=1e-12)


def test_template_placement_equals_the_oracle(demo, otl, banks):
    assert banks["margin"] > 1e-10, "an accept decision of this seed lies within FP64 rounding of the minimal match"
    assert banks["T"] == len(banks["idx_o"]) and banks["used"] == banks["used_o"]
    assert np.array_equal(banks["idx_g"], banks["idx_o"])
    assert np.array_equal(banks["coords"], banks["tpl"])
    for j in range(0, banks["T"], 97):
        mc, qp = otl.physical(*banks["tpl"][:, j])
        assert banks["phys"][0, j] == mc and banks["phys"][1, j] == qp
    print(f"bank: {banks['T']} templates from {banks['used']} candidates, decision margin {banks['margin']:.2e}")


def check_assignment(otl, tpl, pts, tile, match):
    """Every point's tile against the oracle: near-best always, the oracle's tile wherever
    the best two templates are separated; returns the largest match error."""
    t_o, best, second = otl.assign(pts, tpl)
    sep = best - second > 2 * MATCH_TOL
    assert np.array_equal(tile[sep], t_o[sep])
    chosen = np.array([otl.match(pts[0, i], pts[1, i], tpl[0, tile[i]], tpl[1, tile[i]]) for i in range(len(tile))])
    assert np.all(chosen >= best - MATCH_TOL)
    err = np.abs(match.astype(np.float64) - chosen)
    assert err.max() <= MATCH_TOL, err.max()
    return err.max(), 1.0 - sep.mean()


def test_tensor_core_assignment_against_the_oracle(m, torch, demo, otl, gtl, banks):
    tpl = banks["tpl"]
    # several 256-sample CTAs and a ragged tail; the templates themselves; their images
    pts = workloads.uniform_points(2048 + 77, demo.x_lo, demo.x_hi, demo.q_lo, demo.q_hi, 103)
    j = np.arange(0, banks["T"], 7)
    img = np.stack([np.where(tpl[0, j] < 24.0, tpl[0, j] + 4.0, tpl[0, j] - 4.0), 1.0 / tpl[1, j]])
    pts = np.concatenate([pts, tpl[:, j], img], axis=1)
    n = pts.shape[1]
    tile = torch.empty(n, dtype=torch.int32, device="cuda")
    match = torch.empty(n, dtype=torch.float32, device="cuda")
    m.mbis_tiling_assign(gtl, n, dev(torch, pts), tile, match)
    torch.cuda.synchronize()
    tile, match = tile.cpu().numpy(), match.cpu().numpy()
    err, amb = check_assignment(otl, tpl, pts, tile, match)
    k = len(j)
    assert np.array_equal(tile[n - 2 * k:n - k], j) and np.array_equal(tile[n - k:], j)
    print(f"assignment: max |match error| {err:.2e}, {100 * amb:.1f}% of points within 2e-4 of a tie")


def test_assignment_over_long_bands_rewrites_the_sample_tiles(m, torch):
    """A finer grid (df = 1/16 Hz, up to 960 live bins: 30 K-blocks per sample, records read
    through L1 instead of shared memory) against the oracle."""
    f_lo, df = 20.0, 1.0 / 16
    nb = workloads.n_bins_for(f_lo, 128.0, df)
    psd = oracle.psd_aligo(f_lo + df * np.arange(nb))
    otl = oracle.Tiling(f_lo, df, nb, psd, 24.0, 26.0, 0.0, 0.0, 1.0, 3.0)
    t = m.mbis_tiling_create(f_lo, df, nb, psd, 24.0, 26.0, 0.0, 0.0, 1.0, 3.0)
    try:
        cand = workloads.uniform_points(6000, 24.0, 26.0, 1.0, 3.0, seed=31)
        idx_o, used_o, margin = otl.bank(cand, 0.995, 400, 4096)
        T, used = m.mbis_tiling_bank(t, cand, 0.995, 400, 4096)
        assert margin > 1e-10 and T == len(idx_o) and used == used_o
        pts = workloads.uniform_points(1500 + 11, 24.0, 26.0, 1.0, 3.0, seed=32)
        n = pts.shape[1]
        tile = torch.empty(n, dtype=torch.int32, device="cuda")
        match = torch.empty(n, dtype=torch.float32, device="cuda")
        m.mbis_tiling_assign(t, n, dev(torch, pts), tile, match)
        torch.cuda.synchronize()
        err, amb = check_assignment(otl, cand[:, idx_o], pts, tile.cpu().numpy(), match.cpu().numpy())
        print(f"long band ({nb} bins, {T} templates): max |match error| {err:.2e}")
    finally:
        m.mbis_tiling_destroy(t)


def test_assignment_edge_cases(m, torch, demo, gtl, banks):
    # points outside the space get no tile; an empty call is a no-op
    pts = np.array([[demo.x_hi + 1.0, demo.x_lo, 21.0], [1.0, demo.q_hi * 2, 3.5]])
    tile = torch.full((3,), 7, dtype=torch.int32, device="cuda")
    match = torch.full((3,), 7.0, dtype=torch.float32, device="cuda")
    m.mbis_tiling_assign(gtl, 3, dev(torch, pts), tile, match)
    m.mbis_tiling_assign(gtl, 0, dev(torch, pts), tile, match)
    torch.cuda.synchronize()
    t = tile.cpu().numpy()
    assert t[0] == -1 and t[1] == -1 and t[2] >= 0 and match.cpu().numpy()[2] > 0.99
    with pytest.raises(m.MbisError):           # a pool point outside the space is refused
        m.mbis_tiling_set_pool(gtl, 3, dev(torch, pts))


@pytest.fixture(scope="module")
def event(demo):
    w = demo.workload
    spec = w.events[0]
    ev, th, _ = make_event(w, spec)
    return w, spec, ev, th


@pytest.fixture(scope="module")
def ctx(m, event):
    w, spec, ev, th = event
    c = gpu_context(m, ev, w, spec, th, m.MIXED)
    set_metric(m, c, dict(ids=np.array([workloads.MC, workloads.Q], dtype=np.int32), mean=np.array([25.0, 3.5]),
                          chol=np.diag([0.1, 0.1]), scale=1.0, lo=np.array([24.0, 1.0]), hi=np.array([28.0, 6.0]),
                          flags=0))
    yield c
    m.mbis_destroy(c)


def full_rows(th, theta_phys):
    out = np.tile(th, (theta_phys.shape[1], 1))
    out[:, workloads.MC], out[:, workloads.Q] = theta_phys[0], theta_phys[1]
    return out


def test_lists_mixture_draws_and_weights_equal_the_oracle(m, torch, demo, otl, gtl, banks, event, ctx):
    """On a pool without near ties the GPU's tiles, lists and draws are the oracle's, and the
    importance-sampling estimate matches the oracle's on the same draws."""
    w, spec, ev, th = event
    tpl = banks["tpl"]
    T = banks["T"]
    raw = workloads.uniform_points(1 << 14, demo.x_lo, demo.x_hi, demo.q_lo, demo.q_hi, demo.pool_seed)
    t_o, best, second = otl.assign(raw, tpl)
    pool = np.ascontiguousarray(raw[:, best - second > 2 * MATCH_TOL])
    N = pool.shape[1]
    m.mbis_tiling_set_pool(gtl, N, dev(torch, pool))
    tile_of = torch.empty(N, dtype=torch.int32, device="cuda")
    members = torch.empty(N, dtype=torch.int32, device="cuda")
    counts = m.mbis_tiling_pool(gtl, T, tile_of, members)
    torch.cuda.synchronize()
    t_o = t_o[best - second > 2 * MATCH_TOL]
    count_o, offset_o, members_o = oracle.tiling_lists(t_o, T)
    assert np.array_equal(tile_of.cpu().numpy(), t_o)
    assert np.array_equal(counts, count_o) and np.array_equal(members.cpu().numpy(), members_o)
    # template likelihoods: the GPU's against the oracle's, then the oracle's into both mixtures
    ll_tpl_o = oracle.loglike_batch(ev, full_rows(th, banks["phys"]))
    ll_tpl_g = torch.empty(T, dtype=torch.float64, device="cuda")
    m.mbis_loglike(ctx, T, dev(torch, banks["phys"]), ll_tpl_g)
    torch.cuda.synchronize()
    assert np.abs(ll_tpl_g.cpu().numpy() - ll_tpl_o).max() <= LOGL_TOL
    m.mbis_tiling_set_loglike(gtl, dev(torch, ll_tpl_o))
    c_o, m_o = oracle.tiling_mixture(count_o, ll_tpl_o)
    n, seed = 8192 + 33, demo.draw_seed
    theta = torch.empty((2, n), dtype=torch.float64, device="cuda")
    coords = torch.empty((2, n), dtype=torch.float64, device="cuda")
    lq, lp, ll = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
    pidx = torch.empty(n, dtype=torch.int32, device="cuda")
    m.mbis_tiling_draw(gtl, seed, 1000, n, theta, lq, lp, coords=coords, pool_index=pidx)
    m.mbis_loglike(ctx, n, theta, ll)
    s = m.mbis_reduce(ctx, n, ll, lp, lq)
    torch.cuda.synchronize()
    idx_o, tile_d, lr_o = oracle.tiling_draw(seed, 1000, n, c_o, m_o, ll_tpl_o, count_o, offset_o, members_o, N)
    assert np.array_equal(pidx.cpu().numpy(), idx_o)
    assert np.array_equal(coords.cpu().numpy(), pool[:, idx_o])
    phys = np.array([otl.physical(*pool[:, i]) for i in idx_o]).T
    assert np.array_equal(theta.cpu().numpy(), phys)
    lp_o = -math.log((demo.x_hi - demo.x_lo) * (demo.q_hi - demo.q_lo))
    assert np.all(lp.cpu().numpy() == lp_o)
    assert np.abs(lq.cpu().numpy() - (lp_o + lr_o)).max() <= 1e-12
    ll_o = oracle.loglike_batch(ev, full_rows(th, phys))
    assert np.abs(ll.cpu().numpy() - ll_o).max() <= LOGL_TOL
    r = oracle.reduce(ll_o, np.full(n, lp_o), lp_o + lr_o)
    assert s["ess"] == pytest.approx(r["ess"], rel=1e-3)
    assert abs(s["log_z"] - r["log_z"]) <= 1e-3
    print(f"tiled proposal on {N} pool points: ESS {s['ess']:.0f} of {n} ({100 * s['ess'] / n:.1f}%), "
          f"log Z {s['log_z']:.4f} (oracle {r['log_z']:.4f})")


def test_full_size_pool_covers_the_four_modes(m, torch, demo, otl, gtl, banks, ctx):
    """The demonstration at full size: a 2^22-point pool (tiles checked on a sample against
    the oracle), template likelihoods and draws on the device.  The posterior is symmetric
    between the two chirp-mass periods (equal halves of the weight) and every mode of
    (period, q < 1 or q > 1) is drawn."""
    T, N = banks["T"], demo.n_pool
    pool = workloads.uniform_points(N, demo.x_lo, demo.x_hi, demo.q_lo, demo.q_hi, demo.pool_seed + 1)
    m.mbis_tiling_set_pool(gtl, N, dev(torch, pool))
    tile_of = torch.empty(N, dtype=torch.int32, device="cuda")
    members = torch.empty(N, dtype=torch.int32, device="cuda")
    counts = m.mbis_tiling_pool(gtl, T, tile_of, members)
    torch.cuda.synchronize()
    tile_of, members = tile_of.cpu().numpy(), members.cpu().numpy()
    assert counts.sum() == N and np.array_equal(counts, np.bincount(tile_of, minlength=T))
    order = np.argsort(tile_of, kind="stable")
    assert np.array_equal(members, order)      # grouped by tile, each tile in pool order
    sub = np.random.default_rng(7).choice(N, 512, replace=False)
    check_assignment(otl, banks["tpl"], pool[:, sub], tile_of[sub], np.array(
        [otl.match(pool[0, i], pool[1, i], *banks["tpl"][:, tile_of[i]]) for i in sub], dtype=np.float32))
    ll_tpl = torch.empty(T, dtype=torch.float64, device="cuda")
    m.mbis_loglike(ctx, T, dev(torch, banks["phys"]), ll_tpl)
    m.mbis_tiling_set_loglike(gtl, ll_tpl)
    n = 1 << 18
    theta = torch.empty((2, n), dtype=torch.float64, device="cuda")
    coords = torch.empty((2, n), dtype=torch.float64, device="cuda")
    lq, lp, ll, wt = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(4))
    m.mbis_tiling_draw(gtl, demo.draw_seed, 0, n, theta, lq, lp, coords=coords)
    m.mbis_loglike(ctx, n, theta, ll)
    s = m.mbis_reduce(ctx, n, ll, lp, lq, wt)
    torch.cuda.synchronize()
    x, q, wts = coords[0].cpu().numpy(), coords[1].cpu().numpy(), wt.cpu().numpy()
    low = x < demo.mc_base
    assert abs(wts[low].sum() - 0.5) < 0.02
    for a in (low, ~low):
        for b in (q < 1.0, q >= 1.0):
            assert wts[a & b].sum() > 0.01
    # the same estimate from a second batch of draws agrees within its Monte-Carlo error
    m.mbis_tiling_draw(gtl, demo.draw_seed, n, n, theta, lq, lp, coords=coords)
    m.mbis_loglike(ctx, n, theta, ll)
    s2 = m.mbis_reduce(ctx, n, ll, lp, lq)
    assert abs(s2["log_z"] - s["log_z"]) < 5.0 / math.sqrt(s["ess"])
    print(f"full pool: {T} tiles, ESS {s['ess']:.0f} of {n} ({100 * s['ess'] / n:.1f}%), log Z {s['log_z']:.4f}, "
          f"weight below Mc period boundary {wts[low].sum():.3f}, q < 1: {wts[q < 1].sum():.3f}")


def test_state_and_argument_errors(m, torch, demo, psd):
    w = demo.workload
    t = m.mbis_tiling_create(w.f_lo, w.df, w.n_bins, psd, demo.x_lo, demo.x_hi, demo.mc_period, demo.mc_base,
                             demo.q_lo, demo.q_hi)
    try:
        pts = dev(torch, [[21.0], [3.5]])
        out = torch.empty(1, dtype=torch.int32, device="cuda")
        with pytest.raises(m.MbisError):
            m.mbis_tiling_assign(t, 1, pts, out)          # no bank
        with pytest.raises(m.MbisError):
            m.mbis_tiling_bank(t, [[30.0], [2.0]], 0.99, 10, 10)   # candidate outside the space
        with pytest.raises(m.MbisError):
            m.mbis_tiling_bank(t, [[21.0], [2.0]], 1.5, 10, 10)    # minimal match out of range
        m.mbis_tiling_bank(t, [[21.0, 25.0], [3.5, 1 / 3.5]], 0.99, 10, 10)
        assert m.mbis_tiling_templates(t)[0].shape == (2, 1)       # the image is not a second template
        th = torch.empty((2, 4), dtype=torch.float64, device="cuda")
        lq, lp = torch.empty(4, dtype=torch.float64, device="cuda"), torch.empty(4, dtype=torch.float64, device="cuda")
        with pytest.raises(m.MbisError):
            m.mbis_tiling_draw(t, 1, 0, 4, th, lq, lp)   # no mixture
        m.mbis_tiling_set_pool(t, 1, pts)
        with pytest.raises(m.MbisError):
            m.mbis_tiling_set_loglike(t, dev(torch, [-math.inf]))  # nothing to draw
    finally:
        m.mbis_tiling_destroy(t)
    with pytest.raises(m.MbisError):
        m.mbis_tiling_create(w.f_lo, w.df, w.n_bins, psd, 20.0, 28.0, 4.0, 24.0, 0.0, 6.0)  # q_lo = 0
