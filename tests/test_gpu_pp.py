"""P-P self-consistency (Sec. III A) through the C ABI: the device credible levels against
the oracle, and a population of the two-parameter demonstration analysed with the tiled
proposal whose levels of the true (x, q) are uniform."""
import math

import numpy as np
import pytest

import oracle
import workloads
from gpu_common import m, torch  # noqa: F401

pytestmark = pytest.mark.gpu


def test_credible_levels_equal_the_oracle(m, torch):
    rng = np.random.default_rng(3)
    n, P = 100003, 5
    theta = rng.normal(size=(P, n))
    theta[2, :1000] = 0.25                      # ties with the reference
    w = rng.exponential(size=n) * 1e-30
    w[::97] = 0.0                               # zero weights are skipped
    ref = np.array([0.1, -0.5, 0.25, 1.7, -3.0])
    want = oracle.credible_levels(theta, w, ref)
    out = torch.empty(P, dtype=torch.float64, device="cuda")
    m.mbis_credible_levels(n, torch.tensor(theta, device="cuda"), torch.tensor(w, device="cuda"), ref, out)
    assert np.abs(out.cpu().numpy() - want).max() <= 1e-12
    with pytest.raises(m.MbisError):
        m.mbis_credible_levels(0, torch.tensor(theta, device="cuda"), torch.tensor(w, device="cuda"), ref, out)


@pytest.fixture(scope="module")
def tiled(m, torch):
    from paper_2410_05190_gb300 import pp
    d = workloads.tiled_demo()
    w = d.workload
    psd = oracle.psd_aligo(w.f_lo + w.df * np.arange(w.n_bins))
    t = m.mbis_tiling_create(w.f_lo, w.df, w.n_bins, psd, d.x_lo, d.x_hi, d.mc_period, d.mc_base, d.q_lo, d.q_hi)
    cand = workloads.uniform_points(d.n_candidates, d.x_lo, d.x_hi, d.q_lo, d.q_hi, d.candidate_seed)
    m.mbis_tiling_bank(t, cand, d.min_match, d.stop_after, d.max_templates)
    _, phys, _ = m.mbis_tiling_templates(t)
    pool = workloads.uniform_points(1 << 20, d.x_lo, d.x_hi, d.q_lo, d.q_hi, d.pool_seed)
    m.mbis_tiling_set_pool(t, pool.shape[1], torch.tensor(pool, device="cuda"))
    q_max = max(d.q_hi, 1 / d.q_lo)
    an = pp.TiledAnalysis(m, torch, t, phys, (d.mc_base, d.mc_base + d.mc_period), (1.0, q_max), 1 << 15)
    yield d, psd, an
    m.mbis_tiling_destroy(t)


def test_tiled_population_is_self_consistent(m, torch, tiled):
    from oracle.events import make_event
    from paper_2410_05190_gb300 import pp
    d, psd, an = tiled
    w = d.workload
    spec = w.events[0]
    _, th0, dl = make_event(w, spec, noise=False)          # the common distance: SNR 15 at the demo source
    v, x, y = workloads.network(w.detectors)
    ev = oracle.OracleEvent(w.f_lo, w.df, w.n_bins, np.tile(psd, (2, 1)), v, x, y, gmst=spec.gmst, marg=w.marg)
    dets = m.make_detectors(v, x, y)
    pop = workloads.tiled_population(d, 96)
    lv, eff = [], []
    for src in pop:
        th = th0.copy()
        th[workloads.MC] = d.mc_base + math.fmod(src["x"], d.mc_period)
        th[workloads.Q] = max(src["q"], 1.0 / src["q"])
        th[workloads.PHIC] = src["phic"]
        th[workloads.DL] = dl
        s = oracle.make_strain(ev, th, src["noise_seed"], True)
        strain = (s[..., 0] + 1j * s[..., 1]).astype(np.complex64)
        levels, summ = an.run(strain, np.tile(psd, (2, 1)), dets, w.f_lo, w.df, th, spec.gmst,
                              [src["x"], src["q"]], src["draw_seed"])
        lv.append(levels)
        eff.append(summ["ess"] / an.n)
    lv = np.array(lv)
    p_x, p_q = pp.ks_pvalue(lv[:, 0]), pp.ks_pvalue(lv[:, 1])
    comb = pp.combined_pvalue([p_x, p_q])
    print(f"P-P over {len(pop)} sources: KS p(x) = {p_x:.3f}, p(q) = {p_q:.3f}, combined {comb:.3f}; "
          f"median efficiency {np.median(eff):.3f}")
    assert min(p_x, p_q, comb) > 1e-3
    assert np.median(eff) > 0.1
