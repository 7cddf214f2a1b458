"""The pSGLD sampler (Eq. pSGLD) and the stage-1 optimiser (L1 objective +
Adam, Sec. 3.2) on the GPU vs the FP64 oracle through the C ABI: chains with
identical Philox streams compared in metres after K steps, the L1 gradient,
and exact resume of the moment state."""
import numpy as np
import pytest

from oracle import spider_oracle as O
from paper_2508_12117_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def cat1():
    return synth.make_catalog(1)


def test_psgld_chain_matches_oracle(cat1):
    eps, b2, pe = 2e-5, 0.99, 1e-5       # ~eps km per step along the gradient
    seeds = [7000 + t for t in range(300)]
    ctx = binding.Context.from_catalog(cat1, update=binding.UPDATE_PSGLD, beta2=b2, upd_eps=pe)
    for s in seeds:
        ctx.spider_sgld_step(eps, s)
    th, step = ctx.spider_get_state()
    _, v = ctx.spider_get_moments()
    P = O.problem_from_catalog(cat1)
    to, _, vo = O.run_updates(P, cat1.init_xyzt, eps, seeds, update="psgld", beta2=b2, eps_p=pe)
    dx_m = np.abs(th[:, :3] - to[:, :3]).max() * 1e3
    dt_ms = np.abs(th[:, 3] - to[:, 3]).max() * 1e3
    moved = np.abs(to[:, :3] - cat1.init_xyzt[:, :3]).max() * 1e3
    print(f"pSGLD, {len(seeds)} steps: max |dx| {dx_m:.4f} m (chain moved up to {moved:.1f} m), "
          f"max |dt0| {dt_ms:.5f} ms, v rel-L2 {rel_l2(v, vo):.2e}")
    assert step == len(seeds)
    assert dx_m <= 1.0
    assert rel_l2(v, vo) <= 1e-3
    ctx.close()


def test_l1_gradient_matches_oracle(cat1):
    P = O.problem_from_catalog(cat1)
    rng = np.random.default_rng(3)
    theta = cat1.init_xyzt + np.c_[rng.normal(0, 0.05, (cat1.M, 3)), rng.normal(0, 0.01, cat1.M)]
    ctx = binding.Context.from_catalog(cat1, loss=binding.LOSS_L1)
    ctx.spider_set_state(theta, 0)
    g, lp = ctx.spider_grad_logpost(0)
    L, go, info = O.log_posterior(P, theta, loss="l1")
    # a residual within FP32 rounding of 0 may take the other sign; count them
    near0 = int((np.abs(info["r"]) < 1e-6).sum())
    rel = rel_l2(g, go)
    print(f"L1 full batch: gradient rel-L2 {rel:.3e} (residuals within 1 us of 0: {near0}), "
          f"logpost {lp:.8e} vs {L:.8e}")
    assert rel <= 1e-5 + 1e-3 * near0
    assert abs(lp - L) <= 1e-6 * abs(L)
    ctx.close()


def test_adam_l1_stage1_matches_oracle(cat1):
    eta = 1e-3
    seeds = [9000 + t for t in range(200)]
    ctx = binding.Context.from_catalog(cat1, update=binding.UPDATE_ADAM, loss=binding.LOSS_L1,
                                       beta1=0.9, beta2=0.99, upd_eps=1e-5)
    for s in seeds:
        ctx.spider_sgld_step(eta, s)
    th, _ = ctx.spider_get_state()
    P = O.problem_from_catalog(cat1)
    to, mo, vo = O.run_updates(P, cat1.init_xyzt, eta, seeds, update="adam", loss="l1",
                               beta1=0.9, beta2=0.99, eps_p=1e-5)
    dx_m = np.abs(th[:, :3] - to[:, :3]).max() * 1e3
    moved = np.abs(to[:, :3] - cat1.init_xyzt[:, :3]).max() * 1e3
    # the L1 objective decreases along the run (stage 1 is an optimiser)
    r0 = np.abs(O.residuals(P, cat1.init_xyzt, np.arange(P.N))[0]).sum()
    r1 = np.abs(O.residuals(P, th, np.arange(P.N))[0]).sum()
    print(f"Adam + L1, {len(seeds)} steps: max |dx| {dx_m:.4f} m (moved up to {moved:.1f} m), "
          f"sum|r| {r0:.3f} -> {r1:.3f} s")
    assert dx_m <= 1.0
    assert r1 < r0
    ctx.close()


def test_moments_resume_exactly(cat1):
    eps = 1e-3
    a = binding.Context.from_catalog(cat1, update=binding.UPDATE_PSGLD)
    for s in range(1, 6):
        a.spider_sgld_step(eps, s)
    th, step = a.spider_get_state()
    m, v = a.spider_get_moments()
    for s in range(6, 11):
        a.spider_sgld_step(eps, s)
    ta, _ = a.spider_get_state()
    b = binding.Context.from_catalog(cat1, update=binding.UPDATE_PSGLD)
    b.spider_set_state(th, step)
    b.spider_set_moments(m, v)
    for s in range(6, 11):
        b.spider_sgld_step(eps, s)
    tb, _ = b.spider_get_state()
    assert np.array_equal(ta, tb)
    a.close()
    b.close()


def test_sgld_keeps_no_moments(cat1):
    ctx = binding.Context.from_catalog(cat1)
    with pytest.raises(binding.SpiderError):
        ctx.spider_get_moments()
    ctx.close()


def test_update_config_is_validated(cat1):
    for bad in (dict(update=7), dict(loss=3), dict(beta2=1.0), dict(beta1=-0.1), dict(upd_eps=0.0)):
        with pytest.raises(binding.SpiderError):
            binding.Context.from_catalog(cat1, **bad)


def test_stage1_outlier_mask_matches_oracle():
    # Laplace(0, 5 ms) noise + 2 % U(-0.5, 0.5) s outliers (the 100k-event recipe, scaled)
    s = synth.scaled_spec(3, 4000, batch_n=1 << 16)
    cat = synth.make_catalog(s)
    ctx = binding.Context.from_catalog(cat, update=binding.UPDATE_ADAM, loss=binding.LOSS_L1)
    for t in range(20):
        ctx.spider_sgld_step(1e-3, 300 + t)
    th, _ = ctx.spider_get_state()
    keep, med, mad = ctx.spider_outlier_mask(4.0)
    P = O.problem_from_catalog(cat)
    r_caller = O.residuals(P, th, np.arange(P.N))[0]      # caller's observation order
    ko, mo, ao = O.mad_filter(r_caller, 4.0)
    near = np.abs(np.abs(r_caller - mo) - 4.0 * ao) < 1e-5
    diff = keep != ko
    print(f"stage-1 mask: N {P.N}, kept {keep.sum()} (oracle {ko.sum()}), median {med[0]*1e3:.4f} ms "
          f"(oracle {mo*1e3:.4f}), MAD {mad[0]*1e3:.4f} ms (oracle {ao*1e3:.4f}), "
          f"differing {diff.sum()} all near the cut: {bool((~near[diff]).sum() == 0)}")
    assert abs(med[0] - mo) <= 2e-6 and abs(mad[0] - ao) <= 2e-6
    assert not diff[~near].any()
    # the next stage runs on the kept observations
    nxt = binding.Context(th, cat.i[keep], cat.j[keep], cat.k[keep], cat.dt[keep], cat.stations,
                          binding.net_for_catalog(cat),
                          binding.config_for_catalog(cat, update=binding.UPDATE_PSGLD))
    nxt.spider_sgld_step(2e-5, 1)
    nxt.spider_sync()
    nxt.close()
    ctx.close()


@pytest.mark.parametrize("wid", [1, 2])
def test_linearisation_mask_matches_oracle(wid):
    cat = synth.make_catalog(wid)
    ctx = binding.Context.from_catalog(cat)
    rng = np.random.default_rng(wid)
    theta = cat.init_xyzt + np.c_[rng.normal(0, 0.1, (cat.M, 3)), np.zeros(cat.M)]
    ctx.spider_set_state(theta, 0)
    keep = ctx.spider_linearisation_mask(0.05)
    P = O.problem_from_catalog(cat)
    ko, rel = O.linearisation_filter(P, theta, 0.05)
    st = P.stations[P.k]
    dT = np.abs(P.model(theta[P.j, :3], st)[0] - P.model(theta[P.i, :3], st)[0])
    near = np.abs(rel * dT - 0.05 * dT) <= 3e-6          # within the FP32 travel-time accuracy of the cut
    diff = keep != ko
    print(f"workload {wid}: kept {keep.sum()} of {P.N} (oracle {ko.sum()}), differing {diff.sum()}, "
          f"all near the cut: {bool(not diff[~near].any())}")
    assert not diff[~near].any()
    ctx.close()


def test_uq_summaries_match_oracle(cat1):
    eps = cat1.spec.hyper.eps
    ctx = binding.Context.from_catalog(cat1, thin=2, sample_cap=300)
    for t in range(600):
        ctx.spider_sgld_step(eps, 40_000 + t)
    samples = ctx.spider_samples(300)
    uq = ctx.spider_uq(cat1.true_xyzt, 0.5, 99.5)
    med, half, calib, ess = O.uq_stats(samples, cat1.true_xyzt, 0.5, 99.5)
    print(f"UQ over {samples.shape[0]} samples: median |d| {np.abs(uq['median'] - med).max():.2e} km, "
          f"half-width |d| {np.abs(uq['halfwidth'] - half).max():.2e} km, ESS rel "
          f"{np.abs(uq['ess'] / ess - 1).max():.2e}, mean half-width x {half[:, 0].mean() * 1e3:.1f} m, "
          f"median ESS {np.median(ess):.1f}")
    assert np.abs(uq["median"] - med).max() <= 1e-9
    assert np.abs(uq["halfwidth"] - half).max() <= 1e-9
    assert np.array_equal(uq["calib"], calib)
    assert np.abs(uq["ess"] / ess - 1).max() <= 1e-9
    nt = ctx.spider_uq(None)
    assert np.isnan(nt["calib"]).all()
    ctx.close()


def test_noise_ramp_matches_oracle(cat1):
    # stage 2 (noise off) then stage 3 (linear ramp to full amplitude), pSGLD
    eps = 2e-5
    ctx = binding.Context.from_catalog(cat1, update=binding.UPDATE_PSGLD)
    P = O.problem_from_catalog(cat1)
    theta, m, v = cat1.init_xyzt, None, None
    schedule = [0.0] * 20 + [k / 20 for k in range(1, 21)]
    for t, ns in enumerate(schedule):
        ctx.spider_set_noise_scale(ns)
        ctx.spider_sgld_step(eps, 60_000 + t)
        theta, m, v = O.run_updates(P, theta, eps, [60_000 + t], update="psgld", noise_scale=ns,
                                    m0=m, v0=v, t0=t)
    th, _ = ctx.spider_get_state()
    dx_m = np.abs(th[:, :3] - theta[:, :3]).max() * 1e3
    print(f"noise ramp, {len(schedule)} steps: max |dx| {dx_m:.4f} m")
    assert dx_m <= 1.0
    with pytest.raises(binding.SpiderError):
        ctx.spider_set_noise_scale(-1.0)
    ctx.close()
