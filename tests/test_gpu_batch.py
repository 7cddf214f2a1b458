"""Many catalogs x chains in one context (one launch per kernel, one CUDA graph
per SGLD step) reproduce independent single-catalog samplers and the oracle."""
import numpy as np
import pytest

from oracle import spider_oracle as O
from paper_2508_12117_gb300 import binding, synth

pytestmark = pytest.mark.gpu
GOLDEN = 0x9E3779B97F4A7C15


@pytest.fixture(scope="module")
def cats():
    a = synth.make_catalog(1)
    b = synth.make_catalog(synth.scaled_spec(2, 700, n_faults=1, region_km=6.0, n_stations=12))
    b.spec.forward = "homogeneous"      # one network for the whole batch
    return [a, b]


def test_batch_full_batch_matches_single_contexts(cats):
    chains = 2
    net = binding.Net(binding.TT_HOMOGENEOUS, v0=6.0)
    cfg = binding.make_config(sigma=0.01, kappa=0.03, thin=1, sample_cap=4)
    bat = binding.Context.batch(cats, chains, net, cfg)
    g_b, lp_b = bat.spider_grad_logpost(0)
    singles, off, lp_sum = [], 0, 0.0
    for ci, cat in enumerate(cats):
        for h in range(chains):
            ctx = binding.Context(cat.init_xyzt, cat.i, cat.j, cat.k, cat.dt, cat.stations, net,
                                  binding.make_config(sigma=0.01, kappa=0.03, chain=h, catalog=ci,
                                                      thin=1, sample_cap=4))
            g, lp = ctx.spider_grad_logpost(0)
            assert np.array_equal(g_b[off:off + cat.M], g)          # bit for bit
            lp_sum += lp
            singles.append((ctx, off, cat))
            off += cat.M
    assert abs(lp_b - lp_sum) <= 1e-9 * abs(lp_sum)
    # SGLD in full batch: only the noise depends on the seed -> identical chains
    for s in range(1, 6):
        bat.spider_sgld_step(1e-4, s)
        for ctx, _, _ in singles:
            ctx.spider_sgld_step(1e-4, s)
    th_b, step = bat.spider_get_state()
    assert step == 5
    for ctx, off, cat in singles:
        th, _ = ctx.spider_get_state()
        assert np.array_equal(th_b[off:off + cat.M], th)
        ctx.close()
    bat.close()


def test_batch_minibatch_matches_oracle(cats):
    chains = 2
    net = binding.Net(binding.TT_HOMOGENEOUS, v0=6.0)
    B, bn = 512, 1500
    cfg = binding.make_config(sigma=0.01, kappa=0.03, batch_n=bn, block_obs=B)
    bat = binding.Context.batch(cats, chains, net, cfg)
    eps, seeds = 1e-5, [77, 78, 79]
    for s in seeds:
        bat.spider_sgld_step(eps, s)
    th_b, _ = bat.spider_get_state()
    off, sub = 0, 0
    for ci, cat in enumerate(cats):
        for h in range(chains):
            P = O.problem_from_catalog(cat, batch_n=bn, model=O.Model("homogeneous", v0=6.0))
            P.block_obs = B
            P.sigma = 0.01
            th = cat.init_xyzt.copy()
            for s in seeds:
                key = (s ^ ((GOLDEN * sub) & 0xFFFFFFFFFFFFFFFF)) & 0xFFFFFFFFFFFFFFFF
                sel = np.sort(O.minibatch_obs(P.order, B, O.select_blocks(P.N, B, bn, key)))
                _, g, _ = O.log_posterior(P, th, sel)
                th = O.sgld_update(th, g, eps, O.langevin_noise(P.M, s, chain=h, catalog=ci))
            dx = np.abs(th_b[off:off + cat.M, :3] - th[:, :3]).max() * 1e3
            print(f"catalog {ci} chain {h}: max |dx| after {len(seeds)} minibatch steps {dx:.4f} m")
            assert dx <= 0.05
            off += cat.M
            sub += 1
    bat.close()


def test_batch_minibatch_matches_single_contexts(cats):
    # sub-problem s of the batch draws its blocks with key seed ^ (s * golden): a
    # single context stepped with that key walks the identical chain, bit for bit
    # (noise off: the batch keys its noise with the untransformed seed)
    chains = 2
    net = binding.Net(binding.TT_HOMOGENEOUS, v0=6.0)
    B, bn = 512, 1500
    cfg = binding.make_config(sigma=0.01, kappa=0.03, batch_n=bn, block_obs=B, thin=1, sample_cap=1,
                              noise_scale=0.0)
    bat = binding.Context.batch(cats, chains, net, cfg)
    seeds = [31, 32, 33, 34]
    for s in seeds:
        bat.spider_sgld_step(1e-5, s)
    th_b, _ = bat.spider_get_state()
    off, sub = 0, 0
    for ci, cat in enumerate(cats):
        for h in range(chains):
            ctx = binding.Context(cat.init_xyzt, cat.i, cat.j, cat.k, cat.dt, cat.stations, net,
                                  binding.make_config(sigma=0.01, kappa=0.03, batch_n=bn, block_obs=B,
                                                      chain=h, catalog=ci, thin=1, sample_cap=1,
                                                      noise_scale=0.0))
            for s in seeds:
                ctx.spider_sgld_step(1e-5, (s ^ ((GOLDEN * sub) & 0xFFFFFFFFFFFFFFFF)) & 0xFFFFFFFFFFFFFFFF)
            th, _ = ctx.spider_get_state()
            assert np.array_equal(th_b[off:off + cat.M], th), (ci, h)
            ctx.close()
            off += cat.M
            sub += 1
    bat.close()


def test_batched_mlp_workload_stays_finite():
    # the 16-catalog x 4-chain workload with the BF16 network: 25 steps stay finite
    # and every sub-problem moves by less than the prior width allows
    specs = synth.batch_specs(16)
    cats16 = [synth.make_catalog(s) for s in specs]
    h = specs[0].hyper
    net = binding.Net(binding.TT_MLP, mlp=synth.batch_network())
    cfg = binding.make_config(sigma=h.sigma, kappa=h.kappa, p=h.p, ell=h.ell, eps_w=h.eps_w,
                              sig_e=h.sig_e, sig_c=h.sig_c, batch_n=h.batch_n, block_obs=h.block_obs,
                              precision=binding.BF16, thin=1, sample_cap=1)
    bat = binding.Context.batch(cats16, 4, net, cfg)
    th0, _ = bat.spider_get_state()
    for s in range(25):
        bat.spider_sgld_step(h.eps, 100 + s)
    th, _ = bat.spider_get_state()
    move = np.abs(th - th0)[:, :3].max()
    print(f"batched workload, 25 steps: max move {move:.3f} km")
    assert np.isfinite(th).all() and move < 10.0
    bat.close()


def test_batched_bf16_mlp_gradient_matches_oracle_per_subproblem():
    """Three catalogs of uneven sizes drawn with the batched recipe, two chains
    each, one BF16 tensor-core network (6 -> 4 x 128, strong network part): the
    full-batch gradient of every sub-problem, read from the batched context,
    against the FP64 oracle on that catalog alone (BF16 gradient bound 5e-3
    rel-L2)."""
    specs = [synth.scaled_spec(2, m, n_faults=1, region_km=8.0, n_stations=s, hidden=128)
             for m, s in ((600, 14), (1500, 20), (3000, 30))]
    cats3 = [synth.make_catalog(s) for s in specs]
    net_w = synth.strong_mlp_weights(128, 5)
    net = binding.Net(binding.TT_MLP, mlp=net_w)
    h = specs[0].hyper
    cfg = binding.make_config(sigma=h.sigma, kappa=h.kappa, p=h.p, ell=h.ell, eps_w=h.eps_w,
                              sig_e=h.sig_e, sig_c=h.sig_c, block_obs=h.block_obs,
                              precision=binding.BF16)
    chains = 2
    bat = binding.Context.batch(cats3, chains, net, cfg)
    g_b, _ = bat.spider_grad_logpost(0)
    off = 0
    for ci, cat in enumerate(cats3):
        P = O.problem_from_catalog(cat, batch_n=0, model=O.Model("mlp", net=net_w))
        _, go, _ = O.log_posterior(P, cat.init_xyzt, None)
        for ch in range(chains):
            g = g_b[off:off + cat.M]
            rel = float(np.linalg.norm(g - go) / np.linalg.norm(go))
            print(f"catalog {ci} ({cat.M} events) chain {ch}: BF16 gradient rel-L2 {rel:.2e}")
            assert rel <= 5e-3
            off += cat.M
    bat.close()
