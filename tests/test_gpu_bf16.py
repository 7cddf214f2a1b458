"""BF16 tensor-core form (tcgen05 hidden layers, FP32 everything else) vs the
FP64 oracle.

Gates, each on a quantity the reverse sweep decides:
  * the network part of the Jacobian, r dtau/dx, rel-L2 <= 1.5e-2 (a numpy
    emulation of the BF16 operand rounding gives 2.7e-3 to 5e-3 on these nets;
    a wrong or missing sweep gives ~1);
  * T within 2 % of the largest network part of T (emulation: 0.5 %);
  * the gradient, rel-L2 <= 5e-3 (the stated BF16 tolerance), on the
    configured network and on a network whose learned part is about a fifth
    of dT/dx (emulation: 1.2e-3), where a broken sweep moves the gradient by
    far more than the tolerance;
  * positions after 1000 SGLD steps on the 10k-event MLP workload within 10 m
    of the oracle's chain, with identical Philox streams and minibatches.
"""
import numpy as np
import pytest

from mlp_gates import measure, random_pairs, rel_l2, with_net
from oracle import spider_oracle as O
from paper_2508_12117_gb300 import binding, synth

pytestmark = pytest.mark.gpu

GRAD_TOL_BF16 = 5e-3
JNET_TOL_BF16 = 1.5e-2
T_FRAC_BF16 = 0.02


def _nets(H):
    return {"config": synth.mlp_weights(H, 555 + H), "strong": synth.strong_mlp_weights(H, 556 + H)}


@pytest.mark.parametrize("H", [64, 128, 256])
@pytest.mark.parametrize("kind", ["config", "strong"])
def test_tt_mlp_bf16_vs_oracle(H, kind):
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    src, rcv = random_pairs(3 * 128 * 152 + 77, H)     # several tiles per CTA, ragged tail
    m = measure(torch, _nets(H)[kind], binding.BF16, src, rcv)
    print(f"BF16 H={H} {kind}: max|dT| {m['err_t_max']*1e6:.2f} us of network part max "
          f"{m['net_t_max']*1e3:.3f} ms; J rel-L2 {m['rel_j']:.2e}; network part of J "
          f"(share {m['jnet_share']:.2e}) rel-L2 {m['rel_jnet']:.2e}")
    assert m["err_t_max"] <= T_FRAC_BF16 * m["net_t_max"] + 2e-6
    assert m["rel_jnet"] <= JNET_TOL_BF16
    assert m["rel_j"] <= 2e-2


@pytest.mark.parametrize("kind", ["config", "strong"])
def test_bf16_gradient_full_batch_mlp128(kind):
    cat = synth.make_catalog(2)
    if kind == "strong":
        cat = with_net(cat, synth.strong_mlp_weights(128, 9128))
    ctx = binding.Context.from_catalog(cat, precision=binding.BF16)
    g, lp = ctx.spider_grad_logpost(0)
    ctx.close()
    P = O.problem_from_catalog(cat)
    L, go, _ = O.log_posterior(P, cat.init_xyzt)
    rel = rel_l2(g, go)
    print(f"BF16 H=128 {kind} full batch: gradient rel-L2 {rel:.3e}, logpost {lp:.8e} vs {L:.8e}")
    assert rel <= GRAD_TOL_BF16


@pytest.mark.parametrize("kind", ["config", "strong"])
def test_bf16_gradient_minibatch_mlp256(kind):
    s = synth.scaled_spec(3, 20000, batch_n=1 << 17)
    cat = synth.make_catalog(s)
    if kind == "strong":
        cat = with_net(cat, synth.strong_mlp_weights(256, 9256))
    ctx = binding.Context.from_catalog(cat, precision=binding.BF16)
    g, lp = ctx.spider_grad_logpost(7)
    ctx.close()
    P = O.problem_from_catalog(cat)
    sel = P.batch(7)
    L, go, _ = O.log_posterior(P, cat.init_xyzt, sel)
    rel = rel_l2(g, go)
    print(f"BF16 H=256 {kind} minibatch: gradient rel-L2 {rel:.3e}")
    assert rel <= GRAD_TOL_BF16


def _chain(cat, precision, eps, seeds, bn):
    ctx = binding.Context.from_catalog(cat, precision=precision, batch_n=bn)
    for s in seeds:
        ctx.spider_sgld_step(eps, s)
    th, step = ctx.spider_get_state()
    ctx.close()
    assert step == len(seeds)
    return th


def test_bf16_chain_1000_steps_10k_events():
    """1000 SGLD steps of the 10k-event MLP workload (minibatches of 2^14
    observations, the step size of the workload's recipe for that N/n) in BF16
    against the oracle's chain in FP64: positions within 10 m."""
    cat = synth.make_catalog(2)
    bn = 1 << 14
    eps = synth._eps_for(cat.spec.hyper.kappa, cat.spec.n_obs_stations, cat.N / bn)
    seeds = [31_000 + t for t in range(1000)]
    th = _chain(cat, binding.BF16, eps, seeds, bn)
    P = O.problem_from_catalog(cat, batch_n=bn)
    to, _ = O.run_chain(P, cat.init_xyzt, eps, seeds)
    dx_m = np.abs(th[:, :3] - to[:, :3]).max() * 1e3
    dt_ms = np.abs(th[:, 3] - to[:, 3]).max() * 1e3
    moved_m = np.abs(to[:, :3] - cat.init_xyzt[:, :3]).max() * 1e3
    print(f"BF16 chain, 1000 steps, 10k events: max |dx| {dx_m:.4f} m, max |dt0| {dt_ms:.5f} ms "
          f"(oracle chain moved up to {moved_m:.1f} m)")
    assert dx_m <= 10.0


def test_bf16_chain_strong_network():
    """300 steps of the same workload with the strong network (BF16 rounding
    is a sizeable part of each gradient's error budget): positions within 10 m."""
    cat = with_net(synth.make_catalog(2), synth.strong_mlp_weights(128, 9128))
    bn = 1 << 14
    eps = synth._eps_for(cat.spec.hyper.kappa, cat.spec.n_obs_stations, cat.N / bn)
    seeds = [41_000 + t for t in range(300)]
    th = _chain(cat, binding.BF16, eps, seeds, bn)
    P = O.problem_from_catalog(cat, batch_n=bn)
    to, _ = O.run_chain(P, cat.init_xyzt, eps, seeds)
    dx_m = np.abs(th[:, :3] - to[:, :3]).max() * 1e3
    moved_m = np.abs(to[:, :3] - cat.init_xyzt[:, :3]).max() * 1e3
    print(f"BF16 chain, strong network, 300 steps: max |dx| {dx_m:.4f} m "
          f"(oracle chain moved up to {moved_m:.1f} m)")
    assert dx_m <= 10.0
