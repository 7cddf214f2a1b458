"""FP8 tensor-core form (E4M3 hidden-layer operands with per-column weight
scales and per-row activation scales, FP32 accumulation, FP32 everything
else) vs the FP64 oracle.

Gates (a numpy emulation of the E4M3 operand rounding and scaling gives the
figures in brackets on these nets; a wrong or missing reverse sweep gives ~1):
  * network part of the Jacobian, r dtau/dx, rel-L2 <= 0.25 [0.04-0.15];
  * T within 20 % of the largest network part of T [5-12 %];
  * the gradient, rel-L2 <= 3e-2, on the configured network and on a network
    whose learned part is about a fifth of dT/dx [1.4e-2];
  * positions after 300 SGLD steps on the 10k-event MLP workload: printed,
    and within 10 m of the oracle's chain.
"""
import numpy as np
import pytest

from mlp_gates import measure, random_pairs, rel_l2, with_net
from oracle import spider_oracle as O
from paper_2508_12117_gb300 import binding, synth

pytestmark = pytest.mark.gpu

GRAD_TOL_FP8 = 3e-2
JNET_TOL_FP8 = 0.25
T_FRAC_FP8 = 0.20


def _nets(H):
    return {"config": synth.mlp_weights(H, 777 + H), "strong": synth.strong_mlp_weights(H, 778 + H)}


@pytest.mark.parametrize("H", [128, 256])
@pytest.mark.parametrize("kind", ["config", "strong"])
def test_tt_mlp_fp8_vs_oracle(H, kind):
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    src, rcv = random_pairs(3 * 128 * 152 + 77, H + 1)  # several tiles per CTA, ragged tail
    m = measure(torch, _nets(H)[kind], binding.FP8, src, rcv)
    print(f"FP8 H={H} {kind}: max|dT| {m['err_t_max']*1e6:.2f} us of network part max "
          f"{m['net_t_max']*1e3:.3f} ms; J rel-L2 {m['rel_j']:.2e}; network part of J "
          f"(share {m['jnet_share']:.2e}) rel-L2 {m['rel_jnet']:.2e}")
    assert m["err_t_max"] <= T_FRAC_FP8 * m["net_t_max"] + 2e-6
    assert m["rel_jnet"] <= JNET_TOL_FP8
    assert m["rel_j"] <= 0.1


def test_fp8_rejects_width_64():
    net = synth.mlp_weights(64, 5)
    with pytest.raises(Exception):
        binding.NetDevice(binding.Net(binding.TT_MLP, mlp=net), precision=binding.FP8)


@pytest.mark.parametrize("kind", ["config", "strong"])
def test_fp8_gradient_full_batch_mlp128(kind):
    cat = synth.make_catalog(2)
    if kind == "strong":
        cat = with_net(cat, synth.strong_mlp_weights(128, 9128))
    ctx = binding.Context.from_catalog(cat, precision=binding.FP8)
    g, lp = ctx.spider_grad_logpost(0)
    ctx.close()
    P = O.problem_from_catalog(cat)
    L, go, _ = O.log_posterior(P, cat.init_xyzt)
    rel = rel_l2(g, go)
    print(f"FP8 H=128 {kind} full batch: gradient rel-L2 {rel:.3e}, logpost {lp:.8e} vs {L:.8e}")
    assert rel <= GRAD_TOL_FP8


@pytest.mark.parametrize("kind", ["config", "strong"])
def test_fp8_gradient_minibatch_mlp256(kind):
    s = synth.scaled_spec(3, 20000, batch_n=1 << 17)
    cat = synth.make_catalog(s)
    if kind == "strong":
        cat = with_net(cat, synth.strong_mlp_weights(256, 9256))
    ctx = binding.Context.from_catalog(cat, precision=binding.FP8)
    g, lp = ctx.spider_grad_logpost(7)
    ctx.close()
    P = O.problem_from_catalog(cat)
    sel = P.batch(7)
    L, go, _ = O.log_posterior(P, cat.init_xyzt, sel)
    rel = rel_l2(g, go)
    print(f"FP8 H=256 {kind} minibatch: gradient rel-L2 {rel:.3e}")
    assert rel <= GRAD_TOL_FP8


def test_fp8_chain_300_steps_10k_events():
    cat = synth.make_catalog(2)
    bn = 1 << 14
    eps = synth._eps_for(cat.spec.hyper.kappa, cat.spec.n_obs_stations, cat.N / bn)
    seeds = [51_000 + t for t in range(300)]
    ctx = binding.Context.from_catalog(cat, precision=binding.FP8, batch_n=bn)
    for s in seeds:
        ctx.spider_sgld_step(eps, s)
    th, _ = ctx.spider_get_state()
    ctx.close()
    P = O.problem_from_catalog(cat, batch_n=bn)
    to, _ = O.run_chain(P, cat.init_xyzt, eps, seeds)
    dx_m = np.abs(th[:, :3] - to[:, :3]).max() * 1e3
    print(f"FP8 chain, 300 steps, 10k events: max |dx| {dx_m:.4f} m")
    assert dx_m <= 10.0
