"""FP8 tensor-core form (E4M3 hidden-layer operands with per-column weight
scales and per-row activation scales, FP32 accumulation, FP32 everything
else) vs the FP64 oracle.  The gate on the gradient is rel-L2 <= 3e-2; the
travel-time and Jacobian errors are measured, printed and bounded."""
import numpy as np
import pytest

from oracle import spider_oracle as O
from paper_2508_12117_gb300 import binding, synth

pytestmark = pytest.mark.gpu

GRAD_TOL_FP8 = 3e-2


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _tt(torch, nd, src, rcv):
    P = src.shape[0]
    s4 = torch.zeros(P, 4, device="cuda"); s4[:, :3] = torch.from_numpy(src).cuda()
    r4 = torch.zeros(P, 4, device="cuda"); r4[:, :3] = torch.from_numpy(rcv).cuda()
    Th = torch.empty(P, device="cuda"); Tl = torch.empty(P, device="cuda")
    J = torch.empty(P, 4, device="cuda")
    nd.spider_tt_pairs(P, s4.data_ptr(), r4.data_ptr(), Th.data_ptr(), Tl.data_ptr(), J.data_ptr())
    torch.cuda.synchronize()
    return Th.double().cpu().numpy() + Tl.double().cpu().numpy(), J.cpu().numpy()[:, :3]


@pytest.mark.parametrize("H", [128, 256])
def test_tt_mlp_fp8_vs_oracle(H):
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    net = synth.mlp_weights(H, 777 + H)
    rng = np.random.default_rng(H + 1)
    P = 3 * 128 * 152 + 77                 # every CTA gets several tiles, ragged tail
    src = np.c_[rng.uniform(0, 60, P), rng.uniform(0, 60, P), rng.uniform(2, 16, P)].astype(np.float32)
    rcv = np.c_[rng.uniform(-10, 70, P), rng.uniform(-10, 70, P), np.zeros(P)].astype(np.float32)
    nd = binding.NetDevice(binding.Net(binding.TT_MLP, mlp=net), precision=binding.FP8)
    T, J = _tt(torch, nd, src, rcv)
    To, Jo = O.tt_mlp(src.astype(np.float64), rcv.astype(np.float64), net)
    d = src.astype(np.float64) - rcv
    r = np.sqrt((d * d).sum(1))
    net_part = np.abs(To - r * net["b"][4][0])
    errT = np.abs(T - To)
    relJ = rel_l2(J, Jo)
    print(f"FP8 H={H}: max|dT| {errT.max()*1e6:.2f} us, rms|dT| {np.sqrt((errT**2).mean())*1e6:.2f} us, "
          f"network part rms {np.sqrt((net_part**2).mean())*1e3:.3f} ms, J rel-L2 {relJ:.2e}")
    assert np.isfinite(T).all() and np.isfinite(J).all()
    assert errT.max() <= 0.15 * net_part.max() + 2e-6
    assert relJ <= 0.1
    nd.close()


def test_fp8_rejects_width_64():
    net = synth.mlp_weights(64, 5)
    with pytest.raises(Exception):
        binding.NetDevice(binding.Net(binding.TT_MLP, mlp=net), precision=binding.FP8)


def test_fp8_gradient_full_batch_mlp128():
    cat = synth.make_catalog(2)
    ctx = binding.Context.from_catalog(cat, precision=binding.FP8)
    g, lp = ctx.spider_grad_logpost(0)
    P = O.problem_from_catalog(cat)
    L, go, _ = O.log_posterior(P, cat.init_xyzt)
    rel = rel_l2(g, go)
    print(f"FP8 H=128 full batch: gradient rel-L2 {rel:.3e}, logpost {lp:.8e} vs {L:.8e}")
    assert rel <= GRAD_TOL_FP8
    ctx.close()


def test_fp8_gradient_minibatch_mlp256():
    s = synth.scaled_spec(3, 20000, batch_n=1 << 17)
    cat = synth.make_catalog(s)
    ctx = binding.Context.from_catalog(cat, precision=binding.FP8)
    g, lp = ctx.spider_grad_logpost(7)
    P = O.problem_from_catalog(cat)
    sel = P.batch(7)
    L, go, _ = O.log_posterior(P, cat.init_xyzt, sel)
    rel = rel_l2(g, go)
    print(f"FP8 H=256 minibatch: gradient rel-L2 {rel:.3e}")
    assert rel <= GRAD_TOL_FP8
    ctx.close()
