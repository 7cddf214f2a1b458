"""The allocation-free travel-time entry point agrees with the allocating one.

spider_tt_pairs_noalloc serves callers that may not allocate device memory
(fixed arenas, allocator-free hot paths); its scratch lives in static device
memory shared by all calls.  Two calls in a row must each reproduce
spider_tt_pairs on the same inputs, whether this file runs alone in a fresh
process or after every other test."""
import numpy as np
import pytest

from paper_2508_12117_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _inputs(torch, P, seed):
    rng = np.random.default_rng(seed)
    src = np.c_[rng.uniform(0, 60, P), rng.uniform(0, 60, P), rng.uniform(2, 16, P)].astype(np.float32)
    rcv = np.c_[rng.uniform(-10, 70, P), rng.uniform(-10, 70, P), np.zeros(P)].astype(np.float32)
    s4 = torch.zeros(P, 4, device="cuda"); s4[:, :3] = torch.from_numpy(src).cuda()
    r4 = torch.zeros(P, 4, device="cuda"); r4[:, :3] = torch.from_numpy(rcv).cuda()
    return s4, r4


@pytest.mark.parametrize("H,kind", [(128, "config"), (256, "config"), (256, "strong")])
def test_no_alloc_matches_allocating_entry_point_twice(H, kind):
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    w = synth.mlp_weights(H, 4242 + H) if kind == "config" else synth.strong_mlp_weights(H, 4243 + H)
    net = binding.Net(binding.TT_MLP, mlp=w)
    P = 70001                               # many tiles and a ragged tail
    s4, r4 = _inputs(torch, P, H)
    ref_hi, ref_lo = torch.empty(P, device="cuda"), torch.empty(P, device="cuda")
    ref_J = torch.empty(P, 4, device="cuda")
    nd = binding.NetDevice(net)
    nd.spider_tt_pairs(P, s4.data_ptr(), r4.data_ptr(), ref_hi.data_ptr(), ref_lo.data_ptr(),
                       ref_J.data_ptr())
    torch.cuda.synchronize()
    ref_T = ref_hi.double() + ref_lo.double()
    for call in range(2):
        hi, lo = torch.full((P,), np.nan, device="cuda"), torch.full((P,), np.nan, device="cuda")
        J = torch.full((P, 4), np.nan, device="cuda")
        binding.spider_tt_pairs_noalloc(net, P, s4.data_ptr(), r4.data_ptr(), hi.data_ptr(),
                                        lo.data_ptr(), J.data_ptr())
        torch.cuda.synchronize()
        T = hi.double() + lo.double()
        # the same tolerances as the FP32 parity tests: |dT| <= 1 us, J rel-L2 <= 1e-5
        assert float((T - ref_T).abs().max()) <= 1e-6, call
        dJ = (J[:, :3].double() - ref_J[:, :3].double()).norm() / ref_J[:, :3].double().norm()
        assert float(dJ) <= 1e-5, call
        # the network part r dtau/dx = J - (T / r^2)(x - s) on its own, which the
        # whole-J check cannot see when the network is small next to the bias
        d = s4[:, :3].double() - r4[:, :3].double()
        r2 = (d * d).sum(1, keepdim=True)
        jn = J[:, :3].double() - (T[:, None] / r2) * d
        jn_ref = ref_J[:, :3].double() - (ref_T[:, None] / r2) * d
        assert float((jn - jn_ref).norm() / jn_ref.norm()) <= 1e-5, call
    nd.close()


def test_no_alloc_rejects_sizes_beyond_its_limit():
    torch = pytest.importorskip("torch")
    net = binding.Net(binding.TT_MLP, mlp=synth.mlp_weights(128, 1))
    with pytest.raises(binding.SpiderError) as e:
        binding.spider_tt_pairs_noalloc(net, (1 << 20) + 1, 0, 0, 0)
    assert e.value.code == -1
    bad = synth.mlp_weights(128, 2)
    bad["W"][2][3, 5] = np.nan
    with pytest.raises(binding.SpiderError) as e:
        binding.spider_tt_pairs_noalloc(binding.Net(binding.TT_MLP, mlp=bad), 10, 0, 0, 0)
    assert e.value.code == -1
    homo = binding.Net(binding.TT_HOMOGENEOUS, v0=6.0)
    with pytest.raises(binding.SpiderError) as e:
        binding.spider_tt_pairs_noalloc(homo, 10, 0, 0, 0)
    assert e.value.code == -6
