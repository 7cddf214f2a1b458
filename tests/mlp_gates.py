"""Shared measurements of a device travel-time form against the FP64 oracle.

T = r tau(x, s) and dT/dx = tau (x - s)/r + r dtau/dx.  With a network whose
learned part is small next to the output bias (the configured Xavier x 0.1
nets), the geometric term tau (x - s)/r is almost all of dT/dx, so a gate on the
whole Jacobian cannot see the reverse sweep.  The measurements below therefore
split off the network part on both sides:

  device: J_net = J - (T / r) (x - s) / r     (T, J as the kernel returns them)
  oracle: J_net = r dtau/dx                   (`mlp_tau`, computed directly)

and the network part of T is T - r b5 (b5 the output bias)."""
import numpy as np

from oracle import spider_oracle as O
from paper_2508_12117_gb300 import binding


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def random_pairs(n, seed):
    """Sources over a 60 x 60 km region at 2-16 km depth, surface receivers."""
    rng = np.random.default_rng(seed)
    src = np.c_[rng.uniform(0, 60, n), rng.uniform(0, 60, n), rng.uniform(2, 16, n)].astype(np.float32)
    rcv = np.c_[rng.uniform(-10, 70, n), rng.uniform(-10, 70, n), np.zeros(n)].astype(np.float32)
    return src, rcv


def tt_on_device(torch, nd, src, rcv):
    """T (hi + lo, FP64 on the host) and J (P x 3) from spider_tt_pairs."""
    P = src.shape[0]
    s4 = torch.zeros(P, 4, device="cuda"); s4[:, :3] = torch.from_numpy(src).cuda()
    r4 = torch.zeros(P, 4, device="cuda"); r4[:, :3] = torch.from_numpy(rcv).cuda()
    Th = torch.empty(P, device="cuda"); Tl = torch.empty(P, device="cuda")
    J = torch.empty(P, 4, device="cuda")
    nd.spider_tt_pairs(P, s4.data_ptr(), r4.data_ptr(), Th.data_ptr(), Tl.data_ptr(), J.data_ptr())
    torch.cuda.synchronize()
    return Th.double().cpu().numpy() + Tl.double().cpu().numpy(), J.cpu().numpy()[:, :3].astype(np.float64)


def measure(torch, net, precision, src, rcv):
    """Errors of one device form on the given pairs, as a dict:
    err_t_max (s), net_t_max (largest |network part of T|, s), rel_j (whole J),
    rel_jnet (network part of J), jnet_share (|r dtau/dx| / |dT/dx|)."""
    nd = binding.NetDevice(binding.Net(binding.TT_MLP, mlp=net), precision=precision)
    try:
        T, J = tt_on_device(torch, nd, src, rcv)
    finally:
        nd.close()
    s64, r64 = src.astype(np.float64), rcv.astype(np.float64)
    tau_o, dtau_o = O.mlp_tau(s64, r64, net)
    d = s64 - r64
    r = np.sqrt((d * d).sum(1))
    To = r * tau_o
    Jo_net = r[:, None] * dtau_o
    Jo = (tau_o / r)[:, None] * d + Jo_net
    J_net = J - (T / r / r)[:, None] * d
    net_t = np.abs(To - r * float(net["b"][4][0]))
    assert np.isfinite(T).all() and np.isfinite(J).all()
    return dict(err_t_max=float(np.abs(T - To).max()), net_t_max=float(net_t.max()),
                rel_j=rel_l2(J, Jo), rel_jnet=rel_l2(J_net, Jo_net),
                jnet_share=float(np.linalg.norm(Jo_net) / np.linalg.norm(Jo)))


def with_net(cat, net):
    """The catalog with another travel-time network (same observations)."""
    import dataclasses
    return dataclasses.replace(cat, net=net)
