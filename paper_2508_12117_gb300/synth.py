"""Seeded synthetic double-difference catalogs: the shared INPUT generator.

Both the CUDA path (tests, bench) and the FP64 oracle consume what this module
draws; neither side's arithmetic lives here.  The only physics in this file is
the "true medium" used to synthesise observed differential times (a
homogeneous or a linear-gradient velocity, evaluated with their textbook
closed forms), which plays the role of the unknown Earth: the inference under
test never evaluates it.

What is drawn (all FP64, numpy PCG64 streams seeded with 20250817 + workload id):
  * event clouds: uniform boxes (tiny workload) or planar fault patches
    (strike U[0,180), dip U[45,90], 5 x 3 km, N(0, 0.2 km) off-plane);
  * origin times U(0, 1000) s;
  * surface stations on a grid or uniform over the region plus 10 km margins;
  * initial catalog = truth + N(0, 0.5 km) per coordinate, + N(0, 0.1 s) in t0
    (the "single-event locations" a relocation starts from, Sec. 3.2);
  * directed k-nearest-neighbour event pairs within 2 km of each other in the
    initial catalog, observed at the event's nearest stations;
  * dd times tau_obs = (T_ik + t0_i) - (T_jk + t0_j) + noise (Eq. 1);
  * a seeded random travel-time MLP 6 -> 4 x H SiLU -> 1 (Xavier-uniform
    x 0.1, hidden biases 0, output bias 1/5.5) standing in for EikoNet.

Events are listed in Morton (Z-curve) order of their initial positions and
observations in (i, j, k) order, as a catalog prepared for relocation would be.
The Morton key is defined once, in words, in the docstring of `morton_order`.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 20250817
PAIR_RADIUS_KM = 2.0


# --------------------------------------------------------------------------
# workload descriptions
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Hyper:
    """Likelihood / prior / sampler hyper-parameters of one workload.

    Defaults follow Sec. 4 and Table 1 (kappa 0.03 s, p 0.25, ell 40 km,
    centroid sigma 0.01 km / 0.01 s) and Sec. 4.1 (event prior sigma
    0.5 km / 0.1 s around the initial catalog)."""
    sigma: float = 0.005
    kappa: float = 0.03
    p: float = 0.25
    ell: float = 40.0
    eps_w: float = 1e-5
    sig_e: tuple = (0.5, 0.5, 0.5, 0.1)
    sig_c: tuple = (0.01, 0.01, 0.01, 0.01)
    eps: float = 1e-4          # SGLD step size
    batch_n: int = 0           # observations per minibatch, 0 = full batch
    block_obs: int = 4096      # observations per minibatch block


@dataclasses.dataclass
class Spec:
    name: str
    wid: int                   # workload id (seed offset)
    n_events: int
    n_stations: int
    n_neighbours: int
    n_obs_stations: int        # stations observing each event (nearest ones)
    layout: str                # "box" or "faults"
    n_faults: int = 0
    region_km: float = 10.0
    medium: str = "homogeneous"  # true medium: "homogeneous" (6 km/s) or "gradient" (5 + 0.05 z)
    noise: str = "normal"        # "normal" or "laplace_outliers"
    noise_s: float = 0.01
    outlier_frac: float = 0.0
    forward: str = "homogeneous"  # model the path evaluates: "homogeneous" or "mlp"
    hidden: int = 0
    hyper: Hyper = dataclasses.field(default_factory=Hyper)


def _eps_for(kappa, s_obs, n_over_b):
    # step size inside the plain-SGLD stability bound of the whitened t0
    # curvature (about s_obs / kappa^2 per event, times N/n)
    return 0.2 * kappa * kappa / (s_obs * max(1.0, n_over_b))


def spec(wid: int) -> Spec:
    """The five synthetic workloads (sizes of the paper's catalogs, Sec. 3.7)."""
    if wid == 1:
        h = Hyper(sigma=0.01, eps=1e-4, batch_n=0)
        return Spec("tiny-200ev-analytic", 1, 200, 10, 10, 10, "box", region_km=10.0,
                    medium="homogeneous", noise="normal", noise_s=0.01,
                    forward="homogeneous", hyper=h)
    if wid == 2:
        # full batch: an event's ~400 dd observations all act in every step, so
        # the curvature per origin time is ~20x that of the minibatch workloads
        # (a step of 0.2 kappa^2 / 10 grows the error ~3x per step)
        h = Hyper(sigma=0.005, eps=_eps_for(0.03, 200, 1.0), batch_n=0)
        return Spec("mlp128-10kev-2Mdd", 2, 10_000, 50, 20, 10, "faults", n_faults=5,
                    region_km=20.0, medium="gradient", noise="normal", noise_s=0.005,
                    forward="mlp", hidden=128, hyper=h)
    if wid == 3:
        h = Hyper(sigma=math.sqrt(2.0) * 0.005, eps=_eps_for(0.03, 20, 50e6 / 2 ** 20),
                  batch_n=2 ** 20)
        return Spec("mlp256-100kev-50Mdd", 3, 100_000, 100, 25, 20, "faults", n_faults=50,
                    region_km=60.0, medium="gradient", noise="laplace_outliers",
                    noise_s=0.005, outlier_frac=0.02, forward="mlp", hidden=256, hyper=h)
    if wid == 4:
        h = Hyper(sigma=0.005, eps=_eps_for(0.03, 20, 200e6 / 2 ** 22), batch_n=2 ** 22)
        return Spec("mlp256-1Mev-200Mdd", 4, 1_000_000, 200, 10, 20, "faults", n_faults=500,
                    region_km=150.0, medium="gradient", noise="normal", noise_s=0.005,
                    forward="mlp", hidden=256, hyper=h)
    raise ValueError(f"unknown workload id {wid}")


def batch_specs(n: int = 16, minibatch: int = 1 << 18) -> List[Spec]:
    """The batched workload: n catalogs of uneven sizes (events log-uniform in
    [1k, 200k], stations U{20..150}, neighbours U{10..25}, 10 observing
    stations per event, faults at the 1M-event catalog's density, N(0, 5 ms)
    noise), all read through one 6 -> 4 x 128 network; minibatches of
    `minibatch` observations per catalog."""
    rng = np.random.default_rng(SEED_BASE + 5)
    draws = []
    for c in range(n):
        M = int(round(math.exp(rng.uniform(math.log(1000.0), math.log(200000.0)))))
        S = int(rng.integers(20, 151))
        K = int(rng.integers(10, 26))
        draws.append((M, S, K))
    # one step size for every sub-problem (a batched step takes one eps): inside
    # the stability bound of the catalog with the most observations per
    # minibatch observation (about M K 10 dd observations per catalog)
    n_over_b = max(M * K * 10 for M, _, K in draws) / minibatch
    out = []
    for c, (M, S, K) in enumerate(draws):
        nf = max(1, int(round(M / 2000)))
        region = max(10.0, 150.0 * math.sqrt(nf / 500.0))
        h = Hyper(sigma=0.005, eps=_eps_for(0.03, 20, n_over_b), batch_n=minibatch)
        out.append(Spec(f"batch{c:02d}-{M}ev", 50 + c, M, S, K, 10, "faults", n_faults=nf,
                        region_km=region, medium="gradient", noise="normal", noise_s=0.005,
                        forward="mlp", hidden=128, hyper=h))
    return out


def batch_network() -> dict:
    """The network shared by the batched workload."""
    return mlp_weights(128, SEED_BASE + 105)


def scaled_spec(wid: int, n_events: int, n_faults: Optional[int] = None,
                region_km: Optional[float] = None, n_stations: Optional[int] = None,
                batch_n: Optional[int] = None, hidden: Optional[int] = None) -> Spec:
    """A smaller catalog drawn with the recipe of workload `wid` (same fault
    density, neighbours and stations per event), used for bounded samples."""
    s = spec(wid)
    s = dataclasses.replace(s, hyper=dataclasses.replace(s.hyper))
    frac = n_events / s.n_events
    s.n_events = n_events
    if s.layout == "faults":
        s.n_faults = n_faults if n_faults is not None else max(1, round(s.n_faults * frac))
        s.region_km = region_km if region_km is not None else max(
            10.0, s.region_km * math.sqrt(max(frac, 1e-9)))
    elif region_km is not None:
        s.region_km = region_km
    if n_stations is not None:
        s.n_stations = n_stations
    if batch_n is not None:
        s.hyper.batch_n = batch_n
    if hidden is not None:
        s.hidden = hidden
    s.name = f"{s.name}-scaled-{n_events}ev"
    return s


@dataclasses.dataclass
class Catalog:
    spec: Spec
    true_xyzt: np.ndarray      # (M, 4) FP64 truth (km, km, km, s)
    init_xyzt: np.ndarray      # (M, 4) FP64 initial catalog theta_0 (also the prior mean)
    stations: np.ndarray       # (S, 3) FP64 (km, z positive down)
    i: np.ndarray              # (N,) int32 first event
    j: np.ndarray              # (N,) int32 second event
    k: np.ndarray              # (N,) int32 station
    dt: np.ndarray             # (N,) FP64 observed differential time (s)
    net: Optional[dict] = None  # MLP weights (FP32), see `mlp_weights`

    @property
    def M(self):
        return self.true_xyzt.shape[0]

    @property
    def N(self):
        return self.i.shape[0]

    @property
    def S(self):
        return self.stations.shape[0]


# --------------------------------------------------------------------------
# ordering
# --------------------------------------------------------------------------
def morton_order(xyz: np.ndarray) -> np.ndarray:
    """Z-curve order of points (returns the permutation new -> old).

    Key: per axis c, lo_c = min, ext = max over axes of (max_c - lo_c),
    scale = 2097151 / ext (0 if ext == 0), q_c = floor((c - lo_c) * scale)
    clamped to [0, 2097151]; bit b of q_x, q_y, q_z goes to key bit 3b, 3b+1,
    3b+2.  Ties keep the original order (stable sort)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    lo = xyz.min(axis=0)
    ext = float((xyz.max(axis=0) - lo).max()) if xyz.shape[0] else 0.0
    scale = 2097151.0 / ext if ext > 0 else 0.0
    q = np.floor((xyz - lo) * scale)
    q = np.clip(q, 0, 2097151).astype(np.uint64)
    key = np.zeros(xyz.shape[0], dtype=np.uint64)
    for b in range(21):
        for a in range(3):
            key |= ((q[:, a] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + a)
    return np.argsort(key, kind="stable")


# --------------------------------------------------------------------------
# the "true medium" used only to synthesise observations
# --------------------------------------------------------------------------
def _true_tt(src: np.ndarray, rcv: np.ndarray, medium: str) -> np.ndarray:
    d = src - rcv
    r = np.sqrt((d * d).sum(axis=-1))
    if medium == "homogeneous":
        return r / 6.0
    v0, g = 5.0, 0.05
    vs = v0 + g * src[..., 2]
    vr = v0 + g * rcv[..., 2]
    x = g * g * r * r / (2.0 * vs * vr)
    return np.log1p(x + np.sqrt(x * (2.0 + x))) / g


# --------------------------------------------------------------------------
# drawing
# --------------------------------------------------------------------------
def _events(s: Spec, rng: np.random.Generator) -> np.ndarray:
    M = s.n_events
    if s.layout == "box":
        L = s.region_km
        xyz = np.stack([rng.uniform(0, L, M), rng.uniform(0, L, M), rng.uniform(5, 15, M)], 1)
        return xyz
    nf = s.n_faults
    sizes = np.full(nf, M // nf)
    sizes[: M - sizes.sum()] += 1
    cx = rng.uniform(0, s.region_km, nf)
    cy = rng.uniform(0, s.region_km, nf)
    cz = rng.uniform(3, 15, nf)
    strike = np.deg2rad(rng.uniform(0, 180, nf))
    dip = np.deg2rad(rng.uniform(45, 90, nf))
    fid = np.repeat(np.arange(nf), sizes)
    a = rng.uniform(-2.5, 2.5, M)      # along strike
    b = rng.uniform(-1.5, 1.5, M)      # along dip
    c = rng.normal(0.0, 0.2, M)        # off plane
    st, dp = strike[fid], dip[fid]
    us = np.stack([np.sin(st), np.cos(st), np.zeros(M)], 1)
    ud = np.stack([np.cos(st) * np.cos(dp), -np.sin(st) * np.cos(dp), np.sin(dp)], 1)
    un = np.cross(us, ud)
    xyz = np.stack([cx[fid], cy[fid], cz[fid]], 1) + a[:, None] * us + b[:, None] * ud + c[:, None] * un
    xyz[:, 2] = np.maximum(xyz[:, 2], 0.5)
    return xyz


def _stations(s: Spec, rng: np.random.Generator) -> np.ndarray:
    if s.layout == "box":
        # 5 x 2 grid spanning 40 x 40 km, centred on the event box
        c = s.region_km / 2.0
        xs = c + np.linspace(-20.0, 20.0, 5)
        ys = c + np.array([-20.0, 20.0])
        X, Y = np.meshgrid(xs, ys, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), np.zeros(10)], 1)[: s.n_stations]
    lo, hi = -10.0, s.region_km + 10.0
    S = s.n_stations
    return np.stack([rng.uniform(lo, hi, S), rng.uniform(lo, hi, S), np.zeros(S)], 1)


def mlp_weights(hidden: int, seed: int) -> dict:
    """Seeded travel-time network 6 -> H -> H -> H -> H -> 1 (SiLU hidden).

    Weights are (out, in) row-major FP32, Xavier-uniform scaled by 0.1; hidden
    biases are 0 and the output bias is 1/5.5 s/km (a mean slowness)."""
    rng = np.random.default_rng(seed)
    dims = [6, hidden, hidden, hidden, hidden, 1]
    W, b = [], []
    for l in range(5):
        fi, fo = dims[l], dims[l + 1]
        bound = math.sqrt(6.0 / (fi + fo)) * 0.1
        W.append(rng.uniform(-bound, bound, size=(fo, fi)).astype(np.float32))
        b.append(np.zeros(fo, dtype=np.float32))
    b[4][0] = np.float32(1.0 / 5.5)
    return {"H": hidden, "W": W, "b": b}


def strong_mlp_weights(hidden: int, seed: int, first_scale: float = 1.0 / 20.0) -> dict:
    """A travel-time network whose learned part is a large share of tau.

    Same shapes and biases as `mlp_weights`, but the hidden and output layers
    are Xavier-uniform at full scale and the first layer is Xavier-uniform x
    `first_scale` (the inputs are coordinates in km spanning tens of km, so
    1/20 keeps the first pre-activations of order one).  Over a 60 x 60 km
    region tau then varies by about 50 % (roughly 0.18 to 0.27 s/km) and
    r dtau/dx is about a fifth of dT/dx by rel-L2, so an error anywhere in the
    reverse sweep shows in the Jacobian and in the gradient.  first_scale = 1
    gives a network whose output dominates tau entirely."""
    rng = np.random.default_rng(seed)
    dims = [6, hidden, hidden, hidden, hidden, 1]
    W, b = [], []
    for l in range(5):
        fi, fo = dims[l], dims[l + 1]
        bound = math.sqrt(6.0 / (fi + fo)) * (first_scale if l == 0 else 1.0)
        W.append(rng.uniform(-bound, bound, size=(fo, fi)).astype(np.float32))
        b.append(np.zeros(fo, dtype=np.float32))
    b[4][0] = np.float32(1.0 / 5.5)
    return {"H": hidden, "W": W, "b": b}


def make_catalog(s, chunk: int = 1 << 24) -> Catalog:
    """Draw one catalog.  `s` is a workload id or a `Spec`."""
    if isinstance(s, int):
        s = spec(s)
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(SEED_BASE + s.wid)
    M = s.n_events
    xyz = _events(s, rng)
    t0 = rng.uniform(0.0, 1000.0, M)
    sta = _stations(s, rng)
    init = np.concatenate([xyz + rng.normal(0.0, 0.5, (M, 3)),
                           (t0 + rng.normal(0.0, 0.1, M))[:, None]], 1)
    init[:, 2] = np.maximum(init[:, 2], 0.2)
    true = np.concatenate([xyz, t0[:, None]], 1)

    # list events in Morton order of the initial catalog
    perm = morton_order(init[:, :3])
    true, init = true[perm].copy(), init[perm].copy()

    # directed k-nearest neighbours within 2 km (initial positions)
    K = s.n_neighbours
    tree = cKDTree(init[:, :3])
    kq = min(K + 1, M)
    dist, nb = tree.query(init[:, :3], k=kq, distance_upper_bound=PAIR_RADIUS_KM, workers=-1)
    dist = np.asarray(dist, dtype=np.float64).reshape(M, kq)
    nb = np.asarray(nb).reshape(M, kq).astype(np.int64)
    ok = np.isfinite(dist) & (nb < M) & (nb != np.arange(M)[:, None])
    # the K nearest valid neighbours (by distance), then listed by ascending j
    order = np.argsort(np.where(ok, dist, np.inf), axis=1, kind="stable")[:, :K]
    near = np.take_along_axis(np.where(ok, nb, M), order, axis=1)
    near = np.sort(near, axis=1)
    valid = near < M
    n_valid = valid.sum(axis=1)

    # observing stations: the event's nearest ones, ascending index
    so = min(s.n_obs_stations, sta.shape[0])
    stree = cKDTree(sta)
    _, sts = stree.query(init[:, :3], k=so, workers=-1)
    sts = np.sort(np.asarray(sts).reshape(M, so), axis=1).astype(np.int32)

    pi = np.repeat(np.arange(M, dtype=np.int32), n_valid)
    pj = near[valid].astype(np.int32)
    N = pi.shape[0] * so
    i_obs = np.repeat(pi, so)
    j_obs = np.repeat(pj, so)
    k_obs = sts[pi].reshape(-1)

    dt = np.empty(N, dtype=np.float64)
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        ii, jj, kk = i_obs[a:b], j_obs[a:b], k_obs[a:b]
        Ti = _true_tt(true[ii, :3], sta[kk], s.medium)
        Tj = _true_tt(true[jj, :3], sta[kk], s.medium)
        n = b - a
        if s.noise == "normal":
            e = rng.normal(0.0, s.noise_s, n)
        else:
            e = rng.laplace(0.0, s.noise_s, n)
            out = rng.random(n) < s.outlier_frac
            e[out] = rng.uniform(-0.5, 0.5, int(out.sum()))
        dt[a:b] = (Ti + true[ii, 3]) - (Tj + true[jj, 3]) + e

    net = mlp_weights(s.hidden, SEED_BASE + 100 + s.wid) if s.forward == "mlp" else None
    return Catalog(s, true, init, sta, i_obs, j_obs, k_obs.astype(np.int32), dt, net)


def shuffled_events(cat: Catalog, seed: int = 7) -> Catalog:
    """The same catalog with events listed in a random order (observations
    relabelled and shuffled too): exercises the library's own reordering."""
    rng = np.random.default_rng(seed)
    M = cat.M
    perm = rng.permutation(M)            # new position -> old event
    inv = np.empty(M, dtype=np.int64)
    inv[perm] = np.arange(M)
    oo = rng.permutation(cat.N)
    return Catalog(cat.spec, cat.true_xyzt[perm].copy(), cat.init_xyzt[perm].copy(),
                   cat.stations.copy(), inv[cat.i[oo]].astype(np.int32),
                   inv[cat.j[oo]].astype(np.int32), cat.k[oo].copy(), cat.dt[oo].copy(),
                   cat.net)
