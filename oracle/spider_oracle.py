"""FP64 oracle of the SPIDER sampling step.  TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and `bench.py`'s CPU-baseline and
reference legs may import or run anything in this directory; the product path
(the CUDA library and its binding) never does and shares no code with it.

It is a plain, slow, single-threaded restatement of what one SGLD step of
SPIDER (Ross et al., arXiv 2508.12117) computes, in float64, written from the
paper's definitions.  Each function names the passage it follows.  Where the
paper is silent or ambiguous the reading taken is stated in the docstring:

  R1  centroid prior (Sec. 3.1, centroid equations): the prior is placed on
      the current catalog centroid mean_m(theta_m), centred on the centroid
      of the initial catalog theta_0.
  R2  edge weights w_e (Eq. correlation_decay) are computed once from the
      initial catalog, normalised to mean 1 over all observations of each
      station group, frozen, and never differentiated.
  R3  the weight floor epsilon of Eq. correlation_decay is a parameter eps_w
      (default 1e-5); the step size is a separate parameter eps.
  R4  Sigma_g follows Eq. marginal_sigma (with W^{1/2}); the group g is the
      station (single phase).
  R5  a minibatch is a set of whole blocks of consecutive observations in
      canonical order, chosen without replacement by a keyed Feistel
      permutation; its likelihood is the exact Gaussian marginal of the
      selected observations, scaled by N / n_selected (Eq. sgd).
  R6  the Langevin noise of event m uses one Philox4x32-10 call with counter
      (m, chain, catalog, 'NOIS') and key = the step's seed; Box-Muller maps
      words (w0, w1) to (x, y) and (w2, w3) to (z, t0).
  R7  constants of the log density (log det Sigma, sigma normalisers) are
      dropped: they do not depend on theta under R2.
  R8  canonical order: events renumbered by the Morton key of their initial
      positions (ties by index), observations sorted by (i, j, k) in the new
      numbering, ties by original index.
  R9  stage 1 (Sec. 3.2, Eq. stage1loss with an L1 norm): the objective is
      -(N/n) sum_n |r_n| plus the same event and centroid priors (they keep
      the common translation of the catalog determined); d|r|/dr = sign(r),
      0 at r = 0.
  R10 pSGLD follows Eq. pSGLD as printed: v = beta2 v + (1 - beta2) g*g,
      V = 1 / (sqrt(v) + eps_p), theta += eps V g + sqrt(2 eps V) eta (the
      Gamma correction term of the original pSGLD paper is not printed and is
      omitted); v starts at 0.
  R11 the stage-1 optimiser is Adam with bias correction, t = 1, 2, ...:
      m = beta1 m + (1 - beta1) g, v = beta2 v + (1 - beta2) g*g,
      theta += eta (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps_p),
      an ascent on the objective of R9.
  R12 outlier rejection after stage 1 ("residuals greater than 4 median
      absolute deviations", Sec. 3.2/4): an observation is kept when
      |r - median(r)| <= 4 MAD with MAD = median |r - median(r)| (no
      normal-consistency factor), per catalog, over all its observations at
      the stage-1 solution; an even count takes the mean of the two middle
      values.
  R14 posterior summaries (Sec. 3.5, 4.1, 5): percentiles by linear
      interpolation between order statistics at rank (n - 1) p / 100; the
      credible half-width is half the [lo, hi] percentile interval; the
      calibration value is the fraction of samples below the truth; the
      effective sample size is n / tau with tau = 1 + 2 sum_t rho_t over the
      lags t >= 1 while the sample autocorrelation rho_t stays positive.
  R13 linearisation error (Proposition 1; Sec. 4 keeps observations whose
      error is at most 5 %): for observation (i, j, k) the non-linear
      difference dT = T(x_j, s_k) - T(x_i, s_k) and the linearised one
      grad_x T(x_i, s_k) . (x_j - x_i); the error is relative to |dT|.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np

# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
# as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies, Weyl key bumps.
# ---------------------------------------------------------------------------
_M32 = np.uint64(0xFFFFFFFF)
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)
TAG_NOISE = 0x4E4F4953    # 'NOIS'
TAG_FEISTEL = 0x46454953  # 'FEIS'


def philox4x32_10(ctr, key) -> np.ndarray:
    """ctr (..., 4) and key (..., 2) unsigned 32-bit words -> (..., 4) words."""
    ctr = np.asarray(ctr, dtype=np.uint64)
    key = np.asarray(key, dtype=np.uint64)
    c0, c1, c2, c3 = (ctr[..., a] & _M32 for a in range(4))
    k0, k1 = key[..., 0] & _M32, key[..., 1] & _M32
    for rnd in range(10):
        if rnd:
            k0 = (k0 + PHILOX_W0) & _M32
            k1 = (k1 + PHILOX_W1) & _M32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & _M32,
                          (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & _M32)
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def seed_key(seed: int) -> tuple:
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & 0xFFFFFFFF, seed >> 32)


def unit_from_word(w) -> np.ndarray:
    """(floor(w / 2^9) + 1/2) * 2^-23: exact in float32 and float64, in (0, 1)."""
    w = np.asarray(w, dtype=np.uint64)
    return ((w >> np.uint64(9)).astype(np.float64) + 0.5) * (2.0 ** -23)


def box_muller(wa, wb):
    """Two words -> two standard normals (Box and Muller 1958)."""
    u1, u2 = unit_from_word(wa), unit_from_word(wb)
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad * np.cos(2.0 * math.pi * u2), rad * np.sin(2.0 * math.pi * u2)


def langevin_noise(M: int, seed: int, chain: int = 0, catalog: int = 0) -> np.ndarray:
    """eta ~ N(0, I) of Sec. 3.2 for every event, reading R6.  (M, 4)."""
    m = np.arange(M, dtype=np.uint64)
    ctr = np.stack([m, np.full(M, chain, np.uint64), np.full(M, catalog, np.uint64),
                    np.full(M, TAG_NOISE, np.uint64)], -1)
    k0, k1 = seed_key(seed)
    w = philox4x32_10(ctr, np.array([k0, k1], dtype=np.uint64))
    x, y = box_muller(w[:, 0], w[:, 1])
    z, t = box_muller(w[:, 2], w[:, 3])
    return np.stack([x, y, z, t], -1)


# ---------------------------------------------------------------------------
# minibatch selection (reading R5)
# ---------------------------------------------------------------------------
def feistel_index(s: int, n_blocks: int, seed: int) -> int:
    """The s-th element of a keyed permutation of [0, n_blocks).

    Balanced 4-round Feistel network on 2h bits (h = half of the bit width of
    n_blocks - 1, at least 1), round function = low h bits of word 0 of
    Philox4x32-10(counter (R, round, 0, 'FEIS'), key = seed); values outside
    [0, n_blocks) are walked around the cycle until they fall inside."""
    bits = max(2, (n_blocks - 1).bit_length())
    bits += bits & 1
    h = bits // 2
    mask = (1 << h) - 1
    k = np.array(seed_key(seed), dtype=np.uint64)
    x = s
    while True:
        L, R = x >> h, x & mask
        for rnd in range(4):
            F = int(philox4x32_10(np.array([R, rnd, 0, TAG_FEISTEL], dtype=np.uint64), k)[0]) & mask
            L, R = R, L ^ F
        x = (L << h) | R
        if x < n_blocks:
            return x


def select_blocks(n_obs: int, block_obs: int, batch_n: int, seed: int) -> np.ndarray:
    """Block ids of one minibatch, in selection order.  Full batch (all blocks,
    ascending) when batch_n == 0 or batch_n >= n_obs."""
    nb = -(-n_obs // block_obs)
    if batch_n <= 0 or batch_n >= n_obs:
        return np.arange(nb, dtype=np.int64)
    n_sel = min(nb, -(-batch_n // block_obs))
    return np.array([feistel_index(s, nb, seed) for s in range(n_sel)], dtype=np.int64)


# ---------------------------------------------------------------------------
# canonical order (reading R8)
# ---------------------------------------------------------------------------
def morton_perm(xyz: np.ndarray) -> np.ndarray:
    """Events ordered by their Morton key (new -> old).  Key: per-axis minimum
    lo_c, ext = largest per-axis extent, q_c = floor((c - lo_c) * 2097151/ext)
    clamped to 21 bits, bit b of (q_x, q_y, q_z) at key bits (3b, 3b+1, 3b+2)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    M = xyz.shape[0]
    lo = xyz.min(axis=0)
    ext = float((xyz.max(axis=0) - lo).max()) if M else 0.0
    scale = 2097151.0 / ext if ext > 0 else 0.0
    q = np.clip(np.floor((xyz - lo) * scale), 0, 2097151).astype(np.uint64)
    key = np.zeros(M, dtype=np.uint64)
    one = np.uint64(1)
    for b in range(21):
        for a in range(3):
            key |= ((q[:, a] >> np.uint64(b)) & one) << np.uint64(3 * b + a)
    return np.argsort(key, kind="stable").astype(np.int64)


def canonical_order(init_xyz, i, j, k, reorder: bool = True):
    """(event permutation new->old, observation order) of reading R8."""
    M = init_xyz.shape[0]
    ev = morton_perm(init_xyz[:, :3]) if reorder else np.arange(M, dtype=np.int64)
    rank = np.empty(M, dtype=np.int64)
    rank[ev] = np.arange(M)
    a, b = rank[np.asarray(i)], rank[np.asarray(j)]
    kk = np.asarray(k, dtype=np.int64)
    key = (a * M + b) * (int(kk.max()) + 1 if kk.size else 1) + kk
    if key.size == 0 or np.all(key[1:] >= key[:-1]):
        order = np.arange(key.size, dtype=np.int64)
    else:
        order = np.lexsort((kk, b, a))     # stable: ties keep input order
    return ev, order


def minibatch_obs(order: np.ndarray, block_obs: int, blocks: np.ndarray) -> np.ndarray:
    """Observation indices (caller numbering) of the selected blocks."""
    parts = [order[b * block_obs:(b + 1) * block_obs] for b in blocks]
    return np.concatenate(parts) if parts else np.zeros(0, dtype=np.int64)


# ---------------------------------------------------------------------------
# edge weights, Eq. correlation_decay (readings R2, R3)
# ---------------------------------------------------------------------------
def edge_weights(init_xyz, i, j, k, n_stations, ell, p, eps_w) -> np.ndarray:
    d = np.linalg.norm(init_xyz[i, :3] - init_xyz[j, :3], axis=1)
    w = (d / ell) ** p + eps_w
    tot = np.bincount(k, weights=w, minlength=n_stations)
    cnt = np.bincount(k, minlength=n_stations)
    mean = np.where(cnt > 0, tot / np.maximum(cnt, 1), 1.0)
    return w / mean[k]


# ---------------------------------------------------------------------------
# travel-time models T(x; s) and dT/dx (Sec. 2.1)
# ---------------------------------------------------------------------------
def tt_homogeneous(src, rcv, v):
    """T = |x - s| / c and grad_x T = (x - s) / (c r)  (Sec. 2.1, homogeneous medium)."""
    d = src - rcv
    r = np.sqrt((d * d).sum(-1))
    return r / v, d / (v * r)[..., None]


def tt_linear_gradient(src, rcv, v0, g):
    """Velocity v = v0 + g z:  T = arccosh(1 + g^2 r^2 / (2 v_s v_r)) / g,
    written as log1p(X + sqrt(X (2 + X))) / g with X = g^2 r^2 / (2 v_s v_r).
    Derivatives: dT/dX = 1 / (g sqrt(X (2 + X))); dX/dx_h = g^2 (x_h - s_h)/(v_s v_r);
    dX/dz = g^2 (z - s_z)/(v_s v_r) - X g / v_s."""
    d = src - rcv
    r2 = (d * d).sum(-1)
    vs = v0 + g * src[..., 2]
    vr = v0 + g * rcv[..., 2]
    X = g * g * r2 / (2.0 * vs * vr)
    T = np.log1p(X + np.sqrt(X * (2.0 + X))) / g
    dTdX = 1.0 / (g * np.sqrt(X * (2.0 + X)))
    dX = g * g * d / (vs * vr)[..., None]
    dX[..., 2] -= X * g / vs
    return T, dTdX[..., None] * dX


def _silu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return z * s, s * (1.0 + z * (1.0 - s))


def mlp_tau(src, rcv, net: dict):
    """tau = MLP([x; s]) with SiLU hidden layers and its source gradient dtau/dx.

    Forward in float64 with the given (float32) weights; the gradient by the
    reverse-mode chain (Sec. 3.2 computes gradients with reverse-mode
    automatic differentiation):
      delta_L = W_out^T * silu'(z_L),  delta_{l-1} = (W_l^T delta_l) * silu'(z_{l-1}),
      dtau/dx = (W_1^T delta_1)[source part]."""
    W = [np.asarray(w, dtype=np.float64) for w in net["W"]]
    b = [np.asarray(v, dtype=np.float64) for v in net["b"]]
    x = np.concatenate([src, rcv], -1)
    h = x
    dsil = []
    for l in range(len(W) - 1):
        z = h @ W[l].T + b[l]
        h, ds = _silu(z)
        dsil.append(ds)
    tau = (h @ W[-1].T + b[-1])[..., 0]
    delta = W[-1][0][None, :] * dsil[-1]
    for l in range(len(W) - 2, 0, -1):
        delta = (delta @ W[l]) * dsil[l - 1]
    dtau = (delta @ W[0])[..., :3]
    return tau, dtau


def tt_mlp(src, rcv, net: dict):
    """T = |x - s| * tau(x, s), tau = MLP([x; s]) (see `mlp_tau`), and
    dT/dx = tau (x - s)/r + r dtau/dx."""
    tau, dtau = mlp_tau(src, rcv, net)
    d = src - rcv
    r = np.sqrt((d * d).sum(-1))
    T = r * tau
    dT = tau[..., None] * d / r[..., None] + r[..., None] * dtau
    return T, dT


@dataclass
class Model:
    kind: str                 # "homogeneous" | "gradient" | "mlp"
    v0: float = 6.0
    g: float = 0.05
    net: Optional[dict] = None

    def __call__(self, src, rcv):
        if self.kind == "homogeneous":
            return tt_homogeneous(src, rcv, self.v0)
        if self.kind == "gradient":
            return tt_linear_gradient(src, rcv, self.v0, self.g)
        return tt_mlp(src, rcv, self.net)


# ---------------------------------------------------------------------------
# whitened likelihood, Eqs. marginal_sigma and the correlated Gaussian
# ---------------------------------------------------------------------------
def group_nodes(ev_i, ev_j, st, n_stations):
    """Nodes of the latent field b: one per (event, station) met by the
    observations; returns node ids of both ends and the (event, station) of
    each node (event-major order)."""
    key_i = ev_i.astype(np.int64) * n_stations + st
    key_j = ev_j.astype(np.int64) * n_stations + st
    uniq, inv = np.unique(np.concatenate([key_i, key_j]), return_inverse=True)
    n = ev_i.shape[0]
    return inv[:n], inv[n:], uniq // n_stations, uniq % n_stations


def whiten_dense(r, ev_i, ev_j, st, w, sigma, kappa, n_stations):
    """q = Sigma^{-1} r and r^T Sigma^{-1} r with Sigma built element by element.

    Per station group g: Sigma_g[e, f] = sigma^2 [e == f]
      + kappa^2 sqrt(w_e w_f) (A_g A_g^T)[e, f], where row e of A_g has +1 at
    event i_e and -1 at event j_e (Delta b = b_i - b_j)."""
    import scipy.linalg as sla
    q = np.zeros_like(r)
    quad = 0.0
    for g in np.unique(st):
        idx = np.nonzero(st == g)[0]
        E = idx.size
        S = np.zeros((E, E))
        for a in range(E):
            for c in range(E):
                ia, ja, ic, jc = ev_i[idx[a]], ev_j[idx[a]], ev_i[idx[c]], ev_j[idx[c]]
                aat = int(ia == ic) - int(ia == jc) - int(ja == ic) + int(ja == jc)
                S[a, c] = kappa ** 2 * math.sqrt(w[idx[a]] * w[idx[c]]) * aat
            S[a, a] += sigma ** 2
        cf = sla.cho_factor(S, lower=True)
        qg = sla.cho_solve(cf, r[idx])
        q[idx] = qg
        quad += float(r[idx] @ qg)
    return q, quad


def whiten_woodbury(r, ev_i, ev_j, st, w, sigma, kappa, n_stations):
    """Same quantities through the push-through (Woodbury) identity:
    Sigma^{-1} = sigma^{-2} (I - B (lambda I + B^T B)^{-1} B^T), B = W^{1/2} A,
    lambda = sigma^2 / kappa^2; the inner system (one block per station group,
    since nodes are (event, station)) is solved by a sparse direct LU."""
    if kappa == 0.0:
        return r / sigma ** 2, float(r @ r) / sigma ** 2
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    ni, nj, _, _ = group_nodes(ev_i, ev_j, st, n_stations)
    E = r.shape[0]
    V = int(max(ni.max(), nj.max())) + 1 if E else 0
    sw = np.sqrt(w)
    rows = np.concatenate([np.arange(E), np.arange(E)])
    cols = np.concatenate([ni, nj])
    vals = np.concatenate([sw, -sw])
    B = sp.csr_matrix((vals, (rows, cols)), shape=(E, V))
    lam = sigma ** 2 / kappa ** 2
    K = (B.T @ B + lam * sp.identity(V)).tocsc()
    u = B.T @ r
    z = spla.splu(K).solve(u)
    q = (r - B @ z) / sigma ** 2
    quad = float(r @ r - u @ z) / sigma ** 2
    return q, quad


# ---------------------------------------------------------------------------
# the problem: catalog + model + hyper-parameters
# ---------------------------------------------------------------------------
@dataclass
class Problem:
    init: np.ndarray          # (M, 4) theta_0, prior mean
    stations: np.ndarray      # (S, 3)
    i: np.ndarray
    j: np.ndarray
    k: np.ndarray
    dt: np.ndarray            # FP64 observed differential times
    model: Model
    sigma: float
    kappa: float
    p: float
    ell: float
    eps_w: float
    sig_e: np.ndarray
    sig_c: np.ndarray
    batch_n: int = 0
    block_obs: int = 4096
    reorder: bool = True
    w: Optional[np.ndarray] = None

    def __post_init__(self):
        self.i = np.asarray(self.i, dtype=np.int64)
        self.j = np.asarray(self.j, dtype=np.int64)
        self.k = np.asarray(self.k, dtype=np.int64)
        self.sig_e = np.asarray(self.sig_e, dtype=np.float64)
        self.sig_c = np.asarray(self.sig_c, dtype=np.float64)
        if self.w is None:
            self.w = edge_weights(self.init, self.i, self.j, self.k, self.stations.shape[0],
                                  self.ell, self.p, self.eps_w)
        self.ev_perm, self.order = canonical_order(self.init, self.i, self.j, self.k,
                                                   self.reorder)

    @property
    def M(self):
        return self.init.shape[0]

    @property
    def N(self):
        return self.i.shape[0]

    def batch(self, seed: int) -> np.ndarray:
        """Observation indices of the minibatch keyed by `seed` (reading R5)."""
        blocks = select_blocks(self.N, self.block_obs, self.batch_n, seed)
        return np.sort(minibatch_obs(self.order, self.block_obs, blocks))


def problem_from_catalog(cat, hyper=None, reorder=True, batch_n=None, model=None):
    """Build an oracle `Problem` from a synthetic catalog and its hyper-parameters."""
    h = hyper or cat.spec.hyper
    if model is None:
        if cat.spec.forward == "mlp":
            model = Model("mlp", net=cat.net)
        else:
            model = Model("homogeneous", v0=6.0)
    return Problem(cat.init_xyzt.copy(), cat.stations.copy(), cat.i, cat.j, cat.k, cat.dt,
                   model, h.sigma, h.kappa, h.p, h.ell, h.eps_w, np.array(h.sig_e),
                   np.array(h.sig_c), h.batch_n if batch_n is None else batch_n,
                   h.block_obs, reorder)


def travel_times(prob: Problem, theta, sel):
    """T and dT/dx for every (event, station) pair met by observations `sel`."""
    ii, jj, kk = prob.i[sel], prob.j[sel], prob.k[sel]
    S = prob.stations.shape[0]
    ni, nj, nev, nst = group_nodes(ii, jj, kk, S)
    T, dT = prob.model(theta[nev, :3], prob.stations[nst])
    return ni, nj, nev, nst, T, dT


def residuals(prob: Problem, theta, sel):
    """r_n = tau_obs_n - [(T_ik + t0_i) - (T_jk + t0_j)]  (Eq. 1)."""
    ni, nj, nev, nst, T, dT = travel_times(prob, theta, sel)
    ii, jj = prob.i[sel], prob.j[sel]
    r = prob.dt[sel] - ((T[ni] + theta[ii, 3]) - (T[nj] + theta[jj, 3]))
    return r, (ni, nj, nev, nst, T, dT)


def log_posterior(prob: Problem, theta, sel=None, whiten="woodbury", loss="whitened"):
    """log p(theta | tau) up to constants (R7) and its gradient, for the
    observation subset `sel` (None = all) scaled by N / |sel| (Eq. sgd):

      L = (N/n) sum_g -1/2 r_g^T Sigma_g^{-1} r_g
          - 1/2 sum_m |(theta_m - mu_m) / sigma_e|^2        (event prior)
          - 1/2 |(mean(theta) - mean(theta_0)) / sigma_c|^2 (centroid prior, R1)

    With loss="l1" the data term is -(N/n) sum_n |r_n| instead (R9).
    Returns (L, grad (M, 4), info dict)."""
    theta = np.asarray(theta, dtype=np.float64)
    M, N = prob.M, prob.N
    if sel is None:
        sel = np.arange(N)
    n = sel.shape[0]
    scale = N / n if n else 0.0
    r, (ni, nj, nev, nst, T, dT) = residuals(prob, theta, sel)
    if loss == "l1":
        # -|r| has derivative -sign(r); in the notation below q = sign(r), and
        # quad = 2 sum |r| so that -1/2 quad = -sum |r|
        q = np.sign(r)
        quad = 2.0 * float(np.abs(r).sum())
    else:
        fn = whiten_woodbury if whiten == "woodbury" else whiten_dense
        q, quad = fn(r, prob.i[sel], prob.j[sel], prob.k[sel], prob.w[sel], prob.sigma,
                     prob.kappa, prob.stations.shape[0])
    # d(-1/2 r^T Sigma^-1 r)/dT_p = sum_{n: p = (i_n,k_n)} q_n - sum_{n: p = (j_n,k_n)} q_n
    V = T.shape[0]
    s_node = np.bincount(ni, weights=q, minlength=V) - np.bincount(nj, weights=q, minlength=V)
    grad = np.zeros((M, 4))
    for a in range(3):
        grad[:, a] = np.bincount(nev, weights=s_node * dT[:, a], minlength=M)
    grad[:, 3] = np.bincount(nev, weights=s_node, minlength=M)
    grad *= scale
    loglik = -0.5 * quad * scale
    dev = (theta - prob.init) / prob.sig_e
    logprior = -0.5 * float((dev * dev).sum())
    grad += -(theta - prob.init) / prob.sig_e ** 2
    c = theta.mean(axis=0) - prob.init.mean(axis=0)
    logcen = -0.5 * float(((c / prob.sig_c) ** 2).sum())
    grad += -(c / (M * prob.sig_c ** 2))[None, :]
    info = dict(r=r, q=q, T=T, dT=dT, nodes=(nev, nst), scale=scale, loglik=loglik,
                logprior=logprior, logcen=logcen, n=n)
    return loglik + logprior + logcen, grad, info


# ---------------------------------------------------------------------------
# SGLD (Sec. 3.2): theta <- theta + eps grad log p_hat + sqrt(2 eps) eta
# ---------------------------------------------------------------------------
def sgld_update(theta, grad, eps, noise, noise_scale=1.0):
    return theta + eps * grad + noise_scale * math.sqrt(2.0 * eps) * noise


def sgld_step(prob: Problem, theta, eps, seed, noise_scale=1.0, chain=0, catalog=0):
    """One SGLD step with the minibatch and the noise both keyed by `seed`."""
    sel = None if (prob.batch_n <= 0 or prob.batch_n >= prob.N) else prob.batch(seed)
    _, g, _ = log_posterior(prob, theta, sel)
    eta = langevin_noise(prob.M, seed, chain, catalog)
    return sgld_update(theta, g, eps, eta, noise_scale)


def run_chain(prob: Problem, theta0, eps, seeds, noise_scale=1.0, thin=1,
              chain=0, catalog=0, callback: Optional[Callable] = None):
    """Iterate `sgld_step` over the given per-step seeds; returns the final
    state and the thinned samples (every `thin`-th state, after the update)."""
    theta = np.array(theta0, dtype=np.float64)
    samples = []
    for t, s in enumerate(seeds):
        theta = sgld_step(prob, theta, eps, s, noise_scale, chain, catalog)
        if (t + 1) % thin == 0:
            samples.append(theta.copy())
        if callback is not None:
            callback(t, theta)
    return theta, samples


# ---------------------------------------------------------------------------
# pSGLD (Eq. pSGLD, R10) and the stage-1 Adam optimiser (Sec. 3.2, R11)
# ---------------------------------------------------------------------------
def psgld_update(theta, grad, v, eps, beta2, eps_p, noise, noise_scale=1.0):
    """One pSGLD update; returns (theta', v')."""
    v = beta2 * v + (1.0 - beta2) * grad * grad
    V = 1.0 / (np.sqrt(v) + eps_p)
    theta = theta + eps * V * grad + noise_scale * np.sqrt(2.0 * eps * V) * noise
    return theta, v


def adam_update(theta, grad, m, v, t, eta, beta1, beta2, eps_p):
    """One Adam ascent step (t = 1, 2, ...); returns (theta', m', v')."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta + eta * mh / (np.sqrt(vh) + eps_p), m, v


def run_updates(prob: Problem, theta0, eps, seeds, update="sgld", loss="whitened", beta1=0.9,
                beta2=0.99, eps_p=1e-5, noise_scale=1.0, chain=0, catalog=0, m0=None, v0=None, t0=0):
    """Iterate one update rule ("sgld", "psgld" or "adam") over the per-step
    seeds (minibatch and noise keyed by the seed); t0 steps were taken before.
    Returns (theta, m, v)."""
    theta = np.array(theta0, dtype=np.float64)
    m = np.zeros_like(theta) if m0 is None else np.array(m0, dtype=np.float64)
    v = np.zeros_like(theta) if v0 is None else np.array(v0, dtype=np.float64)
    for t, s in enumerate(seeds):
        sel = None if (prob.batch_n <= 0 or prob.batch_n >= prob.N) else prob.batch(s)
        _, g, _ = log_posterior(prob, theta, sel, loss=loss)
        if update == "adam":
            theta, m, v = adam_update(theta, g, m, v, t0 + t + 1, eps, beta1, beta2, eps_p)
            continue
        eta = langevin_noise(prob.M, s, chain, catalog)
        if update == "psgld":
            theta, v = psgld_update(theta, g, v, eps, beta2, eps_p, eta, noise_scale)
        else:
            theta = sgld_update(theta, g, eps, eta, noise_scale)
    return theta, m, v


def mad_filter(r, k_mad=4.0):
    """Outlier rejection of R12: (keep mask, median, MAD) of the residuals r."""
    r = np.asarray(r, dtype=np.float64)
    med = float(np.median(r))
    mad = float(np.median(np.abs(r - med)))
    return np.abs(r - med) <= k_mad * mad, med, mad


def linearisation_filter(prob: Problem, theta, max_rel=0.05):
    """Keep mask of R13 over all observations (caller order), and the relative
    errors |dT - dT_lin| / |dT|."""
    theta = np.asarray(theta, dtype=np.float64)
    st = prob.stations[prob.k]
    Ti, dTi = prob.model(theta[prob.i, :3], st)
    Tj, _ = prob.model(theta[prob.j, :3], st)
    dT = Tj - Ti
    lin = (dTi * (theta[prob.j, :3] - theta[prob.i, :3])).sum(axis=1)
    err = np.abs(dT - lin)
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = err / np.abs(dT)
    return err <= max_rel * np.abs(dT), rel


def ess_series(x) -> float:
    """Effective sample size of one chain (R14)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    d = x - x.mean()
    c0 = float((d * d).sum())
    tau = 1.0
    if c0 > 0.0:
        for t in range(1, n):
            rho = float((d[:-t] * d[t:]).sum()) / c0
            if not rho > 0.0:
                break
            tau += 2.0 * rho
    return n / tau


def uq_stats(samples, truth=None, lo_pct=0.5, hi_pct=99.5):
    """Per event and coordinate, from samples (n, M, 4) in time order: median,
    credible half-width, calibration value (None without truth) and ESS (R14)."""
    s = np.asarray(samples, dtype=np.float64)
    med = np.percentile(s, 50.0, axis=0)
    half = 0.5 * (np.percentile(s, hi_pct, axis=0) - np.percentile(s, lo_pct, axis=0))
    calib = None if truth is None else (s < np.asarray(truth)[None]).mean(axis=0)
    n, M, _ = s.shape
    ess = np.array([[ess_series(s[:, m, a]) for a in range(4)] for m in range(M)])
    return med, half, calib, ess


def grad_noise_ratio(g, G, eps) -> float:
    """Variance of the stochastic gradient relative to the injected Langevin
    noise (Sec. 3.6, the quantity the step size is tuned against, 0.1-1): the
    update's stochastic part eps (g - G) against the noise sqrt(2 eps) eta,
    eps^2 mean((g - G)^2) / (2 eps), the mean over every event coordinate;
    g is a minibatch gradient and G the full-batch gradient at the same state.
    Linear in eps, as the paper notes."""
    d = np.asarray(g, dtype=np.float64) - np.asarray(G, dtype=np.float64)
    return float(eps * eps * np.mean(d * d) / (2.0 * eps))


def grad_norms(grad) -> np.ndarray:
    """Per-event gradient norm |g_m| (diagnostic, Sec. 3.6)."""
    return np.sqrt((np.asarray(grad, dtype=np.float64) ** 2).sum(axis=1))
