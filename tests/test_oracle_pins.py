"""Pins of the FP64 oracle against facts fixed outside it: closed forms, the
published Philox known-answer vectors, algebraic identities, invariances,
brute-force finite differences and the exact stationary law of discrete
Langevin dynamics on a Gaussian target.  CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import spider_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def tiny_problem(M=12, S=4, K=4, model=None, kappa=0.03, sigma=0.01, seed=0, batch_n=0,
                 block_obs=4096, reorder=True):
    rng = np.random.default_rng(seed)
    xyz = np.stack([rng.uniform(0, 3, M), rng.uniform(0, 3, M), rng.uniform(5, 8, M)], 1)
    t0 = rng.uniform(0, 100, M)
    init = np.concatenate([xyz, t0[:, None]], 1)
    sta = np.stack([rng.uniform(-20, 20, S), rng.uniform(-20, 20, S), np.zeros(S)], 1)
    ii, jj, kk = [], [], []
    for i in range(M):
        others = [j for j in range(M) if j != i]
        nb = rng.choice(others, size=min(K, M - 1), replace=False)
        for j in sorted(nb):
            for k in range(S):
                ii.append(i); jj.append(j); kk.append(k)
    ii, jj, kk = map(np.array, (ii, jj, kk))
    dt = rng.normal(0, 0.3, ii.size) + (t0[ii] - t0[jj])
    model = model or O.Model("homogeneous", v0=6.0)
    return O.Problem(init, sta, ii, jj, kk, dt, model, sigma, kappa, 0.25, 40.0, 1e-5,
                     np.array([0.5, 0.5, 0.5, 0.1]), np.array([0.01] * 4), batch_n,
                     block_obs, reorder)


def random_net(H=8, seed=1, scale=0.5):
    rng = np.random.default_rng(seed)
    dims = [6, H, H, H, H, 1]
    W = [rng.normal(0, scale / math.sqrt(dims[l]), (dims[l + 1], dims[l])) for l in range(5)]
    b = [rng.normal(0, 0.1, dims[l + 1]) for l in range(5)]
    b[4][0] = 1 / 5.5
    return {"H": H, "W": W, "b": b}


# ---------------------------------------------------------------- Philox / noise
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = O.philox4x32_10(np.array(v[:4], np.uint64), np.array(v[4:6], np.uint64))
        assert [int(x) for x in out] == v[6:10]


def test_unit_from_word_range_and_exactness():
    w = np.array([0, 511, 512, 2 ** 32 - 1], dtype=np.uint64)
    u = O.unit_from_word(w)
    assert u[0] == 0.5 * 2.0 ** -23 and u[1] == u[0]
    assert u[2] == 1.5 * 2.0 ** -23
    assert u[3] == 1.0 - 0.5 * 2.0 ** -23
    assert np.all(u.astype(np.float32).astype(np.float64) == u)  # exact in float32


def test_langevin_noise_is_standard_normal():
    eta = O.langevin_noise(200_000, seed=12345)
    assert abs(eta.mean()) < 0.005
    assert abs(eta.var() - 1.0) < 0.01
    c = np.corrcoef(eta.T)
    assert np.all(np.abs(c - np.eye(4)) < 0.01)
    kurt = ((eta - eta.mean(0)) ** 4).mean(0) / eta.var(0) ** 2
    assert np.all(np.abs(kurt - 3.0) < 0.05)
    # a different seed / chain gives a different stream
    assert not np.allclose(O.langevin_noise(10, 1), O.langevin_noise(10, 2))
    assert not np.allclose(O.langevin_noise(10, 1, chain=0), O.langevin_noise(10, 1, chain=1))


# ---------------------------------------------------------------- selection / order
@pytest.mark.parametrize("nb", [1, 2, 3, 5, 17, 64, 100, 1000])
def test_feistel_is_a_permutation(nb):
    for seed in (0, 1, 0xDEADBEEFCAFE):
        out = [O.feistel_index(s, nb, seed) for s in range(nb)]
        assert sorted(out) == list(range(nb))
    if nb >= 17:
        a = [O.feistel_index(s, nb, 1) for s in range(nb)]
        b = [O.feistel_index(s, nb, 2) for s in range(nb)]
        assert a != b


def test_select_blocks_sizes():
    assert list(O.select_blocks(10000, 1000, 0, 5)) == list(range(10))
    assert list(O.select_blocks(10000, 1000, 20000, 5)) == list(range(10))
    sel = O.select_blocks(10500, 1000, 2500, 5)      # 11 blocks, ragged tail
    assert len(sel) == 3 and len(set(sel)) == 3 and max(sel) < 11


def test_morton_order_on_grids():
    # corners of a cube: Z-order is x + 2y + 4z
    pts = np.array([[x, y, z] for x in (0, 1) for y in (0, 1) for z in (0, 1)], float)
    rng = np.random.default_rng(0)
    pts = pts[rng.permutation(8)]
    order = O.morton_perm(pts)
    code = pts[:, 0] + 2 * pts[:, 1] + 4 * pts[:, 2]
    assert list(code[order]) == list(range(8))
    # 4 x 4 x 4 grid: the leading two bits of each quantised axis are the grid
    # coordinate, so the order is the textbook 2-bit Morton order
    g = np.array([[x, y, z] for x in range(4) for y in range(4) for z in range(4)], float)
    g = g[rng.permutation(64)]
    order = O.morton_perm(g)

    def textbook(x, y, z):
        c = 0
        for b in range(2):
            c |= ((x >> b) & 1) << (3 * b) | ((y >> b) & 1) << (3 * b + 1) | ((z >> b) & 1) << (3 * b + 2)
        return c
    codes = [textbook(int(p[0]), int(p[1]), int(p[2])) for p in g[order]]
    assert codes == sorted(codes) and len(set(codes)) == 64


def test_canonical_order_sorted_and_stable():
    P = tiny_problem(M=15, S=3, K=3, seed=3)
    rank = np.empty(P.M, np.int64)
    rank[P.ev_perm] = np.arange(P.M)
    key = np.stack([rank[P.i[P.order]], rank[P.j[P.order]], P.k[P.order]], 1)
    assert all(tuple(key[a]) <= tuple(key[a + 1]) for a in range(len(key) - 1))
    assert sorted(P.order.tolist()) == list(range(P.N))


# ---------------------------------------------------------------- weights
def test_edge_weights_mean_one_per_group_and_monotone():
    P = tiny_problem(M=20, S=3, K=5, seed=2)
    for g in range(3):
        assert abs(P.w[P.k == g].mean() - 1.0) < 1e-12
    d = np.linalg.norm(P.init[P.i, :3] - P.init[P.j, :3], axis=1)
    g0 = P.k == 0
    o = np.argsort(d[g0])
    assert np.all(np.diff(P.w[g0][o]) >= -1e-15)
    # raw form (d/ell)^p + eps: ratio of two weights in one group
    a, b = np.nonzero(g0)[0][:2]
    ratio = ((d[a] / 40) ** 0.25 + 1e-5) / ((d[b] / 40) ** 0.25 + 1e-5)
    assert abs(P.w[a] / P.w[b] - ratio) < 1e-12


# ---------------------------------------------------------------- travel times
def fd_grad(f, src, rcv, h=1e-4):
    g = np.zeros_like(src)
    for a in range(3):
        e = np.zeros(3); e[a] = h
        g[..., a] = (f(src + e, rcv)[0] - f(src - e, rcv)[0]) / (2 * h)
    return g


def test_homogeneous_closed_form():
    T, dT = O.tt_homogeneous(np.array([[3.0, 4.0, 12.0]]), np.array([[0.0, 0.0, 0.0]]), 6.0)
    assert T[0] == 13.0 / 6.0
    assert np.allclose(dT[0], np.array([3, 4, 12]) / (6 * 13), rtol=0, atol=1e-15)
    rng = np.random.default_rng(0)
    src = rng.uniform(-10, 10, (50, 3)); src[:, 2] = rng.uniform(2, 15, 50)
    rcv = np.concatenate([rng.uniform(-30, 30, (50, 2)), np.zeros((50, 1))], 1)
    T, dT = O.tt_homogeneous(src, rcv, 6.0)
    assert np.allclose(np.linalg.norm(dT, axis=1), 1 / 6.0, rtol=1e-14)   # eikonal
    f = lambda s, r: O.tt_homogeneous(s, r, 6.0)
    assert np.allclose(dT, fd_grad(f, src, rcv), rtol=1e-7, atol=1e-10)


def test_linear_gradient_closed_forms():
    v0, g = 5.0, 0.05
    # vertical ray: T = integral dz / (v0 + g z) = ln(v_s / v_r) / g
    src = np.array([[1.0, 2.0, 12.0]]); rcv = np.array([[1.0, 2.0, 0.0]])
    T, _ = O.tt_linear_gradient(src, rcv, v0, g)
    assert abs(T[0] - math.log((v0 + g * 12.0) / v0) / g) < 1e-12
    rng = np.random.default_rng(1)
    src = np.concatenate([rng.uniform(-10, 10, (64, 2)), rng.uniform(2, 15, (64, 1))], 1)
    rcv = np.concatenate([rng.uniform(-30, 30, (64, 2)), np.zeros((64, 1))], 1)
    T, dT = O.tt_linear_gradient(src, rcv, v0, g)
    # eikonal equation at the source: |grad T| = 1 / v(z_s)
    assert np.allclose(np.linalg.norm(dT, axis=1), 1.0 / (v0 + g * src[:, 2]), rtol=1e-10)
    # reciprocity
    Tr, _ = O.tt_linear_gradient(rcv, src, v0, g)
    assert np.allclose(T, Tr, rtol=1e-13)
    # g -> 0 is the homogeneous medium
    Tg, _ = O.tt_linear_gradient(src, rcv, v0, 1e-7)
    Th, _ = O.tt_homogeneous(src, rcv, v0)
    assert np.allclose(Tg, Th, rtol=1e-6)
    f = lambda s, r: O.tt_linear_gradient(s, r, v0, g)
    assert np.allclose(dT, fd_grad(f, src, rcv), rtol=1e-7, atol=1e-10)


def test_mlp_reduces_to_homogeneous():
    net = random_net(H=16)
    net["W"][1][:] = 0; net["W"][2][:] = 0; net["W"][3][:] = 0; net["W"][4][:] = 0
    net["b"][4][0] = 1.0 / 6.0
    rng = np.random.default_rng(2)
    src = np.concatenate([rng.uniform(-10, 10, (20, 2)), rng.uniform(2, 15, (20, 1))], 1)
    rcv = np.concatenate([rng.uniform(-30, 30, (20, 2)), np.zeros((20, 1))], 1)
    T, dT = O.tt_mlp(src, rcv, net)
    Th, dTh = O.tt_homogeneous(src, rcv, 6.0)
    assert np.allclose(T, Th, rtol=1e-15) and np.allclose(dT, dTh, rtol=1e-14, atol=1e-16)


def test_mlp_jacobian_fd_and_autograd():
    torch = pytest.importorskip("torch")
    net = random_net(H=16, scale=1.0)
    rng = np.random.default_rng(3)
    src = np.concatenate([rng.uniform(-10, 10, (30, 2)), rng.uniform(2, 15, (30, 1))], 1)
    rcv = np.concatenate([rng.uniform(-30, 30, (30, 2)), np.zeros((30, 1))], 1)
    T, dT = O.tt_mlp(src, rcv, net)
    f = lambda s, r: O.tt_mlp(s, r, net)
    assert np.allclose(dT, fd_grad(f, src, rcv), rtol=1e-7, atol=1e-9)
    # independent reverse-mode differentiation (library autograd, float64)
    s = torch.tensor(src, dtype=torch.float64, requires_grad=True)
    r = torch.tensor(rcv, dtype=torch.float64)
    h = torch.cat([s, r], 1)
    for l in range(4):
        h = torch.nn.functional.silu(h @ torch.tensor(net["W"][l]).T + torch.tensor(net["b"][l]))
    tau = (h @ torch.tensor(net["W"][4]).T + torch.tensor(net["b"][4]))[:, 0]
    Tt = torch.linalg.norm(s - r, dim=1) * tau
    Tt.sum().backward()
    assert np.allclose(Tt.detach().numpy(), T, rtol=1e-14)
    assert np.allclose(s.grad.numpy(), dT, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- whitening
def test_sigma_elementwise_equals_matrix_form_and_woodbury():
    P = tiny_problem(M=10, S=3, K=4, seed=4)
    rng = np.random.default_rng(4)
    r = rng.normal(0, 0.05, P.N)
    qd, quad_d = O.whiten_dense(r, P.i, P.j, P.k, P.w, P.sigma, P.kappa, 3)
    qw, quad_w = O.whiten_woodbury(r, P.i, P.j, P.k, P.w, P.sigma, P.kappa, 3)
    assert np.allclose(qd, qw, rtol=1e-10, atol=1e-10 * np.abs(qd).max())
    assert abs(quad_d - quad_w) < 1e-10 * abs(quad_d)
    # Sigma_g = sigma^2 I + kappa^2 (W^1/2 A)(W^1/2 A)^T with an explicit incidence matrix
    g = P.k == 1
    ii, jj, ww = P.i[g], P.j[g], P.w[g]
    A = np.zeros((ii.size, P.M))
    A[np.arange(ii.size), ii] += 1.0
    A[np.arange(ii.size), jj] -= 1.0
    B = np.sqrt(ww)[:, None] * A
    Sig = P.sigma ** 2 * np.eye(ii.size) + P.kappa ** 2 * B @ B.T
    assert np.allclose(qd[g], np.linalg.solve(Sig, r[g]), rtol=1e-9, atol=1e-9 * np.abs(qd[g]).max())


def test_sigma_matches_generative_model_by_sampling():
    # r_g = W^1/2 A b + eps with b ~ N(0, kappa^2), eps ~ N(0, sigma^2) (Sec. 3.1):
    # the empirical covariance of simulated residuals matches Sigma_g.
    P = tiny_problem(M=6, S=1, K=3, seed=5, kappa=0.05, sigma=0.02)
    rng = np.random.default_rng(5)
    ns = 400_000
    b = rng.normal(0, P.kappa, (ns, P.M))
    e = rng.normal(0, P.sigma, (ns, P.N))
    sims = np.sqrt(P.w)[None, :] * (b[:, P.i] - b[:, P.j]) + e
    C = sims.T @ sims / ns
    Sinv_r = lambda v: O.whiten_dense(v, P.i, P.j, P.k, P.w, P.sigma, P.kappa, 1)[0]
    Sig = np.linalg.inv(np.stack([Sinv_r(np.eye(P.N)[a]) for a in range(P.N)], 1))
    assert np.abs(C - Sig).max() < 0.02 * np.abs(Sig).max()


def test_isolated_edge_and_kappa_zero():
    sigma, kappa = 0.01, 0.03
    ii, jj, kk = np.array([0, 2]), np.array([1, 3]), np.array([0, 0])
    w = np.array([0.7, 1.3])
    r = np.array([0.02, -0.01])
    q, quad = O.whiten_woodbury(r, ii, jj, kk, w, sigma, kappa, 1)
    expect = r / (sigma ** 2 + 2 * kappa ** 2 * w)
    assert np.allclose(q, expect, rtol=1e-13)
    assert abs(quad - float(r @ expect)) < 1e-10 * quad
    q0, quad0 = O.whiten_woodbury(r, ii, jj, kk, w, sigma, 0.0, 1)
    assert np.allclose(q0, r / sigma ** 2) and abs(quad0 - (r @ r) / sigma ** 2) < 1e-9


def test_star_graph_inner_matrix_has_three_eigenvalues():
    # a hub event paired with 6 others at one station: lambda I + L_W has the
    # eigenvalue lambda (constant vector), lambda + w (leaf differences), and one more
    ii = np.zeros(6, int); jj = np.arange(1, 7); kk = np.zeros(6, int); w = np.ones(6)
    import scipy.sparse as sp
    ni, nj, _, _ = O.group_nodes(ii, jj, kk, 1)
    Bm = sp.csr_matrix((np.r_[np.sqrt(w), -np.sqrt(w)], (np.r_[np.arange(6), np.arange(6)],
                        np.r_[ni, nj])), shape=(6, 7)).toarray()
    lam = 0.01 ** 2 / 0.03 ** 2
    ev = np.linalg.eigvalsh(lam * np.eye(7) + Bm.T @ Bm)
    assert len(np.unique(np.round(ev, 10))) == 3
    assert np.isclose(ev.min(), lam) and np.isclose(ev.max(), lam + 7.0)


# ---------------------------------------------------------------- gradient
def fd_logpost(P, theta, sel=None, h=(1e-5, 1e-5, 1e-5, 1e-6)):
    g = np.zeros_like(theta)
    for m in range(P.M):
        for a in range(4):
            tp, tm = theta.copy(), theta.copy()
            tp[m, a] += h[a]; tm[m, a] -= h[a]
            g[m, a] = (O.log_posterior(P, tp, sel)[0] - O.log_posterior(P, tm, sel)[0]) / (2 * h[a])
    return g


@pytest.mark.parametrize("kind", ["homogeneous", "gradient", "mlp"])
def test_gradient_matches_finite_differences(kind):
    model = {"homogeneous": O.Model("homogeneous", v0=6.0),
             "gradient": O.Model("gradient", v0=5.0, g=0.05),
             "mlp": O.Model("mlp", net=random_net(H=8, scale=1.0))}[kind]
    P = tiny_problem(M=9, S=3, K=3, model=model, seed=6)
    rng = np.random.default_rng(6)
    theta = P.init + np.c_[rng.normal(0, 0.2, (P.M, 3)), rng.normal(0, 0.05, P.M)]
    L, g, _ = O.log_posterior(P, theta)
    gf = fd_logpost(P, theta)
    assert np.linalg.norm(g - gf) <= 1e-6 * np.linalg.norm(g)
    # dense and Woodbury whitening give the same posterior
    Ld, gd, _ = O.log_posterior(P, theta, whiten="dense")
    assert abs(Ld - L) < 1e-9 * abs(L) and np.allclose(gd, g, rtol=1e-8, atol=1e-8 * np.abs(g).max())


def test_minibatch_gradient_matches_finite_differences():
    P = tiny_problem(M=10, S=3, K=4, seed=7, batch_n=24, block_obs=12)
    theta = P.init + 0.1
    sel = P.batch(seed=99)
    assert sel.size == 24
    L, g, info = O.log_posterior(P, theta, sel)
    assert info["scale"] == P.N / 24
    gf = fd_logpost(P, theta, sel)
    assert np.linalg.norm(g - gf) <= 1e-6 * np.linalg.norm(g)


def test_origin_time_shift_invariance():
    P = tiny_problem(M=10, S=3, K=4, seed=8)
    rng = np.random.default_rng(8)
    theta = P.init + np.c_[rng.normal(0, 0.2, (P.M, 3)), rng.normal(0, 0.05, P.M)]
    sel = np.arange(P.N)
    r0, _ = O.residuals(P, theta, sel)
    th = theta.copy(); th[:, 3] += 17.25
    r1, _ = O.residuals(P, th, sel)
    assert np.abs(r1 - r0).max() < 1e-11
    # hence the likelihood gradient has no component along a common t0 shift
    _, g, info = O.log_posterior(P, theta)
    P0 = tiny_problem(M=10, S=3, K=4, seed=8)
    like_t0 = g[:, 3] + (theta[:, 3] - P.init[:, 3]) / P.sig_e[3] ** 2 \
        + (theta[:, 3].mean() - P.init[:, 3].mean()) / (P.M * P.sig_c[3] ** 2)
    assert abs(like_t0.sum()) < 1e-9 * np.abs(like_t0).sum()


def _moved_problem(P, shift=np.zeros(3), phi=0.0):
    """The same catalog with every event, prior mean and station moved rigidly:
    rotated by phi about the vertical axis, then shifted."""
    c, s_ = math.cos(phi), math.sin(phi)
    R = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]])
    init = P.init.copy()
    init[:, :3] = P.init[:, :3] @ R.T + shift
    sta = P.stations @ R.T + shift
    return O.Problem(init, sta, P.i, P.j, P.k, P.dt, P.model, P.sigma, P.kappa, P.p, P.ell,
                     P.eps_w, P.sig_e, P.sig_c, P.batch_n, P.block_obs, P.reorder), R


@pytest.mark.parametrize("kind", ["homogeneous", "gradient"])
def test_rigid_motion_invariance(kind):
    # Homogeneous travel times depend on |x - s| only, linear-gradient ones on the
    # horizontal offset and the two depths; the edge weights depend on
    # inter-event distances, and the priors on theta - theta_0 with equal x and y
    # widths.  Moving events, prior means and stations together rigidly (any
    # shift for the homogeneous model, horizontal ones for the gradient model,
    # rotations about the vertical for both) leaves the log posterior unchanged
    # and turns the position gradient with the motion (a swapped or mis-signed
    # horizontal coordinate anywhere breaks this).
    model = {"homogeneous": O.Model("homogeneous", v0=6.0),
             "gradient": O.Model("gradient", v0=5.0, g=0.05)}[kind]
    P = tiny_problem(M=10, S=4, K=4, seed=21, model=model)
    rng = np.random.default_rng(21)
    d = np.c_[rng.normal(0, 0.2, (P.M, 3)), rng.normal(0, 0.05, P.M)]
    theta = P.init + d
    lp, g, _ = O.log_posterior(P, theta)
    dz = 1.0 if kind == "homogeneous" else 0.0
    for shift, phi in [(np.array([7.5, -3.25, 1.5 * dz]), 0.0), (np.zeros(3), 0.7),
                       (np.array([-2.0, 4.0, 0.5 * dz]), -1.9)]:
        Q, R = _moved_problem(P, shift, phi)
        th = Q.init.copy()
        th[:, :3] += d[:, :3] @ R.T
        th[:, 3] += d[:, 3]
        lq, gq, _ = O.log_posterior(Q, th)
        assert abs(lq - lp) <= 1e-9 * abs(lp)
        assert np.allclose(gq[:, :3], g[:, :3] @ R.T, rtol=1e-8, atol=1e-8 * np.abs(g).max())
        assert np.allclose(gq[:, 3], g[:, 3], rtol=1e-8, atol=1e-8 * np.abs(g).max())


def test_centroid_prior_gradient_is_uniform():
    P = tiny_problem(M=8, S=2, K=3, seed=9)
    theta = P.init + 0.3        # pure translation: the event prior and the centroid pull back
    _, g, info = O.log_posterior(P, theta)
    assert abs(info["logcen"] + 0.5 * ((0.3 / P.sig_c) ** 2).sum()) < 1e-9


def test_minibatch_scaling_is_unbiased_when_iid():
    # with kappa = 0 the observations are independent and the N/n-scaled
    # single-block gradient averages to the full gradient over all blocks
    P = tiny_problem(M=10, S=3, K=4, seed=10, kappa=0.0, batch_n=12, block_obs=12)
    theta = P.init + 0.05
    nb = P.N // 12
    assert P.N % 12 == 0
    _, gfull, _ = O.log_posterior(P, theta)
    acc = np.zeros_like(gfull)
    for b in range(nb):
        sel = np.sort(P.order[b * 12:(b + 1) * 12])
        acc += O.log_posterior(P, theta, sel)[1]
    assert np.allclose(acc / nb, gfull, rtol=1e-10, atol=1e-10 * np.abs(gfull).max())


def _iid_loss(P, theta, sel):
    """-1/2 sum r^2 / sigma^2 over the observations sel (the kappa = 0 data term,
    unscaled), evaluated from the residuals alone."""
    r, _ = O.residuals(P, theta, sel)
    return -0.5 * float(r @ r) / P.sigma ** 2


def test_grad_noise_ratio_zero_for_the_full_batch():
    P = tiny_problem(M=10, S=3, K=4, seed=12)
    theta = P.init + 0.04
    _, G, _ = O.log_posterior(P, theta)
    _, g, _ = O.log_posterior(P, theta, np.arange(P.N))     # a "minibatch" of every observation
    assert O.grad_noise_ratio(g, G, 1e-3) == 0.0


def test_grad_noise_ratio_two_block_iid_closed_form():
    # kappa = 0, two blocks, minibatch = one block: the scaled minibatch
    # gradient is prior + 2 l_b and the full one prior + l_1 + l_2, so for
    # either block g - G = +-(l_1 - l_2) and the ratio is eps/2 mean((l_1 - l_2)^2),
    # with l_b the data-term gradient of block b alone (here by central
    # differences of the iid loss, independently of the oracle's scatter)
    P = tiny_problem(M=8, S=3, K=3, seed=13, kappa=0.0)
    assert P.N % 2 == 0
    half = P.N // 2
    P = tiny_problem(M=8, S=3, K=3, seed=13, kappa=0.0, batch_n=half, block_obs=half)
    rng = np.random.default_rng(13)
    theta = P.init + np.c_[rng.normal(0, 0.05, (P.M, 3)), rng.normal(0, 0.01, P.M)]
    blocks = [np.sort(P.order[b * half:(b + 1) * half]) for b in range(2)]
    h = 1e-6
    ell = []
    for sel in blocks:
        gb = np.zeros_like(theta)
        for m in range(P.M):
            for a in range(4):
                tp, tm = theta.copy(), theta.copy()
                tp[m, a] += h
                tm[m, a] -= h
                gb[m, a] = (_iid_loss(P, tp, sel) - _iid_loss(P, tm, sel)) / (2 * h)
        ell.append(gb)
    want = 0.5 * np.mean((ell[0] - ell[1]) ** 2)
    _, G, _ = O.log_posterior(P, theta)
    for eps in (1e-4, 3e-3):
        for sel in blocks:
            _, g, _ = O.log_posterior(P, theta, sel)
            assert abs(O.grad_noise_ratio(g, G, eps) - eps * want) <= 1e-6 * eps * want


def test_mlp_tau_gradient_by_finite_differences():
    net = random_net(H=16, scale=1.0, seed=4)
    rng = np.random.default_rng(4)
    src = np.concatenate([rng.uniform(-10, 10, (25, 2)), rng.uniform(2, 15, (25, 1))], 1)
    rcv = np.concatenate([rng.uniform(-30, 30, (25, 2)), np.zeros((25, 1))], 1)
    tau, dtau = O.mlp_tau(src, rcv, net)
    h = 1e-5
    for a in range(3):
        sp, sm = src.copy(), src.copy()
        sp[:, a] += h
        sm[:, a] -= h
        fd = (O.mlp_tau(sp, rcv, net)[0] - O.mlp_tau(sm, rcv, net)[0]) / (2 * h)
        assert np.allclose(dtau[:, a], fd, rtol=1e-7, atol=1e-10)
    # T = r tau with its Jacobian split into the geometric and the network part
    T, dT = O.tt_mlp(src, rcv, net)
    d = src - rcv
    r = np.sqrt((d * d).sum(1))
    assert np.allclose(T, r * tau, rtol=1e-15)
    assert np.allclose(dT - (tau / r)[:, None] * d, r[:, None] * dtau, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- SGLD
def test_sgld_stationary_law_on_gaussian_target():
    # theta' = theta + eps * (-h (theta - mu)) + sqrt(2 eps) eta has the exact
    # stationary law N(mu, 1 / (h (1 - eps h / 2))) (discrete Euler chain).
    h, mu, eps = 4.0, 1.5, 0.1
    C = 25_000
    theta = np.full((C, 4), mu)
    acc, acc2, n = 0.0, 0.0, 0
    for t in range(1200):
        g = -h * (theta - mu)
        theta = O.sgld_update(theta, g, eps, O.langevin_noise(C, seed=1000 + t))
        if t >= 200:
            acc += theta.sum(); acc2 += (theta * theta).sum(); n += theta.size
    mean = acc / n
    var = acc2 / n - mean * mean
    exact = 1.0 / (h * (1.0 - eps * h / 2.0))
    assert abs(mean - mu) < 0.005
    assert abs(var / exact - 1.0) < 0.01, (var, exact)


def test_sgld_step_runs_and_is_deterministic():
    P = tiny_problem(M=10, S=3, K=4, seed=11, batch_n=24, block_obs=12)
    a, _ = O.run_chain(P, P.init, 1e-5, [5, 6, 7])
    b, _ = O.run_chain(P, P.init, 1e-5, [5, 6, 7])
    c, _ = O.run_chain(P, P.init, 1e-5, [5, 6, 8])
    assert np.array_equal(a, b) and not np.array_equal(a, c)


# ---------------------------------------------------------------- stage 1, pSGLD, Adam
def test_l1_objective_value_and_gradient():
    # R9: the L1 data term is -(N/n) sum |r|; its gradient is checked against
    # central differences (|r| is smooth away from r = 0, which a generic
    # perturbed state avoids)
    P = tiny_problem(M=8, S=3, K=3, seed=21)
    rng = np.random.default_rng(21)
    theta = P.init + np.c_[rng.normal(0, 0.2, (P.M, 3)), rng.normal(0, 0.05, P.M)]
    L, g, info = O.log_posterior(P, theta, loss="l1")
    r = O.residuals(P, theta, np.arange(P.N))[0]
    assert np.abs(r).min() > 1e-4
    assert abs(info["loglik"] + np.abs(r).sum()) < 1e-9 * np.abs(r).sum()
    gf = np.zeros_like(theta)
    h = (1e-6, 1e-6, 1e-6, 1e-7)
    for m in range(P.M):
        for a in range(4):
            tp, tm = theta.copy(), theta.copy()
            tp[m, a] += h[a]; tm[m, a] -= h[a]
            gf[m, a] = (O.log_posterior(P, tp, loss="l1")[0] - O.log_posterior(P, tm, loss="l1")[0]) / (2 * h[a])
    assert np.linalg.norm(g - gf) <= 1e-5 * np.linalg.norm(g)


def test_adam_constant_gradient_closed_form():
    # R11 with a constant gradient g: the bias-corrected moments are exactly g
    # and g^2, so every step moves eta g / (|g| + eps_p)
    g = np.array([[0.3, -2.0, 1e-3, 5.0]])
    theta = np.zeros((1, 4)); m = np.zeros((1, 4)); v = np.zeros((1, 4))
    eta, eps_p = 1e-3, 1e-5
    for t in range(1, 41):
        theta, m, v = O.adam_update(theta, g, m, v, t, eta, 0.9, 0.99, eps_p)
    assert np.allclose(theta, 40 * eta * g / (np.abs(g) + eps_p), rtol=1e-12, atol=0)


def test_adam_finds_the_map_of_a_gaussian():
    # prior-only catalog (no observations): the log posterior is maximal at theta_0
    P = tiny_problem(M=6, S=2, K=2, seed=22)
    theta = P.init + 0.3
    m = np.zeros_like(theta); v = np.zeros_like(theta)
    for t in range(1, 3001):
        g = -(theta - P.init) / P.sig_e ** 2
        theta, m, v = O.adam_update(theta, g, m, v, t, 1e-2, 0.9, 0.99, 1e-8)
    assert np.abs(theta - P.init).max() < 1e-3


def test_psgld_constant_preconditioner_stationary_law():
    # R10: with v frozen at c (the beta2 -> 1 limit) pSGLD is SGLD with step
    # eps V, V = 1 / (sqrt(c) + eps_p): stationary law N(mu, 1 / (h (1 - eps V h / 2)))
    h, mu, eps, c, eps_p = 4.0, -0.7, 0.05, 0.25, 1e-5
    V = 1.0 / (np.sqrt(c) + eps_p)
    C = 25_000
    theta = np.full((C, 4), mu)
    v = np.full((C, 4), c)
    acc, acc2, n = 0.0, 0.0, 0
    for t in range(1200):
        g = -h * (theta - mu)
        theta, v = O.psgld_update(theta, g, v, eps, 1.0, eps_p, O.langevin_noise(C, seed=5000 + t))
        if t >= 200:
            acc += theta.sum(); acc2 += (theta * theta).sum(); n += theta.size
    mean = acc / n
    var = acc2 / n - mean * mean
    exact = 1.0 / (h * (1.0 - eps * V * h / 2.0))
    assert abs(mean - mu) < 0.005
    assert abs(var / exact - 1.0) < 0.01, (var, exact)


def test_psgld_first_step_closed_form():
    # from v = 0 the first update uses v = (1 - beta2) g^2
    g = np.array([[1.0, -4.0, 0.5, 2.0]])
    eta = np.array([[0.1, 0.2, -0.3, 0.4]])
    eps, b2, eps_p = 1e-3, 0.99, 1e-5
    th, v = O.psgld_update(np.zeros((1, 4)), g, np.zeros((1, 4)), eps, b2, eps_p, eta)
    V = 1.0 / (np.sqrt(1 - b2) * np.abs(g) + eps_p)
    assert np.allclose(th, eps * V * g + np.sqrt(2 * eps * V) * eta, rtol=1e-14, atol=0)
    assert np.allclose(v, (1 - b2) * g * g, rtol=1e-15, atol=0)


def test_mad_filter_small_cases_by_hand():
    keep, med, mad = O.mad_filter([3.0, 1.0, 2.0])
    assert med == 2.0 and mad == 1.0 and keep.all()
    # even count: median 2.5; deviations 1.5, 0.5, 0.5, 7.5 -> MAD 1.0; 10 lies 7.5 > 4 away
    keep, med, mad = O.mad_filter([1.0, 2.0, 3.0, 10.0])
    assert med == 2.5 and mad == 1.0 and keep.tolist() == [True, True, True, False]


def test_mad_of_laplace_and_normal_samples():
    rng = np.random.default_rng(30)
    b, sd = 0.005, 0.005
    _, med, mad = O.mad_filter(rng.laplace(0.0, b, 2_000_000))
    assert abs(med) < 2e-5 and abs(mad / (b * np.log(2.0)) - 1.0) < 0.01      # Laplace MAD = b ln 2
    _, med, mad = O.mad_filter(rng.normal(0.0, sd, 2_000_000))
    assert abs(mad / (sd * 0.6744897501960817) - 1.0) < 0.01                    # normal MAD = 0.6745 sigma


def test_mad_filter_rejects_gross_outliers():
    rng = np.random.default_rng(31)
    n = 500_000
    r = rng.laplace(0.0, 0.005, n)
    out = rng.random(n) < 0.02
    r[out] = rng.uniform(-0.5, 0.5, out.sum())
    keep, med, mad = O.mad_filter(r)
    gross = out & (np.abs(r) > 0.05)
    assert (~keep[gross]).mean() > 0.999
    # Laplace inliers beyond the cut: P(|x - med| > 4 MAD) = exp(-4 MAD / b)
    assert abs((~keep[~out]).mean() - np.exp(-4.0 * mad / 0.005)) < 0.003


def test_linearisation_error_closed_forms():
    # homogeneous medium, c = 6 km/s, station at the origin, event i at distance r
    c = 6.0
    model = O.Model("homogeneous", v0=c)
    st = np.zeros((1, 3))
    xi = np.array([3.0, 4.0, 12.0])                 # r = 13
    n = xi / np.linalg.norm(xi)
    perp = np.cross(n, [0.0, 0.0, 1.0]); perp /= np.linalg.norm(perp)
    cases = [xi + 0.8 * n, xi + 0.8 * perp, xi + np.array([0.01, -0.02, 0.015])]
    init = np.vstack([np.r_[xi, 0.0]] + [np.r_[x, 0.0] for x in cases])
    P = O.Problem(init, st, np.zeros(3, int), np.arange(1, 4), np.zeros(3, int), np.zeros(3), model,
                  0.01, 0.0, 0.25, 40.0, 1e-5, np.ones(4), np.ones(4))
    keep, rel = O.linearisation_filter(P, init, 0.05)
    r = np.linalg.norm(xi)
    # along the ray the travel time is linear: no error
    assert rel[0] < 1e-12 and keep[0]
    # across the ray dT = (sqrt(r^2 + d^2) - r) / c and the linear term vanishes: error 100 %
    assert abs(rel[1] - 1.0) < 1e-9 and not keep[1]
    # small generic offsets: the error is the Hessian term 1/2 dx^T (I - n n^T) dx / (c r) + O(dx^3)
    dx = cases[2] - xi
    H = (np.eye(3) - np.outer(n, n)) / (c * r)
    dT = (np.linalg.norm(cases[2]) - r) / c
    assert abs(rel[2] * abs(dT) - 0.5 * dx @ H @ dx) < 1e-3 * 0.5 * dx @ H @ dx + 1e-12


def test_percentiles_and_halfwidth_by_hand():
    # 4 samples 1, 2, 3, 4 (one event, one coordinate): ranks (n - 1) p / 100
    s = np.zeros((4, 1, 4)); s[:, 0, 0] = [4.0, 1.0, 3.0, 2.0]
    med, half, _, _ = O.uq_stats(s, lo_pct=0.5, hi_pct=99.5)
    assert med[0, 0] == 2.5
    lo, hi = 1.0 + 0.015, 4.0 - 0.015                    # ranks 0.015 and 2.985
    assert abs(half[0, 0] - 0.5 * (hi - lo)) < 1e-12


def test_ess_of_ar1_chains():
    # AR(1) x_t = phi x_{t-1} + e_t has integrated time (1 + phi) / (1 - phi)
    rng = np.random.default_rng(40)
    n = 40_000
    for phi in (0.0, 0.5, 0.8):
        e = rng.normal(size=n)
        x = np.empty(n); x[0] = e[0] / np.sqrt(1 - phi * phi)
        for t in range(1, n):
            x[t] = phi * x[t - 1] + e[t]
        want = n * (1 - phi) / (1 + phi)
        assert abs(O.ess_series(x) / want - 1.0) < 0.1, (phi, O.ess_series(x), want)


def test_calibration_of_an_exact_posterior_is_uniform():
    # truth and samples drawn from the same law: the calibration values are uniform
    rng = np.random.default_rng(41)
    M, n = 1000, 100
    mu = rng.normal(size=(M, 4))
    truth = mu + rng.normal(size=(M, 4))
    samples = mu[None] + rng.normal(size=(n, M, 4))
    _, _, calib, ess = O.uq_stats(samples, truth)
    c = calib.ravel()
    assert abs(c.mean() - 0.5) < 0.01 and abs(c.var() - 1 / 12) < 0.005
    # independent draws: ESS close to n
    assert abs(np.median(ess) / n - 1.0) < 0.15


# ---------------------------------------------------------------- small helpers
def test_box_muller_polar_form():
    """z0 = R cos(2 pi u2), z1 = R sin(2 pi u2) with R^2 = -2 ln u1: the radius
    and the angle of each pair recovered from the words (a swapped sine and
    cosine or a dropped factor fails)."""
    rng = np.random.default_rng(7)
    wa = rng.integers(0, 2 ** 32, 1000, dtype=np.uint64)
    wb = rng.integers(0, 2 ** 32, 1000, dtype=np.uint64)
    z0, z1 = O.box_muller(wa, wb)
    u1, u2 = O.unit_from_word(wa), O.unit_from_word(wb)
    assert np.allclose(z0 * z0 + z1 * z1, -2.0 * np.log(u1), rtol=1e-12, atol=1e-15)
    ang = np.mod(np.arctan2(z1, z0), 2 * math.pi)
    d = np.abs(ang - 2 * math.pi * u2)
    assert np.all(np.minimum(d, 2 * math.pi - d) < 1e-9)
    # the smallest first word gives the largest radius, sqrt(-2 ln 2^-24)
    z0, z1 = O.box_muller(np.array([0], np.uint64), np.array([0], np.uint64))
    assert math.isclose(math.hypot(z0[0], z1[0]), math.sqrt(48 * math.log(2)), rel_tol=1e-12)


def test_seed_key_splits_the_64_bit_seed():
    for s in (0, 1, 0xFFFFFFFF, 0x100000000, 0xDEADBEEFCAFEF00D):
        lo, hi = O.seed_key(s)
        assert 0 <= lo < 2 ** 32 and 0 <= hi < 2 ** 32 and lo + (hi << 32) == s
    assert O.seed_key(-1) == (0xFFFFFFFF, 0xFFFFFFFF)      # two's complement wrap


def test_minibatch_obs_is_the_union_of_the_blocks():
    """Brute force: block b holds canonical positions [b B, (b + 1) B), the last
    block ragged; the minibatch is exactly the observations at those positions."""
    rng = np.random.default_rng(3)
    N, B = 23, 5
    order = rng.permutation(N)
    for blocks in ([4], [0, 2], [3, 1, 4], list(range(5)), []):
        got = O.minibatch_obs(order, B, np.array(blocks, np.int64))
        want = [int(order[p]) for p in range(N) if p // B in blocks]
        assert sorted(got.tolist()) == sorted(want)
    assert O.minibatch_obs(order, B, np.array([4])).size == 3


def test_pair_table_and_homogeneous_travel_times_by_brute_force():
    """Every observation's two nodes are its (event, station) pairs, each pair
    met once, and T of a node is |x - s| / v0 for its own event and station."""
    P = tiny_problem(M=9, S=3, K=3, seed=5)
    sel = np.arange(0, P.N, 2)
    ni, nj, nev, nst, T, dT = O.travel_times(P, P.init, sel)
    pairs = {(int(P.i[o]), int(P.k[o])) for o in sel} | {(int(P.j[o]), int(P.k[o])) for o in sel}
    assert len(nev) == len(pairs) and set(zip(nev.tolist(), nst.tolist())) == pairs
    for a, o in enumerate(sel):
        assert (nev[ni[a]], nst[ni[a]]) == (P.i[o], P.k[o])
        assert (nev[nj[a]], nst[nj[a]]) == (P.j[o], P.k[o])
    for n in range(len(nev)):
        d = P.init[nev[n], :3] - P.stations[nst[n]]
        assert math.isclose(T[n], math.sqrt(float(d @ d)) / 6.0, rel_tol=1e-14)


def test_grad_norms_by_hand():
    g = np.array([[1.0, 2.0, 2.0, 4.0], [0.0, 0.0, 0.0, 0.0], [3.0, 0.0, 4.0, 0.0], [-6.0, 0, 0, 8.0]])
    assert O.grad_norms(g).tolist() == [5.0, 0.0, 5.0, 10.0]
