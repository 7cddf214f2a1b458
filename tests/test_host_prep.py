"""The library's host preparation (canonical order, pair table, minibatch
blocks, half-edge lists, pair -> block incidence, weights, reduced dd times)
checked on the CPU against the oracle's orderings and against structural
invariants, through a test-only harness compiled from the library source."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from oracle import spider_oracle as O
from paper_2508_12117_gb300 import binding, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2508_12117_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("prep")
    so = str(d / "prep_harness.so")
    cmd = ["g++", "-O2", "-fPIC", "-shared", "-std=c++17", "-pthread", "-ffp-contract=off",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           os.path.join(ROOT, "tests", "host", "prep_harness.cpp"), os.path.join(CSRC, "prep.cpp"),
           os.path.join(CSRC, "pieces.cpp"), "-o", so]
    subprocess.run(cmd, check=True, capture_output=True)
    L = C.CDLL(so)
    L.prep_run.restype = C.c_int
    L.prep_get.restype = C.c_int
    L.prep_error.restype = C.c_char_p
    L.pieces_run.restype = C.c_int
    L.pieces_run.argtypes = [C.c_int, C.c_double, C.c_void_p]
    L.pieces_get.restype = C.c_int
    return L


def run_prep(L, cat, **cfg_over):
    a = dict(x=np.ascontiguousarray(cat.init_xyzt), i=np.ascontiguousarray(cat.i, np.int32),
             j=np.ascontiguousarray(cat.j, np.int32), k=np.ascontiguousarray(cat.k, np.int32),
             dt=np.ascontiguousarray(cat.dt), s=np.ascontiguousarray(cat.stations))
    ccat = binding.spider_catalog(cat.M, cat.N, binding._ptr(a["x"], C.c_double),
                                  binding._ptr(a["i"], C.c_int32), binding._ptr(a["j"], C.c_int32),
                                  binding._ptr(a["k"], C.c_int32), binding._ptr(a["dt"], C.c_double), None)
    sta = binding.spider_stations(cat.S, binding._ptr(a["s"], C.c_double))
    cfg = binding.spider_config()
    # defaults written here (the product library is not needed for this test)
    cfg.sigma, cfg.kappa, cfg.p, cfg.ell, cfg.eps_w = 0.01, 0.03, 0.25, 40.0, 1e-5
    for q in range(4):
        cfg.sig_e[q] = 0.5
        cfg.sig_c[q] = 0.01
    cfg.block_obs, cfg.reorder, cfg.thin = 4096, 1, 1
    for key, val in cfg_over.items():
        setattr(cfg, key, val)
    sizes = np.zeros(8, np.int64)
    rc = L.prep_run(C.byref(ccat), C.byref(sta), C.byref(cfg), binding._ptr(sizes, C.c_int64))
    if rc:
        return rc, L.prep_error().decode(), None
    M, N, S, B, NB, P, Q, Lmax = (int(x) for x in sizes)
    spec = dict(ev_old=(M, np.int32), ord=(N, np.int32), pair_off=(M + 1, np.int32),
                pair_st=(P, np.int32), pair_ev=(P, np.int32), obs_l=(N, np.uint32),
                obs_dt=(N, np.float32), obs_sw=(N, np.float32), blk_node_off=(NB + 1, np.int32),
                node_pair=(Q, np.int32), node_he=(Q, np.uint16), blk_he=(2 * N, np.uint16),
                inc_off=(P + 1, np.int32), inc_q=(Q, np.int32), inc_b=(Q, np.int32))
    out = dict(M=M, N=N, S=S, B=B, NB=NB, P=P, Q=Q, L_max=Lmax)
    for name, (n, dt) in spec.items():
        arr = np.empty(max(n, 1), dt)
        assert L.prep_get(name.encode(), arr.ctypes.data_as(C.c_void_p)) == 0
        out[name] = arr[:n]
    return 0, "", out


def check_structure(cat, R, reorder=True):
    M, N, B, NB = R["M"], R["N"], R["B"], R["NB"]
    ev, order = O.canonical_order(cat.init_xyzt, cat.i, cat.j, cat.k, reorder)
    assert np.array_equal(R["ev_old"], ev)                      # Morton renumbering
    assert np.array_equal(R["ord"], order)                      # canonical obs order
    rank = np.empty(M, np.int64); rank[ev] = np.arange(M)
    ia, ja, ka = rank[cat.i[order]], rank[cat.j[order]], cat.k[order]
    # reduced dd times and weights
    t0 = cat.init_xyzt[:, 3]
    dtt = (cat.dt[order] - (t0[cat.i[order]] - t0[cat.j[order]])).astype(np.float32)
    assert np.array_equal(R["obs_dt"], dtt)
    w = O.edge_weights(cat.init_xyzt, cat.i, cat.j, cat.k, cat.S, 40.0, 0.25, 1e-5)[order]
    assert np.allclose(R["obs_sw"].astype(np.float64) ** 2, w, rtol=1e-6)
    # pair table: sorted (event, station) set of all observation ends
    pairs = np.unique(np.r_[ia * cat.S + ka, ja * cat.S + ka])
    assert R["P"] == pairs.size
    assert np.array_equal(R["pair_ev"].astype(np.int64) * cat.S + R["pair_st"], pairs)
    assert np.array_equal(np.bincount(R["pair_ev"], minlength=M), np.diff(R["pair_off"]))
    pid = {int(x): n for n, x in enumerate(pairs)}
    # blocks
    bno = R["blk_node_off"]
    assert bno[0] == 0 and np.all(np.diff(bno) >= 0) and bno[-1] == R["Q"]
    assert R["L_max"] == np.diff(bno).max() and R["L_max"] <= 2 * B
    for b in range(NB):
        e0, e1 = b * B, min(N, (b + 1) * B)
        q0, q1 = bno[b], bno[b + 1]
        nodes = R["node_pair"][q0:q1]
        assert np.all(np.diff(nodes) > 0)                        # sorted, unique
        li = R["obs_l"][e0:e1] & 0xFFFF
        lj = R["obs_l"][e0:e1] >> 16
        assert li.max() < q1 - q0 and lj.max() < q1 - q0
        pi = np.array([pid[int(x)] for x in ia[e0:e1] * cat.S + ka[e0:e1]])
        pj = np.array([pid[int(x)] for x in ja[e0:e1] * cat.S + ka[e0:e1]])
        assert np.array_equal(nodes[li], pi) and np.array_equal(nodes[lj], pj)
        assert set(nodes.tolist()) == set(pi.tolist()) | set(pj.tolist())
        he = R["blk_he"][2 * e0: 2 * e1]
        assert sorted(he.tolist()) == list(range(2 * (e1 - e0)))  # every half-edge once
        beg = R["node_he"][q0:q1].astype(np.int64)
        end = np.r_[beg[1:], 2 * (e1 - e0)]
        assert np.all(end >= beg)
        for l in range(q1 - q0):
            for code in he[beg[l]:end[l]]:
                e, side = code >> 1, code & 1
                assert (lj[e] if side else li[e]) == l
            assert np.all(np.diff(he[beg[l]:end[l]]) > 0)        # observation order
    # incidence: occurrences of each pair, block-ascending
    io = R["inc_off"]
    for p in range(R["P"]):
        qs = R["inc_q"][io[p]:io[p + 1]]
        bs = R["inc_b"][io[p]:io[p + 1]]
        assert np.all(np.diff(bs) > 0)
        for q, b in zip(qs, bs):
            assert bno[b] <= q < bno[b + 1] and R["node_pair"][q] == p
    assert io[-1] == R["Q"]


def test_prep_tiny_catalog(harness):
    cat = synth.make_catalog(1)
    rc, msg, R = run_prep(harness, cat)
    assert rc == 0, msg
    check_structure(cat, R)


def test_prep_shuffled_ragged_blocks(harness):
    cat = synth.shuffled_events(synth.make_catalog(1), seed=4)
    rc, msg, R = run_prep(harness, cat, block_obs=333)
    assert rc == 0, msg
    assert R["NB"] == -(-cat.N // 333)
    check_structure(cat, R)


def test_prep_no_reorder(harness):
    cat = synth.shuffled_events(synth.make_catalog(1), seed=5)
    rc, msg, R = run_prep(harness, cat, block_obs=1000, reorder=0)
    assert rc == 0, msg
    check_structure(cat, R, reorder=False)


def test_prep_fault_catalog_small_blocks(harness):
    s = synth.scaled_spec(2, 1500, n_faults=2, region_km=10.0)
    cat = synth.make_catalog(s)
    rc, msg, R = run_prep(harness, cat, block_obs=2048)
    assert rc == 0, msg
    check_structure(cat, R)


def test_prep_rejects_bad_input(harness):
    cat = synth.make_catalog(1)
    bad = synth.Catalog(cat.spec, cat.true_xyzt, cat.init_xyzt, cat.stations, cat.i.copy(),
                        cat.j.copy(), cat.k.copy(), cat.dt.copy())
    bad.j[10] = bad.i[10]
    rc, msg, _ = run_prep(harness, bad)
    assert rc == -1 and "i == j" in msg
    bad = synth.Catalog(cat.spec, cat.true_xyzt, cat.init_xyzt, cat.stations, cat.i.copy(),
                        cat.j.copy(), cat.k.copy(), cat.dt.copy())
    bad.dt[3] = np.nan
    assert run_prep(harness, bad)[0] == -1
    rc, msg, _ = run_prep(harness, cat, block_obs=0)
    assert rc == -1


def _pieces(L, R, lam, max_n=512):
    sizes = np.zeros(3, np.int64)
    assert L.pieces_run(max_n, lam, sizes.ctypes.data_as(C.c_void_p)) == 0
    G, _, ninv = (int(x) for x in sizes)
    spec = dict(blk_piece_off=(R["NB"] + 1, np.int32), node_piece=(R["Q"], np.uint16),
                node_ppos=(R["Q"], np.uint16), piece_node_off=(G + 1, np.int32),
                piece_nodes=(R["Q"], np.uint16), piece_inv_off=(G + 1, np.int64), inv=(ninv, np.float32),
                mem_rp=(R["Q"] + 1, np.int32), edge_pos=(2 * R["N"], np.uint16), edge_sw=(2 * R["N"], np.float32))
    out = dict(G=G)
    for name, (n, dt) in spec.items():
        arr = np.empty(max(n, 1), dt)
        assert L.pieces_get(name.encode(), arr.ctypes.data_as(C.c_void_p)) == 0
        out[name] = arr[:n]
    return out


@pytest.mark.parametrize("block_obs", [4096, 700])
def test_pieces_are_block_components_with_exact_inverses(harness, block_obs):
    """Pieces are exactly the connected components of each block's local graph
    (scipy), numbered by smallest member, and each stored inverse is
    (lambda I + B^T B)^-1 of its piece, built here element by element from the
    block's observations and inverted by numpy, to FP32 rounding."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    s = synth.scaled_spec(2, 1500, n_faults=2, region_km=10.0)
    cat = synth.make_catalog(s)
    rc, msg, R = run_prep(harness, cat, block_obs=block_obs)
    assert rc == 0, msg
    lam = 0.005 ** 2 / 0.03 ** 2
    T = _pieces(harness, R, lam)
    bno, bpo = R["blk_node_off"], T["blk_piece_off"]
    assert bpo[-1] == T["G"] and T["piece_node_off"][-1] == R["Q"]
    w = R["obs_sw"].astype(np.float64) ** 2
    worst = 0.0
    for b in range(R["NB"]):
        e0, e1 = b * R["B"], min(R["N"], (b + 1) * R["B"])
        q0, q1 = bno[b], bno[b + 1]
        L_ = q1 - q0
        li = (R["obs_l"][e0:e1] & 0xFFFF).astype(np.int64)
        lj = (R["obs_l"][e0:e1] >> 16).astype(np.int64)
        nc, lab = connected_components(coo_matrix((np.ones(e1 - e0), (li, lj)), shape=(L_, L_)),
                                       directed=False)
        assert bpo[b + 1] - bpo[b] == nc
        # numbering by smallest member: relabel scipy's labels in order of first occurrence
        first = {}
        for l in range(L_):
            first.setdefault(int(lab[l]), len(first))
        want_piece = np.array([first[int(x)] for x in lab])
        assert np.array_equal(T["node_piece"][q0:q1], want_piece)
        for c in range(nc):
            g = bpo[b] + c
            mem = T["piece_nodes"][T["piece_node_off"][g]:T["piece_node_off"][g + 1]].astype(np.int64)
            assert np.array_equal(mem, np.nonzero(want_piece == c)[0])
            assert np.array_equal(T["node_ppos"][q0 + mem], np.arange(mem.size))
            # member edge lists: (other end's position, sqrt w) per half-edge,
            # the same multiset as the block's observations touching the member
            for i, l in enumerate(mem):
                m_ = T["piece_node_off"][g] + i
                ent = sorted(zip(T["edge_pos"][T["mem_rp"][m_]:T["mem_rp"][m_ + 1]].tolist(),
                                 T["edge_sw"][T["mem_rp"][m_]:T["mem_rp"][m_ + 1]].tolist()))
                want_ent = []
                for e in np.nonzero((li == l) | (lj == l))[0]:
                    other = lj[e] if li[e] == l else li[e]
                    want_ent.append((int(np.nonzero(mem == other)[0][0]), float(R["obs_sw"][e0 + e])))
                assert ent == sorted(want_ent)
            if b % 7 and c % 3:            # a sample of the inverses
                continue
            n = mem.size
            pos = {int(x): i for i, x in enumerate(mem)}
            K = lam * np.eye(n)
            for e in np.nonzero(want_piece[li] == c)[0]:
                i, j = pos[int(li[e])], pos[int(lj[e])]
                K[i, i] += w[e0 + e]; K[j, j] += w[e0 + e]; K[i, j] -= w[e0 + e]; K[j, i] -= w[e0 + e]
            want = np.linalg.inv(K)
            pk = T["inv"][T["piece_inv_off"][g]:T["piece_inv_off"][g + 1]].astype(np.float64)
            got = pk.reshape(n, n)
            assert np.array_equal(got, got.T)
            worst = max(worst, float(np.abs(got - want).max() / np.abs(want).max()))
    assert worst <= 2e-7, worst
