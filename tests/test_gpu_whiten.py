"""Whitening of minibatch steps through the precomputed inverses of the
block-local components (row a5, Eq. marginal_sigma), against the FP64 oracle
and against the general component solver.

A minibatch step solves every piece whose nodes occur in no other selected
block with its stored inverse, and every unit of pieces that share nodes by
the Schur complement on the shared nodes; units beyond the limits of that path
hand the whole step to the general solver.  Tolerances are the FP32 ones:
gradient rel-L2 <= 1e-5, q = Sigma^-1 r rel-L2 <= 1e-5."""
import numpy as np
import pytest

from oracle import spider_oracle as O
from paper_2508_12117_gb300 import binding, synth

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-5


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def cat2():
    return synth.make_catalog(2)


def _check_against_oracle(ctx, P, cat, seed):
    g, lp = ctx.spider_grad_logpost(seed)
    info = ctx.spider_info()
    sel = P.batch(seed)
    L, go, oinfo = O.log_posterior(P, cat.init_xyzt, sel)
    idx, r, q = ctx.spider_debug_obs(P.N)
    pos = np.searchsorted(sel, idx)
    assert np.array_equal(sel[pos], idx)
    rel_g, rel_q = rel_l2(g, go), rel_l2(q, oinfo["q"][pos])
    return rel_g, rel_q, abs(lp - L) / abs(L), info


@pytest.mark.parametrize("bn,seeds,shared", [(1 << 14, (3, 4), False), (1 << 17, (5, 6), True)])
def test_piece_whitening_matches_oracle(cat2, bn, seeds, shared):
    """4 of 489 blocks rarely share a pair (single pieces only); 32 blocks do
    (units solved through the Schur complement)."""
    ctx = binding.Context.from_catalog(cat2, batch_n=bn)
    P = O.problem_from_catalog(cat2, batch_n=bn)
    for seed in seeds:
        rel_g, rel_q, rel_lp, info = _check_against_oracle(ctx, P, cat2, seed)
        print(f"n = {bn}, seed {seed}: gradient rel-L2 {rel_g:.2e}, q rel-L2 {rel_q:.2e}, logpost rel "
              f"{rel_lp:.1e}; units {info['units']}, fallback {info['fallback']}")
        assert info["piece_inverses"] == 1 and info["piece_whitening"] == 1
        assert info["fallback"] == 0 and (info["units"] > 0 or not shared)
        assert rel_g <= GRAD_TOL and rel_q <= GRAD_TOL and rel_lp <= 1e-5
    ctx.close()


def test_piece_whitening_agrees_with_general_solver(cat2):
    bn = 1 << 15
    a = binding.Context.from_catalog(cat2, batch_n=bn)
    b = binding.Context.from_catalog(cat2, batch_n=bn)
    b.spider_set_tuning([2, 1, 2, 0])          # general component solver only
    for seed in (11, 12):
        ga, la = a.spider_grad_logpost(seed)
        gb, lb = b.spider_grad_logpost(seed)
        _, _, qa = a.spider_debug_obs(cat2.N)
        _, _, qb = b.spider_debug_obs(cat2.N)
        print(f"seed {seed}: gradient rel diff {rel_l2(ga, gb):.2e}, q rel diff {rel_l2(qa, qb):.2e}")
        assert a.spider_info()["fallback"] == 0
        assert rel_l2(ga, gb) <= 2e-6 and rel_l2(qa, qb) <= 2e-6
        assert abs(la - lb) <= 1e-6 * abs(lb)
    a.close()
    b.close()


def test_large_units_fall_back_to_the_general_solver(cat2):
    """Half of the blocks per step: the shared nodes join pieces into units far
    beyond the direct path's limits, the step falls back, and the result is
    still the oracle's."""
    bn = cat2.N // 2
    ctx = binding.Context.from_catalog(cat2, batch_n=bn)
    P = O.problem_from_catalog(cat2, batch_n=bn)
    rel_g, rel_q, _, info = _check_against_oracle(ctx, P, cat2, 21)
    print(f"n = N/2: gradient rel-L2 {rel_g:.2e}, q rel-L2 {rel_q:.2e}, fallback {info['fallback']}")
    assert info["fallback"] == 1
    assert rel_g <= GRAD_TOL and rel_q <= GRAD_TOL
    ctx.close()


def test_piece_whitening_step_is_reproducible(cat2):
    bn = 1 << 14
    eps = synth._eps_for(0.03, 10, cat2.N / bn)
    a = binding.Context.from_catalog(cat2, batch_n=bn)
    b = binding.Context.from_catalog(cat2, batch_n=bn)
    for s in range(5):
        a.spider_sgld_step(eps, 700 + s)
        b.spider_sgld_step(eps, 700 + s)
    ta, _ = a.spider_get_state()
    tb, _ = b.spider_get_state()
    assert np.array_equal(ta, tb)
    a.close()
    b.close()


def test_dense_catalog_units_stay_on_the_data_parallel_path():
    """A catalog drawn with the 100k-event recipe (about 1000 dd observations
    per event, so a pair recurs in ~9 blocks): at 2.6 % of the blocks per step,
    pieces carry up to ~90 shared nodes and units up to ~190.  Every unit is
    solved by the data-parallel Schur path (no hand-over, no fallback) and the
    step matches the oracle."""
    s = synth.scaled_spec(3, 20000, batch_n=1 << 18)
    cat = synth.make_catalog(s)
    ctx = binding.Context.from_catalog(cat)
    P = O.problem_from_catalog(cat)
    for seed in (1, 2, 3):
        rel_g, rel_q, rel_lp, info = _check_against_oracle(ctx, P, cat, seed)
        handed = sum(v for k, v in info.items() if k.startswith("handover_"))
        print(f"seed {seed}: gradient rel-L2 {rel_g:.2e}, q rel-L2 {rel_q:.2e}; units {info['units']}, "
              f"handed over {handed}, fallback {info['fallback']}")
        assert info["fallback"] == 0 and handed == 0 and info["units"] > 0
        assert rel_g <= GRAD_TOL and rel_q <= GRAD_TOL and rel_lp <= 1e-5
    ctx.close()


def test_concurrent_unit_setup_equals_the_serial_order():
    """The size classes of the units' small inverses run side by side on branch
    streams (knob 6 = 1, the default) or one after the other (0): the classes
    take disjoint pieces and units, so gradients and SGLD chains (graph steps)
    are bit-identical.  The dense catalog puts units in every class, up to ~190
    shared nodes."""
    s = synth.scaled_spec(3, 20000, batch_n=1 << 18)
    cat = synth.make_catalog(s)
    a = binding.Context.from_catalog(cat)
    b = binding.Context.from_catalog(cat)
    b.spider_set_tuning([2, 1, 2, 1, 2, 2, 0])
    for seed in (1, 4):
        ga, la = a.spider_grad_logpost(seed)
        gb, lb = b.spider_grad_logpost(seed)
        ia, ib = a.spider_info(), b.spider_info()
        print(f"seed {seed}: units {ia['units']}, fallback {ia['fallback']} / {ib['fallback']}")
        assert ia["units"] > 0 and ia["fallback"] == ib["fallback"]
        assert np.array_equal(ga, gb) and la == lb
    eps = s.hyper.eps
    for k in range(4):
        a.spider_sgld_step(eps, 40 + k)
        b.spider_sgld_step(eps, 40 + k)
    assert a.spider_info()["graph"] == 1 and b.spider_info()["graph"] == 1
    ta, _ = a.spider_get_state()
    tb, _ = b.spider_get_state()
    assert np.array_equal(ta, tb) and np.isfinite(ta).all()
    a.close()
    b.close()
