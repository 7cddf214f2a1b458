"""The bounded device-side waits give up, report SPIDER_E_TIMEOUT and leave the
context usable, without any GPU fault.

spider_set_wait_limit_ns(ctx, 0) makes every CTA that finds a grid-wide
barrier incomplete give up at once, so the cooperative component labelling
(k_cc) times out at its first barrier on any grid of two or more CTAs; the
kernels after it see the recorded error and return without work.  Restoring
the limit, the context must step exactly like a fresh one."""
import numpy as np
import pytest

from paper_2508_12117_gb300 import binding, synth

pytestmark = pytest.mark.gpu

SPIDER_E_TIMEOUT = -5


@pytest.fixture(scope="module")
def cat1():
    return synth.make_catalog(1)


def test_zero_wait_limit_times_out_and_the_context_recovers(cat1):
    eps = cat1.spec.hyper.eps
    a = binding.Context.from_catalog(cat1)
    ref = binding.Context.from_catalog(cat1)
    th0, _ = a.spider_get_state()
    a.spider_set_wait_limit_ns(0)
    # an SGLD step (captured graph): the step gives up, theta stays where it was
    a.spider_sgld_step(eps, 5)
    with pytest.raises(binding.SpiderError) as e:
        a.spider_sync()
    assert e.value.code == SPIDER_E_TIMEOUT
    th1, _ = a.spider_get_state()
    assert np.array_equal(th1, th0)
    # the gradient call reports the same status
    with pytest.raises(binding.SpiderError) as e:
        a.spider_grad_logpost(0)
    assert e.value.code == SPIDER_E_TIMEOUT
    # with the limit still 0 every step gives up; two queued steps report once
    a.spider_sgld_step(eps, 6)
    a.spider_sgld_step(eps, 7)
    with pytest.raises(binding.SpiderError) as e:
        a.spider_sync()
    assert e.value.code == SPIDER_E_TIMEOUT
    # back to the default limit: the same chain as a context that never timed out
    a.spider_set_wait_limit_ns(2_000_000_000)
    a.spider_set_state(th0, 0)
    for s in (11, 12, 13):
        a.spider_sgld_step(eps, s)
        ref.spider_sgld_step(eps, s)
    ta, sa = a.spider_get_state()
    tr, sr = ref.spider_get_state()
    assert sa == sr == 3
    assert np.array_equal(ta, tr)
    ga, la = a.spider_grad_logpost(0)
    gr, lr = ref.spider_grad_logpost(0)
    assert np.array_equal(ga, gr) and la == lr
    a.close()
    ref.close()


def test_wait_limit_is_validated(cat1):
    a = binding.Context.from_catalog(cat1)
    with pytest.raises(binding.SpiderError):
        a.spider_set_wait_limit_ns(601 * 10 ** 9)
    a.close()


def test_zero_wait_limit_in_a_piece_path_step():
    """The same on a minibatch step whitened through the piece inverses: the
    cooperative piece labelling (k_piece_cc) gives up at its first grid barrier,
    the unit, clean-piece and scatter kernels see the error and return, the
    state stays where it was, and after the limit is restored the chain is the
    one a fresh context walks."""
    cat = synth.make_catalog(2)
    bn = 1 << 14
    eps = synth._eps_for(0.03, 10, cat.N / bn)
    a = binding.Context.from_catalog(cat, batch_n=bn)
    ref = binding.Context.from_catalog(cat, batch_n=bn)
    assert a.spider_info()["piece_whitening"] == 1
    th0, _ = a.spider_get_state()
    a.spider_set_wait_limit_ns(0)
    a.spider_sgld_step(eps, 5)
    with pytest.raises(binding.SpiderError) as e:
        a.spider_sync()
    assert e.value.code == SPIDER_E_TIMEOUT
    th1, _ = a.spider_get_state()
    assert np.array_equal(th1, th0)
    a.spider_set_wait_limit_ns(2_000_000_000)
    a.spider_set_state(th0, 0)
    for s in (21, 22, 23):
        a.spider_sgld_step(eps, s)
        ref.spider_sgld_step(eps, s)
    ta, _ = a.spider_get_state()
    tr, _ = ref.spider_get_state()
    assert np.array_equal(ta, tr)
    a.close()
    ref.close()
